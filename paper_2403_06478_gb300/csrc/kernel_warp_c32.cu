// Instantiation of the warp kernel and its traceback variant for 32 band slots per lane (w <= 1023).
#include "kernel_tb.cuh"

namespace agatha {
template cudaError_t launch_warp_c<32>(const DevBatch *, int, cudaStream_t, int, int);
template int occupancy_warp_c<32>();
template cudaError_t launch_tb_c<32>(const DevBatch *, const TbItem *, int32_t, int32_t *, uint8_t *,
                                    uint32_t *, int32_t *, int, cudaStream_t);
template int occupancy_tb_c<32>();
}  // namespace agatha
