// Instantiation of the warp kernel and its traceback variant for 8 band slots per lane (w <= 255).
#include "kernel_tb.cuh"

namespace agatha {
template cudaError_t launch_warp_c<8>(const DevBatch *, int, cudaStream_t, int, int);
template int occupancy_warp_c<8>();
template cudaError_t launch_tb_c<8>(const DevBatch *, const TbItem *, int32_t, int32_t *, uint8_t *,
                                    uint32_t *, int32_t *, int, cudaStream_t);
template int occupancy_tb_c<8>();
}  // namespace agatha
