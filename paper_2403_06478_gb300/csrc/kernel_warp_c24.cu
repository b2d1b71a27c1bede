// Instantiation of the warp kernel and its traceback variant for 24 band slots per lane (w <= 767).
#include "kernel_tb.cuh"

namespace agatha {
template cudaError_t launch_warp_c<24>(const DevBatch *, int, cudaStream_t, int, int);
template int occupancy_warp_c<24>();
template cudaError_t launch_tb_c<24>(const DevBatch *, const TbItem *, int32_t, int32_t *, uint8_t *,
                                    uint32_t *, int32_t *, int, cudaStream_t);
template int occupancy_tb_c<24>();
}  // namespace agatha
