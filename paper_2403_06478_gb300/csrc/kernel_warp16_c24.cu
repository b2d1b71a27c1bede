// Instantiations of the 16-bit packed-lane warp kernel for 24 band slots per
// lane (w <= 767), at two register budgets (resident blocks per SM): the
// autotuner picks one per length class.
#include "kernel_tb.cuh"

namespace agatha {
template cudaError_t launch_warp16_c<24, 3>(const DevBatch *, int, cudaStream_t, int, int);
template int occupancy_warp16_c<24, 3>();
template cudaError_t launch_warp16_c<24, 2>(const DevBatch *, int, cudaStream_t, int, int);
template int occupancy_warp16_c<24, 2>();
template cudaError_t launch_warp16_prio<24, 3>(const DevBatch *, int, cudaStream_t, int, int, int);
template cudaError_t launch_warp16_prio<24, 2>(const DevBatch *, int, cudaStream_t, int, int, int);
// the traceback variants (two-pass and fused) at one budget (no spills)
template cudaError_t launch_tb16_c<24, 2>(const DevBatch *, const TbItem *, int32_t, int32_t *, uint8_t *,
                                          uint32_t *, int32_t *, int, cudaStream_t);
template int occupancy_tb16_c<24, 2>();
template cudaError_t launch_tbf16_c<24, 2>(const DevBatch *, const TbItem *, int32_t, int32_t *, uint8_t *,
                                           uint32_t *, int32_t *, int, cudaStream_t);
template int occupancy_tbf16_c<24, 2>();
}  // namespace agatha
