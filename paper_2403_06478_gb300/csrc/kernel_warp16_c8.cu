// Instantiations of the 16-bit packed-lane warp kernel for 8 band slots per
// lane (w <= 255), at two register budgets (resident blocks per SM): the
// autotuner picks one per length class.
#include "kernel_tb.cuh"

namespace agatha {
template cudaError_t launch_warp16_c<8, 4>(const DevBatch *, int, cudaStream_t, int, int);
template int occupancy_warp16_c<8, 4>();
template cudaError_t launch_warp16_c<8, 3>(const DevBatch *, int, cudaStream_t, int, int);
template int occupancy_warp16_c<8, 3>();
// two pairs per warp, 16 lanes of 8 slots (the 4-slot band of 128 slots)
template cudaError_t launch_warp16_c<8, 3, 16>(const DevBatch *, int, cudaStream_t, int, int);
template int occupancy_warp16_c<8, 3, 16>();
// the traceback variants (two-pass and fused) at one budget (no spills)
template cudaError_t launch_tb16_c<8, 4>(const DevBatch *, const TbItem *, int32_t, int32_t *, uint8_t *,
                                          uint32_t *, int32_t *, int, cudaStream_t);
template int occupancy_tb16_c<8, 4>();
template cudaError_t launch_tbf16_c<8, 4>(const DevBatch *, const TbItem *, int32_t, int32_t *, uint8_t *,
                                           uint32_t *, int32_t *, int, cudaStream_t);
template int occupancy_tbf16_c<8, 4>();
}  // namespace agatha
