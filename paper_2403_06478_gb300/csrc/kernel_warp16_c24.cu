// Instantiations of the 16-bit packed-lane warp kernel for 24 band slots per
// lane (w <= 767), at two register budgets (resident blocks per SM): the
// autotuner picks one per length class.
#include "kernel_warp16.cuh"

namespace agatha {
template cudaError_t launch_warp16_c<24, 3>(const DevBatch *, int, cudaStream_t, int, int);
template int occupancy_warp16_c<24, 3>();
template cudaError_t launch_warp16_c<24, 2>(const DevBatch *, int, cudaStream_t, int, int);
template int occupancy_warp16_c<24, 2>();
}  // namespace agatha
