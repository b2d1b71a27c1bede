// Instantiations of the 16-bit packed-lane warp kernel for 4 band slots per
// lane (w <= 127), at two register budgets (resident blocks per SM): the
// autotuner picks one per length class.
#include "kernel_warp16.cuh"

namespace agatha {
template cudaError_t launch_warp16_c<4, 6>(const DevBatch *, int, cudaStream_t, int, int);
template int occupancy_warp16_c<4, 6>();
template cudaError_t launch_warp16_c<4, 4>(const DevBatch *, int, cudaStream_t, int, int);
template int occupancy_warp16_c<4, 4>();
}  // namespace agatha
