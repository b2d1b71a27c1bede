// Instantiation of the 16-bit packed-lane warp kernel for 16 band slots per
// lane (w <= 511).
#include "kernel_warp16.cuh"

namespace agatha {
template cudaError_t launch_warp16_c<16>(const DevBatch *, int, cudaStream_t, int);
template int occupancy_warp16_c<16>();
}  // namespace agatha
