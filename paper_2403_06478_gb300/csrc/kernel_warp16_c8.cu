// Instantiation of the 16-bit packed-lane warp kernel for 8 band slots per
// lane (w <= 255).
#include "kernel_warp16.cuh"

namespace agatha {
template cudaError_t launch_warp16_c<8>(const DevBatch *, int, cudaStream_t, int);
template int occupancy_warp16_c<8>();
}  // namespace agatha
