// Instantiation of the 16-bit packed-lane warp kernel for 24 band slots per
// lane (w <= 767).
#include "kernel_warp16.cuh"

namespace agatha {
template cudaError_t launch_warp16_c<24>(const DevBatch *, int, cudaStream_t, int);
template int occupancy_warp16_c<24>();
}  // namespace agatha
