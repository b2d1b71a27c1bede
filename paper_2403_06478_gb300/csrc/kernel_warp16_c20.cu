// Instantiation of the 16-bit packed-lane warp kernel for 20 band slots per
// lane (a 640-slot frame, w <= 638) at the larger register budget: the frame
// of the pairs of a 24-slot batch whose own band fits it.
#include "kernel_warp16.cuh"

namespace agatha {
template cudaError_t launch_warp16_c<20, 2>(const DevBatch *, int, cudaStream_t, int, int);
template int occupancy_warp16_c<20, 2>();
template cudaError_t launch_warp16_prio<20, 2>(const DevBatch *, int, cudaStream_t, int, int, int);
}  // namespace agatha
