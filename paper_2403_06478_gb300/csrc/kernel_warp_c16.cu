// Instantiation of the warp kernel for 16 band slots per lane (w <= 511).
#include "kernel_warp.cuh"

namespace agatha {
template cudaError_t launch_warp_c<16>(const DevBatch *, int, cudaStream_t, int, int);
template int occupancy_warp_c<16>();
}  // namespace agatha
