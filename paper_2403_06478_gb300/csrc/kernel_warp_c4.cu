// Instantiation of the warp kernel for 4 band slots per lane (w <= 127).
#include "kernel_warp.cuh"

namespace agatha {
template cudaError_t launch_warp_c<4>(const DevBatch *, int, cudaStream_t, int, int);
template int occupancy_warp_c<4>();
}  // namespace agatha
