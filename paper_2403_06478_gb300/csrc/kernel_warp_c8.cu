// Instantiation of the warp kernel for 8 band slots per lane (w <= 255).
#include "kernel_warp.cuh"

namespace agatha {
template cudaError_t launch_warp_c<8>(const DevBatch *, int, cudaStream_t, int, int);
template int occupancy_warp_c<8>();
}  // namespace agatha
