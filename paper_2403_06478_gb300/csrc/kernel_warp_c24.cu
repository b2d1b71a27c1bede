// Instantiation of the warp kernel for 24 band slots per lane (w <= 767).
#include "kernel_warp.cuh"

namespace agatha {
template cudaError_t launch_warp_c<24>(const DevBatch *, int, cudaStream_t, int, int);
template int occupancy_warp_c<24>();
}  // namespace agatha
