// Instantiation of the warp kernel for 32 band slots per lane (w <= 1023).
#include "kernel_warp.cuh"

namespace agatha {
template cudaError_t launch_warp_c<32>(const DevBatch *, int, cudaStream_t, int, int);
template int occupancy_warp_c<32>();
}  // namespace agatha
