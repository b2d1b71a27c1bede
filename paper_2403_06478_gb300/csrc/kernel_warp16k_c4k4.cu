// Instantiation of the 16-bit packed-lane kernel with 4 warps sharing one
// pair's band, 4 slots per lane each (512 slots: w <= 511), for the
// longest pairs (the autotuner's choice per length class).
#include "kernel_warp16.cuh"

namespace agatha {
template cudaError_t launch_warp16k_c<4, 4, 6>(const DevBatch *, int, cudaStream_t, int, int);
template int occupancy_warp16k_c<4, 4, 6>();
}  // namespace agatha
