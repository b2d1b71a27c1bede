// Instantiation of the 16-bit packed-lane kernel with 2 warps sharing one
// pair's band, 8 slots per lane each (512 slots: w <= 511), for the
// longest pairs (the autotuner's choice per length class).
#include "kernel_warp16.cuh"

namespace agatha {
template cudaError_t launch_warp16k_c<8, 2, 4>(const DevBatch *, int, cudaStream_t, int, int);
template int occupancy_warp16k_c<8, 2, 4>();
}  // namespace agatha
