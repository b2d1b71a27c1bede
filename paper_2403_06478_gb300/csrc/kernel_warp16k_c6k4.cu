// Instantiation of the 16-bit packed-lane kernel with 4 warps sharing one
// pair's band, 6 slots per lane each (768 slots: w <= 767), for the
// longest pairs (the autotuner's choice per length class).
#include "kernel_warp16.cuh"

namespace agatha {
template cudaError_t launch_warp16k_c<6, 4, 4>(const DevBatch *, int, cudaStream_t, int, int);
template int occupancy_warp16k_c<6, 4, 4>();
}  // namespace agatha
