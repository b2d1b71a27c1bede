// Batch preparation on the device: validate every pair, route it to the warp
// kernel or (band too wide) to the block kernel, and order the warp kernel's
// work queue longest-first.
//
// Ordering follows the paper's performance model (Section 4.5): the work of a
// pair is about Cells = Antidiags x Band_width, and the slowest warps dominate
// (the MAX over warps in Table 1).  Uneven bucketing (Section 4.4) spreads the
// longest tasks over different warps; here the persistent kernel's queue hands
// out pairs in decreasing predicted work (longest-processing-time first), so
// the long pairs start first and the short ones fill the tail.  The sort is a
// counting sort over 256 quarter-octave buckets of predicted cells.
#include "agatha_dev.cuh"

namespace agatha {

constexpr int PREP_THREADS = 256;
constexpr int N_BUCKETS = 256;

// Bucket 0 holds the largest predicted work.
__device__ __forceinline__ int32_t work_bucket(int32_t tlen, int32_t qlen, int32_t w) {
    const uint64_t est = predicted_cells(tlen, qlen, w);
    const int32_t lg = 63 - __clzll(est);                    // floor(log2)
    const int32_t frac = lg >= 2 ? (int32_t)((est >> (lg - 2)) & 3) : 0;
    int32_t key = lg * 4 + frac;                              // 4 buckets per octave
    key = key > N_BUCKETS - 1 ? N_BUCKETS - 1 : key;
    return N_BUCKETS - 1 - key;
}

__global__ void prep_classify_kernel(const DevBatch *__restrict__ d_batch, int32_t sort) {
    const DevBatch B = *d_batch;
    if (threadIdx.x == 0) mark_step_begin(B.counters);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < B.n_pairs;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (!pair_valid(B, i)) {
            atomicExch(&B.counters[CTR_ERR], DEV_ERR_BAD_PAIR);
            write_empty_result(B.out + i);
            continue;
        }
        const int32_t tl = B.t_len[i], ql = B.q_len[i];
        const int32_t w = effective_w(B.params.w, tl, ql);
        if (w > B.warp_w_max || (B.narrow_w_max > 0 && w <= B.narrow_w_max)) {
            // too wide for the warp kernel (the block kernel's list), or a band
            // the narrower frame takes (its own list; never both in one batch)
            const int32_t k = atomicAdd(&B.counters[CTR_NWIDE], 1);
            B.wide_order[k] = (int32_t)i;
            continue;
        }
        if (sort) atomicAdd((unsigned long long *)&B.bucket_hist[work_bucket(tl, ql, w)], 1ull);
        else atomicAdd(&B.counters[CTR_NWARP], 1);
    }
}

// Exclusive scan of the bucket histogram (one block); bucket_hist[b] becomes
// the first queue position of bucket b.
__global__ void prep_scan_kernel(const DevBatch *__restrict__ d_batch) {
    const DevBatch B = *d_batch;
    __shared__ int64_t s[N_BUCKETS];
    const int t = threadIdx.x;
    s[t] = B.bucket_hist[t];
    __syncthreads();
    for (int o = 1; o < N_BUCKETS; o <<= 1) {
        const int64_t v = t >= o ? s[t - o] : 0;
        __syncthreads();
        s[t] += v;
        __syncthreads();
    }
    const int64_t incl = s[t];
    B.bucket_hist[t] = incl - B.bucket_hist[t];
    if (t == N_BUCKETS - 1) B.counters[CTR_NWARP] = (int32_t)incl;
}

__global__ void prep_scatter_kernel(const DevBatch *__restrict__ d_batch) {
    const DevBatch B = *d_batch;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < B.n_pairs;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (!pair_valid(B, i)) continue;
        const int32_t tl = B.t_len[i], ql = B.q_len[i];
        const int32_t w = effective_w(B.params.w, tl, ql);
        if (w > B.warp_w_max || (B.narrow_w_max > 0 && w <= B.narrow_w_max)) continue;
        const int32_t b = work_bucket(tl, ql, w);
        const int64_t pos = (int64_t)atomicAdd((unsigned long long *)&B.bucket_hist[b], 1ull);
        B.order[pos] = (int32_t)i;
    }
}

cudaError_t launch_prep(const DevBatch *d_batch, int64_t n_pairs, int32_t sort, cudaStream_t s,
                        int n_sm) {
    // a fixed grid (grid-stride loops) so one captured graph serves any batch size
    (void)n_pairs;
    const int64_t blocks = (int64_t)(n_sm > 0 ? n_sm : 1) * 4;
    prep_classify_kernel<<<(unsigned)blocks, PREP_THREADS, 0, s>>>(d_batch, sort);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess || !sort) return err;
    prep_scan_kernel<<<1, N_BUCKETS, 0, s>>>(d_batch);
    err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    prep_scatter_kernel<<<(unsigned)blocks, PREP_THREADS, 0, s>>>(d_batch);
    return cudaGetLastError();
}

}  // namespace agatha
