// Device-side definitions shared by the alignment kernels of this library.
//
// Coordinates: t indexes the target (reference), q the query, r = t + q is the
// anti-diagonal (paper Section 2.1: cells of one anti-diagonal are
// independent).  Inside the band |t - q| <= w, anti-diagonal r holds the cells
//     t in [ceil((r - w) / 2), floor((r + w) / 2)]
// (clipped to the table).  The kernels index them by a "slot"
//     j = t - B(r),   B(r) = ceil((r - w) / 2),   j in [0, w]
// On anti-diagonals with (r - w) even all w+1 slots are band cells; when it is
// odd slot w is outside the band (t - q = w + 1).  Going from r-1 to r:
//   diagonal predecessor (t-1, q-1) sits in the same slot j on r-2,
//   (t-1, q) [E, E2 input] sits in slot j-1 on r-1 if (r-w) is even, else j,
//   (t, q-1) [F, F2 input] sits in slot j   on r-1 if (r-w) is even, else j+1.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "agatha.h"

namespace agatha {

// "Minus infinity" of the int32 kernels.  Scores are validated on the host to
// stay within +-2^28, so this value is never reached by a real cell and
// subtracting a few penalties from it cannot wrap.
constexpr int32_t K_NEG = -(1 << 29);
constexpr int32_t K_NEG_OUT = AGATHA_NEG_INF;

struct DevParams {
    int32_t a, b, q, e, q2, e2, w, zdrop, end_bonus;
};

// Batch descriptor, resident in device memory so that one captured CUDA graph
// can be replayed for any batch the host stages.
struct DevBatch {
    const uint32_t *q_packed;
    const uint32_t *t_packed;
    int64_t q_words;
    int64_t t_words;
    const int64_t *q_off;
    const int64_t *t_off;
    const int32_t *q_len;
    const int32_t *t_len;
    agatha_result *out;
    int64_t n_pairs;
    // schedule produced by the prep kernels
    int32_t *order;          // pair indices, longest predicted work first
    int32_t *counters;       // queue heads and counts (CTR_*), [3] error word
    int32_t *wide_order;     // pairs whose band is too wide for the warp kernel, or
                             // (narrow_w_max > 0) those the narrower frame takes
    int64_t *bucket_hist;    // scratch for the ordering
    int32_t *ovf_list;       // pairs the 16-bit kernel hands back to the 32-bit one
    const int32_t *h0;       // local extension: the initial score of each pair (else null)
    DevParams params;
    int32_t warp_w_max;      // widest band the warp kernel takes (32*C - 1)
    int32_t narrow_w_max;    // > 0: pairs whose band is at most this go to the
                             // narrow list (a frame of fewer slots per lane)
};

enum : int32_t { CTR_HEAD = 0, CTR_NWARP = 1, CTR_NWIDE = 2, CTR_ERR = 3, CTR_WIDE_HEAD = 4,
                 CTR_NOVF = 5, CTR_OVF_HEAD = 6, CTR_CLS_HEAD = 8, CTR_T_BEGIN = 12, CTR_T_END = 14,
                 CTR_COUNT = 16 };

// Device clock of a step's kernels, in nanoseconds of the GPU's global timer
// (one clock for every SM): counters[CTR_T_BEGIN..+1] holds when the first
// block of the step's first kernel started, counters[CTR_T_END..+1] when the
// last warp of its alignment kernels finished.  Both are 64-bit words inside
// the counters, so they are cleared with them at the start of every step.
// The serving loop reads them to tell whether two launches ran at once.
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void mark_step_begin(int32_t *counters) {
    atomicCAS(reinterpret_cast<unsigned long long *>(counters + CTR_T_BEGIN), 0ull,
              (unsigned long long)global_ns());
}
__device__ __forceinline__ void mark_step_end(int32_t *counters) {
    atomicMax(reinterpret_cast<unsigned long long *>(counters + CTR_T_END),
              (unsigned long long)global_ns());
}

// Which pair list a warp kernel launch walks: the whole ordered queue, the
// pairs the 16-bit kernel handed back, or the part of the ordered queue that
// holds one length class (WARP_LIST_CLASS + c).
enum : int32_t { WARP_LIST_NARROW = -1, WARP_LIST_MAIN = 0, WARP_LIST_OVERFLOW = 1, WARP_LIST_CLASS = 2 };

// Length classes the kernel choice is tuned for, by predicted band cells:
// class 0 >= 2^25, class 1 >= 2^23, class 2 >= 2^21, class 3 the rest.  In
// the ordering's buckets (bucket = 255 - (4 floor(log2 cells) + quarter)),
// class c holds buckets [CLASS_BUCKET[c], CLASS_BUCKET[c + 1]).
constexpr int N_CLASSES = 4;
__host__ __device__ inline int32_t class_first_bucket(int c) {
    return c <= 0 ? 0 : (c == 1 ? 156 : (c == 2 ? 164 : (c == 3 ? 172 : 256)));
}
__host__ __device__ inline int32_t class_of_cells(uint64_t est) {
    int32_t lg = 0;
    while ((est >> lg) > 1) ++lg;                     // floor(log2), est >= 1
    return lg >= 25 ? 0 : (lg >= 23 ? 1 : (lg >= 21 ? 2 : 3));
}
// Predicted band cells of a pair (Section 4.5 model): anti-diagonals x band.
__host__ __device__ inline uint64_t predicted_cells(int32_t tlen, int32_t qlen, int32_t w) {
    return (uint64_t)(tlen + qlen) * (uint64_t)(w + 1) / 2 + 1;
}

// Largest initial score of the local extension (keeps every score in int32
// beside the length bound of pair_valid).
constexpr int32_t LOCAL_H0_MAX = 1 << 24;

// device error codes written to counters[CTR_ERR]
enum : int32_t { DEV_ERR_NONE = 0, DEV_ERR_BAD_PAIR = 1 };

__host__ __device__ inline int32_t floor_div2(int32_t x) { return x >> 1; }   // arithmetic shift
__host__ __device__ inline int32_t ceil_div2(int32_t x) { return -((-x) >> 1); }

__device__ __forceinline__ int32_t gap_cost(const DevParams &p, int32_t l) {
    return min(p.q + l * p.e, p.q2 + l * p.e2);
}

// Band cells of anti-diagonals 0..R of a table (tlen x qlen, effective
// half-width w), R <= tlen + qlen - 2 and the band still inside the table up
// to R: the sum over r of en(r) - st(r) + 1 with en = min(tlen - 1, r,
// floor((r + w) / 2)) and st = max(0, r - qlen + 1, ceil((r - w) / 2)), in
// closed form (each bound is piecewise linear in r, with floor/ceil halves).
__host__ __device__ inline int64_t sum_half_floor(int64_t m) {      // sum_{k=0}^{m} floor(k/2)
    return m < 0 ? 0 : (m * m) / 4;
}
__host__ __device__ inline int64_t sum_floor_half(int64_t a, int64_t b, int64_t c) {
    return b < a ? 0 : sum_half_floor(b + c) - sum_half_floor(a - 1 + c);   // sum_{r=a}^{b} floor((r+c)/2)
}
__host__ __device__ inline int64_t band_cells_through(int32_t tlen, int32_t qlen, int32_t w, int32_t R) {
    if (R < 0) return 0;
    const int64_t T = tlen - 1, Qm = qlen - 1, W = w, RR = R;
    // sum of en: r up to w, floor((r + w) / 2) after, until it reaches T at rT
    const int64_t rT = T <= W ? T : 2 * T - W;
    const int64_t n = RR < rT - 1 ? RR : rT - 1;
    int64_t sen = 0;
    if (n >= 0) sen = n <= W ? n * (n + 1) / 2 : W * (W + 1) / 2 + sum_floor_half(W + 1, n, W);
    if (RR >= rT) sen += T * (RR - rT + 1);
    // sum of st: 0, then ceil((r - w) / 2) from w + 1 while qlen - 1 > w,
    // then r - qlen + 1 (from 2(qlen - 1) - w, or from qlen when qlen - 1 <= w)
    int64_t sst = 0;
    if (Qm <= W) {
        const int64_t m = RR - Qm;
        if (m > 0) sst = m * (m + 1) / 2;
    } else {
        const int64_t rq = 2 * Qm - W;
        sst = sum_floor_half(W + 1, RR < rq - 1 ? RR : rq - 1, 1 - W);
        if (RR >= rq) {
            const int64_t hi = RR - Qm, lo = Qm - W;
            sst += hi * (hi + 1) / 2 - (lo - 1) * lo / 2;
        }
    }
    return sen - sst + RR + 1;
}

// Effective half-width: a band wider than the table changes nothing.
__host__ __device__ inline int32_t effective_w(int32_t w, int32_t tlen, int32_t qlen) {
    int32_t m = tlen > qlen ? tlen : qlen;
    return (w < 0 || w > m) ? m : w;
}

// The largest change of a score from one anti-diagonal to the next: the
// 16-bit lanes are sized from it and take it up to STEP16_MAX.
constexpr int32_t STEP16_MAX = 255;
__host__ __device__ inline int32_t step_change_max(const DevParams &p) {
    int32_t d = p.a > p.b ? p.a : p.b;
    d = d > p.q + p.e ? d : p.q + p.e;
    d = d > p.q2 + p.e2 ? d : p.q2 + p.e2;
    return d > 0 ? d : 1;
}

// One packed word of a stream, zero outside it (reads are clamped).
__device__ __forceinline__ uint32_t load_word(const uint32_t *__restrict__ p, int64_t n_words,
                                              int64_t i) {
    return (i >= 0 && i < n_words) ? __ldg(p + i) : 0u;
}

// 16 consecutive bases starting at base index g (any g, outside reads give 0).
__device__ __forceinline__ uint32_t load16(const uint32_t *__restrict__ p, int64_t n_words,
                                           int64_t g) {
    int64_t wi = g >> 4;                         // floor for negative g too
    uint32_t sh = (uint32_t)(g & 15) * 2u;
    uint32_t lo = load_word(p, n_words, wi);
    uint32_t hi = load_word(p, n_words, wi + 1);
    return __funnelshift_r(lo, hi, sh);
}

// 32 consecutive bases starting at g.
__device__ __forceinline__ uint64_t load32(const uint32_t *__restrict__ p, int64_t n_words,
                                           int64_t g) {
    uint64_t lo = load16(p, n_words, g);
    uint64_t hi = load16(p, n_words, g + 16);
    return lo | (hi << 32);
}

// Reverse the order of the 2-bit fields of a word.
__device__ __forceinline__ uint32_t rev2_32(uint32_t x) {
    x = __brev(x);
    return ((x >> 1) & 0x55555555u) | ((x & 0x55555555u) << 1);
}
__device__ __forceinline__ uint64_t rev2_64(uint64_t x) {
    x = __brevll(x);
    return ((x >> 1) & 0x5555555555555555ull) | ((x & 0x5555555555555555ull) << 1);
}

__device__ __forceinline__ void write_empty_result(agatha_result *o) {
    agatha_result r;
    r.max = 0; r.qe = -1; r.te = -1;
    r.gscore = K_NEG_OUT; r.mqe = K_NEG_OUT; r.mte = K_NEG_OUT;
    r.mqe_t = -1; r.mte_q = -1;
    r.cells = 0;
    r.zdropped = 0; r.reach_end = 0; r.lane16 = 0;
    for (int i = 0; i < 5; ++i) r.pad[i] = 0;
    *o = r;
}

// Band cells of anti-diagonal r (0 when empty).
__device__ __forceinline__ int32_t band_cells_on(int32_t r, int32_t tlen, int32_t qlen, int32_t w) {
    int32_t st = max(max(0, r - qlen + 1), ceil_div2(r - w));
    int32_t en = min(min(tlen - 1, r), floor_div2(r + w));
    return en >= st ? en - st + 1 : 0;
}

// A pair the kernels may align: lengths and offsets inside the streams, and
// scores that keep int32 headroom.
__device__ __forceinline__ bool pair_valid(const DevBatch &B, int64_t i) {
    const int32_t tl = B.t_len[i], ql = B.q_len[i];
    const int64_t to = B.t_off[i], qo = B.q_off[i];
    if (tl < 0 || ql < 0 || tl >= (1 << 24) || ql >= (1 << 24)) return false;
    if (to < 0 || qo < 0) return false;
    if (to + tl > B.t_words * 16 || qo + ql > B.q_words * 16) return false;
    const DevParams &p = B.params;
    const int64_t unit = (int64_t)p.a + p.b + p.q + p.e + p.q2 + p.e2 + (p.end_bonus > 0 ? p.end_bonus : 0);
    if (unit * ((int64_t)tl + ql + 2) >= (int64_t)1 << 28) return false;   // int32 headroom
    return true;
}

// The pairs one warp-kernel launch walks: items[begin..end) (input order
// when items is null), handed out through the queue head *head.
struct WorkList {
    const int32_t *items;
    int32_t *head;
    int32_t begin, end;
};

__device__ __forceinline__ WorkList work_list(const DevBatch &B, int32_t list) {
    WorkList L;
    if (list == WARP_LIST_NARROW) {
        // the pairs whose band fits the narrower frame (unordered; they are
        // the shortest ones)
        L.items = B.wide_order;
        L.head = &B.counters[CTR_WIDE_HEAD];
        L.begin = 0;
        L.end = B.counters[CTR_NWIDE];
    } else if (list == WARP_LIST_OVERFLOW) {
        L.items = B.ovf_list;
        L.head = &B.counters[CTR_OVF_HEAD];
        L.begin = 0;
        L.end = B.counters[CTR_NOVF];
    } else if (list >= WARP_LIST_CLASS) {
        // after the ordering, bucket_hist[b] is the end of bucket b in `order`
        const int c = list - WARP_LIST_CLASS;
        const int32_t b0 = class_first_bucket(c), b1 = class_first_bucket(c + 1);
        L.items = B.order;
        L.head = &B.counters[CTR_CLS_HEAD + c];
        L.begin = b0 > 0 ? (int32_t)B.bucket_hist[b0 - 1] : 0;
        L.end = (int32_t)B.bucket_hist[b1 - 1];
    } else {
        L.items = B.order;
        L.head = &B.counters[CTR_HEAD];
        L.begin = 0;
        L.end = B.order ? B.counters[CTR_NWARP] : (int32_t)B.n_pairs;
    }
    return L;
}

// One pair of a traceback launch: its end cell (from the score path) and
// where its direction table (bytes) and run scratch (uint32) start.
struct TbItem {
    int32_t pair, end_t, end_q, pad;
    int64_t dir_off, ops_off;
};

// Launchers (defined in the .cu files).
cudaError_t launch_prep(const DevBatch *d_batch, int64_t n_pairs, int32_t sort, cudaStream_t s,
                        int n_sm);
template <int C>
cudaError_t launch_warp_c(const DevBatch *d_batch, int n_blocks, cudaStream_t s, int use_fast,
                          int list = WARP_LIST_MAIN);
template <int C>
int occupancy_warp_c();
// MINB: resident blocks per SM the 16-bit kernel's registers are cut for.
// G: lanes per pair (32, or 16 for two pairs per warp).
template <int C, int MINB, int G = 32>
cudaError_t launch_warp16_c(const DevBatch *d_batch, int n_blocks, cudaStream_t s, int use_fast,
                            int list = WARP_LIST_MAIN);
template <int C, int MINB, int G = 32>
int occupancy_warp16_c();
template <int C, int MINB>
cudaError_t launch_warp16_prio(const DevBatch *d_batch, int n_blocks, cudaStream_t s, int use_fast, int list,
                               int priority);
// K warps share one pair's band (C slots per lane of each warp).
template <int C, int K, int MINB>
cudaError_t launch_warp16k_c(const DevBatch *d_batch, int n_blocks, cudaStream_t s, int use_fast, int list);
template <int C, int K, int MINB>
int occupancy_warp16k_c();
template <int C>
cudaError_t launch_tb_c(const DevBatch *d_batch, const TbItem *items, int32_t n_items, int32_t *head,
                        uint8_t *dir, uint32_t *ops, int32_t *n_cigar, int n_blocks, cudaStream_t s);
template <int C>
int occupancy_tb_c();
template <int C, int MINB>
cudaError_t launch_tb16_c(const DevBatch *d_batch, const TbItem *items, int32_t n_items, int32_t *head,
                          uint8_t *dir, uint32_t *ops, int32_t *n_cigar, int n_blocks, cudaStream_t s);
template <int C, int MINB>
int occupancy_tb16_c();
template <int C, int MINB>
cudaError_t launch_tbf16_c(const DevBatch *d_batch, const TbItem *items, int32_t n_items, int32_t *head,
                           uint8_t *dir, uint32_t *ops, int32_t *n_cigar, int n_blocks, cudaStream_t s);
template <int C, int MINB>
int occupancy_tbf16_c();
// Copy each pair's runs (written end first) to dense[dst_off[pair]..] in order.
cudaError_t launch_cigar_gather(const TbItem *items, int32_t n_items, const int32_t *n_cigar,
                                const int64_t *dst_off, const uint32_t *ops, uint32_t *dense,
                                int n_blocks, cudaStream_t s);
cudaError_t launch_plain_kernel(const DevBatch *d_batch, int64_t n_blocks, int32_t w_max,
                                int use_wide_list, cudaStream_t s);
// The local extension (kernel_local.cu), C slots per lane of int32 lanes.
cudaError_t launch_local(int C, const DevBatch *d_batch, int n_blocks, cudaStream_t s);
int local_occupancy(int C);
int plain_kernel_max_w();
cudaError_t plain_kernel_prepare();

}  // namespace agatha
