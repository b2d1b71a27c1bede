// Traceback kernels: the CIGAR of each extension, after the score path has
// found its end cell.
//
// One warp takes one pair from a device queue (longest first, like the score
// kernels).  It recomputes anti-diagonals 0..r_end of the pair's band with
// the warp step of a score kernel in its DIR variant, which writes one
// direction byte per band slot: lane L stores its C bytes of anti-diagonal r
// at table[r * 32C + L*C] with one vector store, so a warp writes a 32C-byte
// row per step, coalesced.  Two kernels share the walk:
//   tb16_kernel  the 16-bit packed-lane step (kernel_warp16.cuh): two cells
//                per instruction, its slot frame B(r) = floor((r-w)/2), bytes
//                2p and 2p+1 of a lane from the halves of register p; a pair
//                whose scores leave the 16-bit range is marked (n = -1) and
//                the host hands it to
//   tb_kernel    the int32 step (kernel_warp.cuh): frame ceil((r-w)/2),
//                bytes in slot order.
// The table lives in HBM (a batch's tables take tens to hundreds of GB; the
// host runs the batch in waves that fit).
//
// Then the warp walks back from the end cell.  Each step moves to anti-
// diagonal r-1 or r-2 and its slot changes by at most one per anti-diagonal
// (see agatha_dev.cuh for the slot frame), so the cells of the next 32
// anti-diagonals that the path can reach lie within +-31 slots of the
// current one.  The warp loads that window (80 or 144 bytes of each of 32
// rows, one row per lane, 16-byte loads; TbLayout) into shared memory with
// one round trip to memory, and lane 0 follows the path through it; a path
// of n steps costs about n/24 memory round trips instead of n.
//
// Walk rule (the reading of the oracle's traceback): in state H the cell's
// byte says which input H took (diagonal, E, F, E2, F2; the int32 kernel
// stores the index, the 16-bit kernel one "differs" bit per input).  A diagonal step
// emits M and moves to (t-1, q-1); E/E2 emit D and move to (t-1, q); F/F2
// emit I and move to (t, q-1).  Whether the gap continues is stored at the
// cell it moves to (the Eo/Fo bits of that cell), so the state is resolved
// there before anything else: continue the gap, or take that cell's H.
// Reaching the virtual row (t = -1) adds q+1 leading insertions, the virtual
// column (q = -1) t+1 leading deletions.
//
// Runs are written end first into the pair's scratch (one uint32 per run,
// (length << 4) | op, op M=0 I=1 D=2); the gather kernel reverses them into
// the caller's order.
#pragma once

#include "kernel_warp16.cuh"

namespace agatha {

constexpr int TB_WIN_ROWS = 32;     // rows (anti-diagonals) per window

// Where a slot's byte sits and which bytes of a row the walk window holds.
// The window covers slots [ws, ws + WB) of 32 rows: every slot the path can
// reach within 31 anti-diagonals of slot jc (|slot change| <= 1 per
// anti-diagonal) when ws <= jc - 31 and ws + WB > jc + 31.  With the 16-bit
// kernel's byte order it must cover whole lanes, so ws is a multiple of WA,
// itself a multiple of C and of 16 (16-byte loads).
template <int C, bool PACKED>
struct TbLayout {
    static constexpr int32_t ROW = 32 * C;
    static constexpr int32_t P = C / 2;
    static constexpr int32_t WA = (PACKED && C > 16) ? 48 : 16;
    static constexpr int32_t WB = (PACKED && C > 16) ? 144 : 80;
    static_assert(WA % 16 == 0 && (!PACKED || WA % C == 0) && WB % WA == 0 && WB >= 62 + WA &&
                      ROW >= WB && (ROW - WB) % WA == 0,
                  "window geometry");
    __device__ __forceinline__ static int32_t frame(int32_t r, int32_t w) {
        return PACKED ? floor_div2(r - w) : ceil_div2(r - w);
    }
    __device__ __forceinline__ static int32_t byte_of(int32_t j) {
        if constexpr (!PACKED) {
            return j;
        } else {
            const int32_t lb = (j / C) * C, jl = j - lb;
            return lb + (jl < P ? 2 * jl : 2 * (jl - P) + 1);
        }
    }
    // H source (0 diagonal, 1 E, 2 F, 3 E2, 4 F2) from a byte
    __device__ __forceinline__ static int32_t source(uint32_t b) {
        if constexpr (!PACKED) {
            const int32_t s = (int32_t)(b & 7u);
            return s > 4 ? 0 : s;           // never written; keeps the walk moving
        } else {
            return (int32_t)(__ffs(~b & 0xfu) ? __ffs(~b & 0xfu) - 1 : 4);
        }
    }
    // whether the gap state k (1 E, 2 F, 3 E2, 4 F2) leaving this cell extended
    __device__ __forceinline__ static bool extended(uint32_t b, int32_t k) {
        return (b >> ((PACKED ? 3 : 2) + k)) & 1u;
    }
};

enum : uint32_t { TB_OP_M = 0, TB_OP_I = 1, TB_OP_D = 2 };

// Walk states: 0..4 = the H source being followed (diagonal, E, F, E2, F2),
// TB_H = decode H at this cell, TB_PEND + k = the gap state k (1..4) arrived
// here and its continuation bit must be read at this cell.
enum : int32_t { TB_DIAG = 0, TB_H = 5, TB_PEND = 5 };

struct TbRuns {
    uint32_t *ops;
    int32_t cap, n;
    uint32_t op, len;
    __device__ __forceinline__ void push(uint32_t o, uint32_t l) {
        if (len > 0 && op == o) { len += l; return; }
        if (len > 0 && n < cap) ops[n] = (len << 4) | op;
        if (len > 0) ++n;
        op = o;
        len = l;
    }
};

// Walk back from (t, q) through the direction table dt of a pair with band
// half-width w.  Returns the number of runs (on every lane).
template <int C, bool PACKED>
__device__ __forceinline__ int32_t tb_walk(uint8_t *__restrict__ win, const uint8_t *dt,
                                           uint32_t *ops, int32_t cap, int32_t t, int32_t q,
                                           int32_t w, int32_t lane) {
    using Lay = TbLayout<C, PACKED>;
    constexpr int32_t ROW = Lay::ROW, WB = Lay::WB, WA = Lay::WA;
    TbRuns runs{ops, cap, 0, 0u, 0u};
    int32_t st = TB_H;
    int32_t done = (t < 0 || q < 0);
    for (;;) {
        t = __shfl_sync(FULL, t, 0);
        q = __shfl_sync(FULL, q, 0);
        done = __shfl_sync(FULL, done, 0);
        if (done) break;
        // window: rows r0 - lane, slots [ws, ws + WB) around the current slot
        const int32_t r0 = t + q;
        const int32_t jc = t - Lay::frame(r0, w);
        int32_t ws = jc - (TB_WIN_ROWS - 1);
        ws = ws < 0 ? 0 : (ws / WA) * WA;
        ws = min(ws, ROW - WB);
        const int32_t rk = r0 - lane;
        if (rk >= 0) {
            const uint4 *src = reinterpret_cast<const uint4 *>(dt + (int64_t)rk * ROW + ws);
            uint4 *dst = reinterpret_cast<uint4 *>(win + lane * WB);
#pragma unroll
            for (int i = 0; i < WB / 16; ++i) dst[i] = __ldcg(src + i);
        }
        __syncwarp();
        if (lane == 0) {
            for (;;) {
                if (t < 0 || q < 0) {
                    if (t < 0 && q >= 0) runs.push(TB_OP_I, (uint32_t)(q + 1));
                    if (q < 0 && t >= 0) runs.push(TB_OP_D, (uint32_t)(t + 1));
                    done = 1;
                    break;
                }
                const int32_t r = t + q;
                if (r < r0 - (TB_WIN_ROWS - 1)) break;          // next window
                const int32_t j = Lay::byte_of(t - Lay::frame(r, w)) - ws;   // in [0, WB)
                const uint32_t b = win[(r0 - r) * WB + j];
                if (st > TB_PEND)                                 // a gap arrived here
                    st = Lay::extended(b, st - TB_PEND) ? st - TB_PEND : TB_H;
                if (st == TB_H) st = Lay::source(b);
                if (st == TB_DIAG) {
                    runs.push(TB_OP_M, 1u); --t; --q; st = TB_H;
                } else if (st & 1) {                              // E, E2: a step in t
                    runs.push(TB_OP_D, 1u); --t; st += TB_PEND;
                } else {                                          // F, F2: a step in q
                    runs.push(TB_OP_I, 1u); --q; st += TB_PEND;
                }
            }
        }
        __syncwarp();
    }
    if (lane == 0) runs.push(0xfu, 1u);                           // flush the last run
    return __shfl_sync(FULL, runs.n, 0);
}

template <int C>
__global__ void __launch_bounds__(WARP_BLOCK_THREADS)
tb_kernel(const DevBatch *__restrict__ d_batch, const TbItem *__restrict__ items, int32_t n_items,
          int32_t *head, uint8_t *dir, uint32_t *ops, int32_t *n_cigar) {
    __shared__ __align__(16) uint8_t win[WARP_BLOCK_THREADS / 32][TB_WIN_ROWS * TbLayout<C, false>::WB];
    const DevBatch B = *d_batch;
    const int lane = threadIdx.x & 31;
    uint8_t *my_win = win[threadIdx.x >> 5];
    for (;;) {
        int32_t k = 0;
        if (lane == 0) k = atomicAdd(head, 1);
        k = __shfl_sync(FULL, k, 0);
        if (k >= n_items) break;
        const TbItem it = items[k];
        uint8_t *dt = dir + it.dir_off;
        {
            WarpPair<C, true> wp;
            wp.run_dir(B, it.pair, lane, it.end_t + it.end_q, dt);
        }
        __syncwarp();   // the table rows this warp wrote are read by other lanes
        const int32_t w = effective_w(B.params.w, B.t_len[it.pair], B.q_len[it.pair]);
        const int32_t n = tb_walk<C, false>(my_win, dt, ops + it.ops_off, it.end_t + it.end_q + 2,
                                            it.end_t, it.end_q, w, lane);
        if (lane == 0) n_cigar[it.pair] = n;
    }
}

// The same on 16-bit lanes; MINB resident blocks per SM as for the score kernel.
template <int C, int MINB>
__global__ void __launch_bounds__(WARP_BLOCK_THREADS, MINB)
tb16_kernel(const DevBatch *__restrict__ d_batch, const TbItem *__restrict__ items, int32_t n_items,
            int32_t *head, uint8_t *dir, uint32_t *ops, int32_t *n_cigar) {
    __shared__ Cold16 cold[WARP_BLOCK_THREADS / 32];
    __shared__ __align__(16) uint8_t win[WARP_BLOCK_THREADS / 32][TB_WIN_ROWS * TbLayout<C, true>::WB];
    const DevBatch B = *d_batch;
    const int lane = threadIdx.x & 31;
    uint8_t *my_win = win[threadIdx.x >> 5];
    for (;;) {
        int32_t k = 0;
        if (lane == 0) k = atomicAdd(head, 1);
        k = __shfl_sync(FULL, k, 0);
        if (k >= n_items) break;
        const TbItem it = items[k];
        uint8_t *dt = dir + it.dir_off;
        bool ok;
        {
            WarpPair16<C, (MINB < 4 && C <= 16) || MINB < 3, false, true> wp(cold[threadIdx.x >> 5]);
            ok = wp.run_dir(B, it.pair, lane, it.end_t + it.end_q, dt);
        }
        if (!ok) {                                  // scores left the 16-bit range
            if (lane == 0) n_cigar[it.pair] = -1;
            continue;
        }
        __syncwarp();
        const int32_t w = effective_w(B.params.w, B.t_len[it.pair], B.q_len[it.pair]);
        const int32_t n = tb_walk<C, true>(my_win, dt, ops + it.ops_off, it.end_t + it.end_q + 2,
                                           it.end_t, it.end_q, w, lane);
        if (lane == 0) n_cigar[it.pair] = n;
    }
}

// Fused score path and traceback on 16-bit lanes: each warp aligns a pair
// exactly as warp16_align_kernel does (results, termination, hand-back of
// pairs that leave the 16-bit range to the int32 score kernel's list) while
// writing the direction bytes of every anti-diagonal it computes, then walks
// back from the end cell it found.  The table of an item has room for every
// anti-diagonal of the pair (tlen + qlen - 1 rows) and its run scratch for
// tlen + qlen runs; a handed-back pair gets n = -1.
template <int C, int MINB>
__global__ void __launch_bounds__(WARP_BLOCK_THREADS, MINB)
tbf16_kernel(const DevBatch *__restrict__ d_batch, const TbItem *__restrict__ items, int32_t n_items,
             int32_t *head, uint8_t *dir, uint32_t *ops, int32_t *n_cigar) {
    __shared__ Cold16 cold[WARP_BLOCK_THREADS / 32];
    __shared__ __align__(16) uint8_t win[WARP_BLOCK_THREADS / 32][TB_WIN_ROWS * TbLayout<C, true>::WB];
    const DevBatch B = *d_batch;
    const int lane = threadIdx.x & 31;
    uint8_t *my_win = win[threadIdx.x >> 5];
    for (;;) {
        int32_t k = 0;
        if (lane == 0) k = atomicAdd(head, 1);
        k = __shfl_sync(FULL, k, 0);
        if (k >= n_items) break;
        const TbItem it = items[k];
        uint8_t *dt = dir + it.dir_off;
        bool ok;
        int32_t et, eq;
        {
            // without the deferred arg-max (DEFER): its saved registers cost
            // more here, beside the direction bits, than the searches they save
            // (measured on the ONT-like batch: 171 against 179 ms)
            WarpPair16<C, (MINB < 4 && C <= 16) || MINB < 3, false, true, true> wp(cold[threadIdx.x >> 5]);
            ok = wp.run(B, it.pair, lane, true, dt);
            et = wp.end_t;
            eq = wp.end_q;
        }
        if (!ok) {                                  // the int32 score kernel takes it
            if (lane == 0) {
                const int32_t slot = atomicAdd(&B.counters[CTR_NOVF], 1);
                B.ovf_list[slot] = it.pair;
                n_cigar[it.pair] = -1;
            }
            continue;
        }
        if (et < 0 || eq < 0) {                     // the maximum is the origin
            if (lane == 0) n_cigar[it.pair] = 0;
            continue;
        }
        __syncwarp();
        const int32_t w = effective_w(B.params.w, B.t_len[it.pair], B.q_len[it.pair]);
        const int32_t n = tb_walk<C, true>(my_win, dt, ops + it.ops_off, et + eq + 2, et, eq, w, lane);
        if (lane == 0) n_cigar[it.pair] = n;
    }
}

template <int C, int MINB>
cudaError_t launch_tbf16_c(const DevBatch *d_batch, const TbItem *items, int32_t n_items, int32_t *head,
                           uint8_t *dir, uint32_t *ops, int32_t *n_cigar, int n_blocks, cudaStream_t s) {
    tbf16_kernel<C, MINB><<<n_blocks, WARP_BLOCK_THREADS, 0, s>>>(d_batch, items, n_items, head, dir, ops,
                                                                  n_cigar);
    return cudaGetLastError();
}

template <int C, int MINB>
int occupancy_tbf16_c() {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, tbf16_kernel<C, MINB>, WARP_BLOCK_THREADS, 0) !=
        cudaSuccess)
        return 1;
    return nb > 0 ? nb : 1;
}

template <int C>
cudaError_t launch_tb_c(const DevBatch *d_batch, const TbItem *items, int32_t n_items, int32_t *head,
                        uint8_t *dir, uint32_t *ops, int32_t *n_cigar, int n_blocks, cudaStream_t s) {
    tb_kernel<C><<<n_blocks, WARP_BLOCK_THREADS, 0, s>>>(d_batch, items, n_items, head, dir, ops, n_cigar);
    return cudaGetLastError();
}

template <int C>
int occupancy_tb_c() {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, tb_kernel<C>, WARP_BLOCK_THREADS, 0) !=
        cudaSuccess)
        return 1;
    return nb > 0 ? nb : 1;
}

template <int C, int MINB>
cudaError_t launch_tb16_c(const DevBatch *d_batch, const TbItem *items, int32_t n_items, int32_t *head,
                          uint8_t *dir, uint32_t *ops, int32_t *n_cigar, int n_blocks, cudaStream_t s) {
    tb16_kernel<C, MINB><<<n_blocks, WARP_BLOCK_THREADS, 0, s>>>(d_batch, items, n_items, head, dir, ops,
                                                                 n_cigar);
    return cudaGetLastError();
}

template <int C, int MINB>
int occupancy_tb16_c() {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, tb16_kernel<C, MINB>, WARP_BLOCK_THREADS, 0) !=
        cudaSuccess)
        return 1;
    return nb > 0 ? nb : 1;
}

}  // namespace agatha
