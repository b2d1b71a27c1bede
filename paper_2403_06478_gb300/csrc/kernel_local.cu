// Local extension from an initial score: the BWA-MEM variant of the
// extension (the paper applies its kernel to BWA-MEM's guided alignment,
// Section 5.9).  The rules are this library's reading of BWA-MEM's published
// extension, stated in include/agatha.h beside agatha_align_batch_local:
//   - the origin holds the seed's score h0 > 0 and the virtual row and column
//     h0 - gap(l), kept only while positive;
//   - a path is kept only while its score stays positive: every state is
//     floored at 0 and a diagonal step out of an empty cell (H = 0) stays
//     empty;
//   - the termination test runs one query row at a time: the row's best cell
//     (lowest t on ties) becomes the best so far when strictly higher, else
//     the Z-drop test may stop the extension; a row without a positive cell
//     ends it.
//
// One warp aligns one pair on int32 lanes, in the same anti-diagonal frame as
// the int32 score kernel (lane L owns slots L*C .. L*C + C - 1 of the band,
// slot j being cell t = B(r) + j with B(r) = ceil((r - w) / 2)), every
// anti-diagonal through one per-cell step that classifies each slot as a band
// cell, a virtual cell or nothing.  The rows are handled without leaving the
// frame: a row q is the cells (t, q) for increasing t, which is exactly the
// way the E state travels (from (t-1, q) to (t, q)), so two more states ride
// along with E: the row's best score so far (RM) and its lowest t (RT).  A
// row is complete on the anti-diagonal of its last band cell,
// t = min(tlen - 1, q + w); at most one row completes per anti-diagonal, in
// increasing q, and its best is then read from the slot of that cell.  The
// cells past the completing row that the frame has already computed (up to w
// anti-diagonals ahead) are dropped with it when the extension stops there.
#include <climits>

#include "kernel_warp.cuh"

namespace agatha {

template <int C>
struct LocalPair {
    using W = typename WarpWin<C>::T;
    const uint32_t *tp, *qp;
    int64_t tw, qw, toff, qoff;
    int32_t tlen, qlen, w, lane, j0, h0;
    DevParams P;
    int32_t oe, oe2;
    // band state: H of r-1 and r-2, the gap states leaving r-1 (floored at
    // 0: 0 is "no live path"), and the row accumulators leaving r-1 (RM = -1:
    // no cell of the row yet)
    int32_t H1[C], H2[C], Eo[C], E2o[C], Fo[C], F2o[C], RM[C], RT[C];
    W Tw, Qw;
    uint32_t Tpf, Qpf;
    int32_t tcnt, qcnt;
    int64_t tpos, qpos;
    // rows (uniform across the warp)
    int32_t gmax, gt, gq, mqe, mqe_t, mte, mte_q, gscore;
    int64_t cells;
    int32_t zdropped;

    __device__ __forceinline__ static int32_t pos(int32_t x) { return x > 0 ? x : 0; }

    __device__ __forceinline__ void init_windows(int32_t r) {
        const int32_t B = ceil_div2(r - w);
        const int64_t tb = (int64_t)B + j0;
        const int64_t qb = (int64_t)r - B - j0;
        if constexpr (C <= 16) {
            Tw = load16(tp, tw, toff + tb) & WarpWin<C>::MASK;
            const uint32_t nat = load16(qp, qw, qoff + qb - C + 1);
            Qw = rev2_32(nat) >> (2 * (16 - C));
        } else {
            Tw = load32(tp, tw, toff + tb) & WarpWin<C>::MASK;
            const uint64_t nat = load32(qp, qw, qoff + qb - C + 1);
            Qw = rev2_64(nat) >> (2 * (32 - C));
        }
        tpos = tb + C;
        qpos = qb + 1;
        Tpf = load16(tp, tw, toff + tpos);
        Qpf = load16(qp, qw, qoff + qpos);
        tpos += 16;
        qpos += 16;
        tcnt = 16;
        qcnt = 16;
    }
    __device__ __forceinline__ void shift_t() {
        Tw = (Tw >> 2) | ((W)(Tpf & 3u) << (2 * C - 2));
        Tpf >>= 2;
        if (--tcnt == 0) {
            Tpf = load16(tp, tw, toff + tpos);
            tpos += 16;
            tcnt = 16;
        }
    }
    __device__ __forceinline__ void shift_q() {
        Qw = ((Qw << 2) | (W)(Qpf & 3u)) & WarpWin<C>::MASK;
        Qpf >>= 2;
        if (--qcnt == 0) {
            Qpf = load16(qp, qw, qoff + qpos);
            qpos += 16;
            qcnt = 16;
        }
    }

    // value of the virtual cell (t, q) (t == -1 or q == -1), 0 when no path
    // with a positive score reaches it
    __device__ __forceinline__ int32_t virtual_H(int32_t t, int32_t q) const {
        if (t == -1 && q == -1) return h0;
        return pos(h0 - gap_cost(P, (t == -1 ? q : t) + 1));
    }

    // One anti-diagonal; then, if a row completes on it, that row's rules.
    // Returns true when the extension ends (stop or last row done).
    __device__ __forceinline__ bool step(int32_t r) {
        const int32_t B = ceil_div2(r - w);
        const int32_t d = (r - w) & 1;
        // the slot below lane 0 (cell (B-1, r-B) of r-1): a virtual row cell
        // only when B == 0; its E states and an empty row accumulator
        int32_t eL = __shfl_up_sync(FULL, Eo[C - 1], 1);
        int32_t e2L = __shfl_up_sync(FULL, E2o[C - 1], 1);
        int32_t rmL = __shfl_up_sync(FULL, RM[C - 1], 1);
        int32_t rtL = __shfl_up_sync(FULL, RT[C - 1], 1);
        int32_t fR = __shfl_down_sync(FULL, Fo[0], 1);
        int32_t f2R = __shfl_down_sync(FULL, F2o[0], 1);
        if (lane == 0) {
            const int32_t ts = B - 1, qs = r - B;
            if (ts == -1 && qs >= -1 && qs < qlen) {
                const int32_t v = virtual_H(ts, qs);
                eL = pos(v - oe);
                e2L = pos(v - oe2);
            } else {
                eL = 0;
                e2L = 0;
            }
            rmL = -1;
            rtL = -1;
        }
        if (lane == 31) { fR = 0; f2R = 0; }
        const W x = Tw ^ Qw;
        const W nm = (x | (x >> 1)) & WarpWin<C>::LOW;     // bit 2*jl: mismatch
        int32_t nH[C], nE[C], nE2[C], nF[C], nF2[C], nRM[C], nRT[C];
#pragma unroll
        for (int jl = 0; jl < C; ++jl) {
            const int32_t t = B + j0 + jl;
            const int32_t q = r - t;
            const int32_t Ein = d ? Eo[jl] : (jl ? Eo[jl - 1] : eL);
            const int32_t E2in = d ? E2o[jl] : (jl ? E2o[jl - 1] : e2L);
            const int32_t RMin = d ? RM[jl] : (jl ? RM[jl - 1] : rmL);
            const int32_t RTin = d ? RT[jl] : (jl ? RT[jl - 1] : rtL);
            const int32_t Fin = d ? (jl < C - 1 ? Fo[jl + 1] : fR) : Fo[jl];
            const int32_t F2in = d ? (jl < C - 1 ? F2o[jl + 1] : f2R) : F2o[jl];
            const int32_t s = ((nm >> (2 * jl)) & 1) ? -P.b : P.a;
            const int32_t k = t - q;
            const bool real = t >= 0 && q >= 0 && t < tlen && q < qlen && k <= w && -k <= w;
            int32_t H, ne, ne2, nf, nf2, rm = -1, rt = -1;
            if (real) {
                const int32_t Hd = H2[jl];               // H(t-1, q-1)
                H = Hd > 0 ? pos(Hd + s) : 0;
                H = max(max(H, Ein), max(max(Fin, E2in), F2in));
                ne = pos(max(H - oe, Ein - P.e));
                nf = pos(max(H - oe, Fin - P.e));
                ne2 = pos(max(H - oe2, E2in - P.e2));
                nf2 = pos(max(H - oe2, F2in - P.e2));
                // the row's best so far: strictly higher keeps the lowest t
                if (H > RMin) { rm = H; rt = t; } else { rm = RMin; rt = RTin; }
            } else if ((t == -1 && q >= -1 && q < qlen) || (q == -1 && t >= 0 && t < tlen)) {
                H = virtual_H(t, q);
                ne = nf = pos(H - oe);
                ne2 = nf2 = pos(H - oe2);
            } else {
                H = 0;
                ne = nf = ne2 = nf2 = 0;
            }
            nH[jl] = H; nE[jl] = ne; nE2[jl] = ne2; nF[jl] = nf; nF2[jl] = nf2; nRM[jl] = rm; nRT[jl] = rt;
        }
#pragma unroll
        for (int jl = 0; jl < C; ++jl) {
            H2[jl] = H1[jl]; H1[jl] = nH[jl];
            Eo[jl] = nE[jl]; E2o[jl] = nE2[jl]; Fo[jl] = nF[jl]; F2o[jl] = nF2[jl];
            RM[jl] = nRM[jl]; RT[jl] = nRT[jl];
        }
        if (r < 0) return false;
        // the row completing on r: its last band cell t = min(tlen-1, q+w) has
        // t + q = r (2q + w = r while q + w < tlen, then q = r - tlen + 1)
        int32_t qc = -1;
        if (((r - w) & 1) == 0) {
            const int32_t qa = (r - w) >> 1;
            if (qa >= 0 && qa < qlen && qa + w < tlen - 1) qc = qa;
        }
        {
            const int32_t qb = r - tlen + 1;
            if (qb >= 0 && qb < qlen && qb + w >= tlen - 1) qc = qb;
        }
        if (qc < 0) return false;
        const int32_t tl = min(tlen - 1, qc + w);
        const int32_t tf = max(0, qc - w);
        // read its row accumulator and H at the slot of (tl, qc)
        const int32_t j = tl - B, owner = j / C, loc = j - owner * C;
        int32_t v_rm = RM[0], v_rt = RT[0], v_h = H1[0];
#pragma unroll
        for (int jl = 1; jl < C; ++jl) {
            if (loc == jl) { v_rm = RM[jl]; v_rt = RT[jl]; v_h = H1[jl]; }
        }
        const int32_t row = __shfl_sync(FULL, v_rm, owner);
        const int32_t row_t = __shfl_sync(FULL, v_rt, owner);
        const int32_t h_end = __shfl_sync(FULL, v_h, owner);
        cells += tl - tf + 1;
        if (tl == tlen - 1 && h_end > 0 && h_end > mte) { mte = h_end; mte_q = qc; }
        if (qc == qlen - 1 && row > 0) { mqe = row; mqe_t = row_t; }
        if (row <= 0) { zdropped = 1; return true; }          // no live cell left
        if (row > gmax) {
            gmax = row; gt = row_t; gq = qc;
        } else if (P.zdrop >= 0) {
            int32_t l = (qc - gq) - (row_t - gt);
            l = l < 0 ? -l : l;
            if (gmax - row > P.zdrop + l * P.e2) { zdropped = 1; return true; }
        }
        if (qc == qlen - 1) {
            if (tl == tlen - 1 && h_end > 0) gscore = h_end;
            return true;                                      // every row done
        }
        if (qc + 1 - w > tlen - 1) { zdropped = 1; return true; }   // the next row has no band cell
        return false;
    }

    __device__ __forceinline__ void run(const DevBatch &Bt, int32_t pair, int32_t lane_) {
        P = Bt.params;
        lane = lane_;
        tp = Bt.t_packed; qp = Bt.q_packed; tw = Bt.t_words; qw = Bt.q_words;
        tlen = Bt.t_len[pair]; qlen = Bt.q_len[pair];
        toff = Bt.t_off[pair]; qoff = Bt.q_off[pair];
        h0 = Bt.h0[pair];
        agatha_result *out = Bt.out + pair;
        gmax = h0; gt = -1; gq = -1;
        mqe = K_NEG_OUT; mqe_t = -1; mte = K_NEG_OUT; mte_q = -1; gscore = K_NEG_OUT;
        cells = 0; zdropped = 0;
        if (tlen > 0 && qlen > 0) {
            w = effective_w(P.w, tlen, qlen);
            oe = P.q + P.e; oe2 = P.q2 + P.e2;
            j0 = lane * C;
#pragma unroll
            for (int i = 0; i < C; ++i) {
                H1[i] = H2[i] = Eo[i] = E2o[i] = Fo[i] = F2o[i] = 0;
                RM[i] = RT[i] = -1;
            }
            // the last row completes on anti-diagonal tlen + qlen - 2 at the latest
            const int32_t last_r = tlen + qlen - 2;
            int32_t r = -2;
            init_windows(r);
            bool stop = step(r);
            while (!stop && r < last_r) {
                ++r;
                if ((r - w) & 1) shift_t(); else shift_q();
                stop = step(r);
            }
        }
        if (lane == 0) {
            agatha_result o;
            o.max = gmax; o.te = gt; o.qe = gq;
            o.gscore = gscore; o.mqe = mqe; o.mqe_t = mqe_t; o.mte = mte; o.mte_q = mte_q;
            o.cells = cells;
            o.zdropped = (uint8_t)zdropped;
            o.reach_end = (uint8_t)(!zdropped && mqe != K_NEG_OUT && mqe + P.end_bonus > gmax);
            o.lane16 = 0;
            for (int i = 0; i < 5; ++i) o.pad[i] = 0;
            *out = o;
        }
    }
};

template <int C>
__global__ void __launch_bounds__(WARP_BLOCK_THREADS)
local_align_kernel(const DevBatch *__restrict__ d_batch) {
    const DevBatch B = *d_batch;
    const int lane = threadIdx.x & 31;
    const WorkList L = work_list(B, WARP_LIST_MAIN);
    for (;;) {
        int32_t k = 0;
        if (lane == 0) k = L.begin + atomicAdd(L.head, 1);
        k = __shfl_sync(FULL, k, 0);
        if (k >= L.end) break;
        const int32_t pair = L.items ? L.items[k] : k;
        if (!L.items && (!pair_valid(B, pair) || !warp_takes(B, pair))) continue;
        const int32_t h0 = B.h0[pair];
        if (h0 < 1 || h0 > LOCAL_H0_MAX) {          // an initial score outside the supported range
            if (lane == 0) {
                atomicExch(&B.counters[CTR_ERR], DEV_ERR_BAD_PAIR);
                write_empty_result(B.out + pair);
            }
            continue;
        }
        LocalPair<C> lp;
        lp.run(B, pair, lane);
    }
    if (lane == 0) mark_step_end(B.counters);
}

// C = 4, 8 or 16 slots per lane (bands up to 511; the state of wider ones
// would not fit the registers)
cudaError_t launch_local(int C, const DevBatch *d_batch, int n_blocks, cudaStream_t s) {
    switch (C) {
        case 4: local_align_kernel<4><<<n_blocks, WARP_BLOCK_THREADS, 0, s>>>(d_batch); break;
        case 8: local_align_kernel<8><<<n_blocks, WARP_BLOCK_THREADS, 0, s>>>(d_batch); break;
        case 16: local_align_kernel<16><<<n_blocks, WARP_BLOCK_THREADS, 0, s>>>(d_batch); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

int local_occupancy(int C) {
    int nb = 0;
    cudaError_t e;
    switch (C) {
        case 4: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, local_align_kernel<4>, WARP_BLOCK_THREADS, 0); break;
        case 8: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, local_align_kernel<8>, WARP_BLOCK_THREADS, 0); break;
        default: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, local_align_kernel<16>, WARP_BLOCK_THREADS, 0); break;
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return nb > 0 ? nb : 1;
}

}  // namespace agatha
