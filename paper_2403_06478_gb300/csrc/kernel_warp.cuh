// Batched persistent kernel: one warp aligns one pair at a time, pulling pair
// indices from a device work queue ordered by predicted band cells.
//
// Layout of a pair's band in the warp: lane L owns the C consecutive slots
// j = L*C .. L*C + C - 1 (slot j is the cell t = B(r) + j of anti-diagonal r,
// see agatha_dev.cuh).  Per slot the lane keeps, in registers,
//   H of r-1 and r-2, and the gap states leaving the cells of r-1:
//   Eo = max(H - q - e, E - e)   (what cell (t+1, q) needs, paper Eq. 2)
//   Fo = max(H - q - e, F - e)   (what cell (t, q+1) needs, paper Eq. 3)
//   E2o, F2o the same with the second gap piece (q2, e2).
// One anti-diagonal is one step of the warp: every lane updates its C cells,
// the only cross-lane inputs are the E states of the left neighbour's last
// slot or the F states of the right neighbour's first slot (warp shuffles).
// The anti-diagonal maximum and its lowest t come from a warp reduction, and
// the exact termination test (Eq. 4-7) runs after every anti-diagonal, so no
// cell beyond the stopping anti-diagonal is ever computed.
//
// Steps near the table's edges (the first w+4 anti-diagonals, where virtual
// row/column cells enter, and the ones that touch t = tlen-1 or q = qlen-1)
// run a masked variant; the bulk in between runs unmasked.
//
// With DIR the same steps also record, per band slot and anti-diagonal, one
// direction byte for the traceback (kernel_tb.cuh) and run to a given end
// anti-diagonal instead of testing termination:
//   bits 0-2  which input H took: 0 diagonal, 1 E, 2 F, 3 E2, 4 F2 (the first
//             of these that equals H)
//   bits 3-6  whether Eo, Fo, E2o, F2o leaving this cell extend the cell's
//             own E, F, E2, F2 (strictly better than opening from H)
#pragma once

#include <climits>
#include <type_traits>

#include "agatha_dev.cuh"

namespace agatha {

constexpr unsigned FULL = 0xffffffffu;
constexpr int WARP_BLOCK_THREADS = 128;

template <int C>
struct WarpWin {
    using T = typename std::conditional<(C <= 16), uint32_t, uint64_t>::type;
    static constexpr T MASK = (C * 2 >= (int)sizeof(T) * 8) ? ~T(0) : ((T(1) << (2 * C)) - 1);
    static constexpr T LOW = (sizeof(T) == 4) ? T(0x55555555u) : T(0x5555555555555555ull);
};

template <int C, bool DIR = false>
struct WarpPair {
    using W = typename WarpWin<C>::T;
    static constexpr int32_t DIR_ROW = 32 * C;   // direction bytes per anti-diagonal
    // static pair data
    const uint32_t *tp, *qp;
    int64_t tw, qw, toff, qoff;
    int32_t tlen, qlen, w, last_r, lane, j0;
    DevParams P;
    int32_t oe, oe2;
    // band state (registers)
    int32_t H1[C], H2[C], Eo[C], E2o[C], Fo[C], F2o[C];
    // base windows: Tw field jl = T[B + j0 + jl], Qw field jl = Q[r - B - j0 - jl]
    W Tw, Qw;
    uint32_t Tpf, Qpf;       // next 16 bases to shift in
    int32_t tcnt, qcnt;      // bases left in Tpf / Qpf
    int64_t tpos, qpos;      // base index of the next refill
    // anti-diagonal bookkeeping (uniform across the warp)
    int32_t gmax, gt, gq, mqe, mqe_t, mte, mte_q, gscore;
    int64_t cells;
    int32_t zdropped;
    uint8_t *dtab;           // DIR: this lane's bytes of anti-diagonal 0

    // DIR: the direction byte of one cell (see the top of this file)
    __device__ __forceinline__ uint32_t dir_bits(int32_t hd, int32_t Ein, int32_t Fin, int32_t E2in,
                                                 int32_t F2in, int32_t H, int32_t hoe,
                                                 int32_t hoe2) const {
        uint32_t b = H == hd ? 0u : (H == Ein ? 1u : (H == Fin ? 2u : (H == E2in ? 3u : 4u)));
        b |= (Ein - P.e > hoe) ? 8u : 0u;
        b |= (Fin - P.e > hoe) ? 16u : 0u;
        b |= (E2in - P.e2 > hoe2) ? 32u : 0u;
        b |= (F2in - P.e2 > hoe2) ? 64u : 0u;
        return b;
    }

    // DIR: this lane's C bytes of anti-diagonal r, one aligned vector store
    __device__ __forceinline__ void store_dir(int32_t r, const uint32_t (&wd)[C / 4]) const {
        uint8_t *p = dtab + (int64_t)r * DIR_ROW;
        if constexpr (C % 16 == 0) {
#pragma unroll
            for (int k = 0; k < C / 16; ++k)
                reinterpret_cast<uint4 *>(p)[k] = make_uint4(wd[4 * k], wd[4 * k + 1], wd[4 * k + 2], wd[4 * k + 3]);
        } else if constexpr (C % 8 == 0) {
#pragma unroll
            for (int k = 0; k < C / 8; ++k)
                reinterpret_cast<uint2 *>(p)[k] = make_uint2(wd[2 * k], wd[2 * k + 1]);
        } else {
            *reinterpret_cast<uint32_t *>(p) = wd[0];
        }
    }

    __device__ __forceinline__ void init_windows(int32_t r) {
        const int32_t B = ceil_div2(r - w);
        const int64_t tb = (int64_t)B + j0;
        const int64_t qb = (int64_t)r - B - j0;
        if constexpr (C <= 16) {
            Tw = load16(tp, tw, toff + tb) & WarpWin<C>::MASK;
            uint32_t nat = load16(qp, qw, qoff + qb - C + 1);
            Qw = rev2_32(nat) >> (2 * (16 - C));
        } else {
            Tw = load32(tp, tw, toff + tb) & WarpWin<C>::MASK;
            uint64_t nat = load32(qp, qw, qoff + qb - C + 1);
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

    // Move the base windows from anti-diagonal r-1 to r.  When (r - w) is odd
    // B(r) = B(r-1) + 1 and the target window slides; otherwise the query
    // window does.
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

    // Global max update, else the Z-drop test (Eq. 4-7).  Returns true to stop.
    __device__ __forceinline__ bool max_and_zdrop(int32_t m, int32_t tstar, int32_t r) {
        const int32_t qstar = r - tstar;
        if (m > gmax) {
            gmax = m; gt = tstar; gq = qstar;
            return false;
        }
        if (tstar >= gt && qstar >= gq && P.zdrop >= 0) {
            int32_t l = (tstar - gt) - (qstar - gq);
            l = l < 0 ? -l : l;
            if (gmax - m > P.zdrop + l * P.e2) return true;
        }
        return false;
    }

    // Lowest-t argmax of the anti-diagonal from per-lane (max, first index).
    __device__ __forceinline__ void warp_argmax(int32_t lm, int32_t li, int32_t B, int32_t &m,
                                                int32_t &tstar) const {
        m = __reduce_max_sync(FULL, lm);
        unsigned ball = __ballot_sync(FULL, lm == m && li >= 0);
        int src = __ffs(ball) - 1;
        int32_t lj = __shfl_sync(FULL, li, src);
        tstar = B + src * C + lj;
    }

    // One anti-diagonal with every edge case handled per cell.
    __device__ __forceinline__ bool masked_step(int32_t r) {
        const int32_t B = ceil_div2(r - w);
        const int32_t d = (r - w) & 1;
        if (!DIR && r >= 0) {
            const int32_t st = max(max(0, r - qlen + 1), B);
            const int32_t en = min(min(tlen - 1, r), floor_div2(r + w));
            if (st > en) { zdropped = 1; return true; }    // the band left the table
            cells += en - st + 1;
        }
        // cross-lane neighbours
        int32_t eL = __shfl_up_sync(FULL, Eo[C - 1], 1);
        int32_t e2L = __shfl_up_sync(FULL, E2o[C - 1], 1);
        int32_t fR = __shfl_down_sync(FULL, Fo[0], 1);
        int32_t f2R = __shfl_down_sync(FULL, F2o[0], 1);
        if (lane == 0) {
            // slot -1 of r-1 is cell (B-1, r-B): a virtual row cell only when B == 0
            const int32_t ts = B - 1, qs = r - B;
            if (ts == -1 && qs >= -1 && qs < qlen) {
                const int32_t v = (qs == -1) ? 0 : -gap_cost(P, qs + 1);
                eL = v - oe; e2L = v - oe2;
            } else {
                eL = K_NEG; e2L = K_NEG;
            }
        }
        if (lane == 31) { fR = K_NEG; f2R = K_NEG; }
        const W x = Tw ^ Qw;
        const W nm = (x | (x >> 1)) & WarpWin<C>::LOW;     // bit 2*jl: mismatch
        int32_t nH[C], nE[C], nE2[C], nF[C], nF2[C];
        uint32_t wd[C / 4];
#pragma unroll
        for (int k = 0; k < C / 4; ++k) wd[k] = 0;
        int32_t lm = INT_MIN, li = -1, te_c = INT_MIN, qe_c = INT_MIN;
#pragma unroll
        for (int jl = 0; jl < C; ++jl) {
            const int32_t t = B + j0 + jl;
            const int32_t q = r - t;
            const int32_t Ein = d ? Eo[jl] : (jl ? Eo[jl - 1] : eL);
            const int32_t E2in = d ? E2o[jl] : (jl ? E2o[jl - 1] : e2L);
            const int32_t Fin = d ? (jl < C - 1 ? Fo[jl + 1] : fR) : Fo[jl];
            const int32_t F2in = d ? (jl < C - 1 ? F2o[jl + 1] : f2R) : F2o[jl];
            const int32_t s = ((nm >> (2 * jl)) & 1) ? -P.b : P.a;
            int32_t H = max(max(H2[jl] + s, Ein), max(max(Fin, E2in), F2in));
            int32_t hoe = H - oe, hoe2 = H - oe2;
            int32_t ne = max(hoe, Ein - P.e), nf = max(hoe, Fin - P.e);
            int32_t ne2 = max(hoe2, E2in - P.e2), nf2 = max(hoe2, F2in - P.e2);
            if constexpr (DIR)
                wd[jl >> 2] |= dir_bits(H2[jl] + s, Ein, Fin, E2in, F2in, H, hoe, hoe2) << (8 * (jl & 3));
            const int32_t k = t - q;
            const bool real = t >= 0 && q >= 0 && t < tlen && q < qlen && k <= w && -k <= w;
            if (real) {
                if (H > lm) { lm = H; li = jl; }
                if (t == tlen - 1) te_c = H;
                if (q == qlen - 1) qe_c = H;
            } else {
                const bool virt = (t == -1 && q >= -1 && q < qlen) || (q == -1 && t >= 0 && t < tlen);
                if (virt) {
                    const int32_t v = (t == -1 && q == -1) ? 0 : -gap_cost(P, (t == -1 ? q : t) + 1);
                    H = v; ne = nf = v - oe; ne2 = nf2 = v - oe2;
                } else {
                    H = K_NEG; ne = nf = ne2 = nf2 = K_NEG;
                }
            }
            nH[jl] = H; nE[jl] = ne; nE2[jl] = ne2; nF[jl] = nf; nF2[jl] = nf2;
        }
#pragma unroll
        for (int jl = 0; jl < C; ++jl) {
            H2[jl] = H1[jl]; H1[jl] = nH[jl];
            Eo[jl] = nE[jl]; E2o[jl] = nE2[jl]; Fo[jl] = nF[jl]; F2o[jl] = nF2[jl];
        }
        if (r < 0) return false;
        if constexpr (DIR) {
            store_dir(r, wd);
            return false;
        }
        // last target row / last query column
        const int32_t te_v = __reduce_max_sync(FULL, te_c);
        if (te_v != INT_MIN && te_v > mte) { mte = te_v; mte_q = r - (tlen - 1); }
        const int32_t qe_v = __reduce_max_sync(FULL, qe_c);
        if (qe_v != INT_MIN && qe_v > mqe) { mqe = qe_v; mqe_t = r - (qlen - 1); }
        int32_t m, tstar;
        warp_argmax(lm, li, B, m, tstar);
        if (max_and_zdrop(m, tstar, r)) { zdropped = 1; return true; }
        if (r == last_r && te_v != INT_MIN && (r - (tlen - 1)) == qlen - 1) gscore = te_v;
        return false;
    }

    // One bulk anti-diagonal: every band cell is a real cell away from the last
    // row/column, so only the band's own edges need care.  D = (r - w) & 1.
    template <int D>
    __device__ __forceinline__ bool fast_step(int32_t r, int32_t vcnt) {
        const int32_t B = ceil_div2(r - w);
        int32_t eL = 0, e2L = 0, fR = 0, f2R = 0;
        if constexpr (D == 0) {
            eL = __shfl_up_sync(FULL, Eo[C - 1], 1);
            e2L = __shfl_up_sync(FULL, E2o[C - 1], 1);
            if (lane == 0) { eL = K_NEG; e2L = K_NEG; }
        } else {
            fR = __shfl_down_sync(FULL, Fo[0], 1);
            f2R = __shfl_down_sync(FULL, F2o[0], 1);
            if (lane == 31) { fR = K_NEG; f2R = K_NEG; }
        }
        const W x = Tw ^ Qw;
        const W nm = (x | (x >> 1)) & WarpWin<C>::LOW;
        int32_t nH[C], nE[C], nE2[C], nF[C], nF2[C];
        uint32_t wd[C / 4];
#pragma unroll
        for (int k = 0; k < C / 4; ++k) wd[k] = 0;
        int32_t lm = INT_MIN, li = -1;
#pragma unroll
        for (int jl = 0; jl < C; ++jl) {
            const int32_t Ein = D ? Eo[jl] : (jl ? Eo[jl - 1] : eL);
            const int32_t E2in = D ? E2o[jl] : (jl ? E2o[jl - 1] : e2L);
            const int32_t Fin = D ? (jl < C - 1 ? Fo[jl + 1] : fR) : Fo[jl];
            const int32_t F2in = D ? (jl < C - 1 ? F2o[jl + 1] : f2R) : F2o[jl];
            const int32_t s = ((nm >> (2 * jl)) & 1) ? -P.b : P.a;
            const int32_t H = max(max(H2[jl] + s, Ein), max(max(Fin, E2in), F2in));
            const bool valid = jl < vcnt;
            // slots outside the band keep their F states at -inf so nothing
            // flows back into the band; their E states only flow further out
            const int32_t hoe = valid ? H - oe : K_NEG;
            const int32_t hoe2 = valid ? H - oe2 : K_NEG;
            if constexpr (DIR)
                wd[jl >> 2] |= dir_bits(H2[jl] + s, Ein, Fin, E2in, F2in, H, hoe, hoe2) << (8 * (jl & 3));
            nE[jl] = max(hoe, Ein - P.e);
            nF[jl] = max(hoe, Fin - P.e);
            nE2[jl] = max(hoe2, E2in - P.e2);
            nF2[jl] = max(hoe2, F2in - P.e2);
            nH[jl] = H;
            if (valid && H > lm) { lm = H; li = jl; }
        }
#pragma unroll
        for (int jl = 0; jl < C; ++jl) {
            H2[jl] = H1[jl]; H1[jl] = nH[jl];
            Eo[jl] = nE[jl]; E2o[jl] = nE2[jl]; Fo[jl] = nF[jl]; F2o[jl] = nF2[jl];
        }
        if constexpr (DIR) {
            store_dir(r, wd);
            return false;
        }
        cells += w + 1 - D;
        int32_t m, tstar;
        warp_argmax(lm, li, B, m, tstar);
        if (max_and_zdrop(m, tstar, r)) { zdropped = 1; return true; }
        return false;
    }

    __device__ __forceinline__ void run(const DevBatch &Bt, int32_t pair, int32_t lane_, bool use_fast) {
        P = Bt.params;
        lane = lane_;
        tp = Bt.t_packed; qp = Bt.q_packed; tw = Bt.t_words; qw = Bt.q_words;
        tlen = Bt.t_len[pair]; qlen = Bt.q_len[pair];
        toff = Bt.t_off[pair]; qoff = Bt.q_off[pair];
        agatha_result *out = Bt.out + pair;
        if (tlen <= 0 || qlen <= 0) {
            if (lane == 0) write_empty_result(out);
            return;
        }
        w = effective_w(P.w, tlen, qlen);
        oe = P.q + P.e; oe2 = P.q2 + P.e2;
        j0 = lane * C;
        last_r = tlen + qlen - 2;
#pragma unroll
        for (int i = 0; i < C; ++i) { H1[i] = H2[i] = Eo[i] = E2o[i] = Fo[i] = F2o[i] = K_NEG; }
        gmax = 0; gt = -1; gq = -1;
        mqe = K_NEG_OUT; mqe_t = -1; mte = K_NEG_OUT; mte_q = -1; gscore = K_NEG_OUT;
        cells = 0; zdropped = 0;

        int32_t r = -2;
        init_windows(r);
        bool stop = masked_step(r);
        const int32_t head_end = min(last_r, w + 1);
        while (!stop && r < head_end) {
            ++r;
            if ((r - w) & 1) shift_t(); else shift_q();
            stop = masked_step(r);
        }
        // bulk: pairs of anti-diagonals (even, odd) starting at r = w + 2
        const int32_t L = min(tlen, qlen);
        const int32_t bulk_last = 2 * L - 3 - w;
        if (use_fast && !stop && r == w + 1) {
            const int32_t vcnt0 = max(0, min(C, w + 1 - j0));
            const int32_t vcnt1 = max(0, min(C, w - j0));
            while (r + 2 <= bulk_last) {
                ++r; shift_q();
                if (fast_step<0>(r, vcnt0)) { stop = true; break; }
                ++r; shift_t();
                if (fast_step<1>(r, vcnt1)) { stop = true; break; }
            }
        }
        while (!stop && r < last_r) {
            ++r;
            if ((r - w) & 1) shift_t(); else shift_q();
            stop = masked_step(r);
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

    // DIR: anti-diagonals 0..r_end of a pair with its direction bytes in
    // dt[r * DIR_ROW + slot] (no termination test: r_end is known).
    __device__ __forceinline__ void run_dir(const DevBatch &Bt, int32_t pair, int32_t lane_,
                                            int32_t r_end, uint8_t *dt) {
        static_assert(DIR, "run_dir needs the direction variant");
        P = Bt.params;
        lane = lane_;
        tp = Bt.t_packed; qp = Bt.q_packed; tw = Bt.t_words; qw = Bt.q_words;
        tlen = Bt.t_len[pair]; qlen = Bt.q_len[pair];
        toff = Bt.t_off[pair]; qoff = Bt.q_off[pair];
        w = effective_w(P.w, tlen, qlen);
        oe = P.q + P.e; oe2 = P.q2 + P.e2;
        j0 = lane * C;
        last_r = r_end;
        dtab = dt + j0;
#pragma unroll
        for (int i = 0; i < C; ++i) { H1[i] = H2[i] = Eo[i] = E2o[i] = Fo[i] = F2o[i] = K_NEG; }
        cells = 0; zdropped = 0;
        int32_t r = -2;
        init_windows(r);
        masked_step(r);
        const int32_t head_end = min(last_r, w + 1);
        while (r < head_end) {
            ++r;
            if ((r - w) & 1) shift_t(); else shift_q();
            masked_step(r);
        }
        const int32_t L = min(tlen, qlen);
        const int32_t bulk_last = min(2 * L - 3 - w, last_r);
        if (r == w + 1) {
            const int32_t vcnt0 = max(0, min(C, w + 1 - j0));
            const int32_t vcnt1 = max(0, min(C, w - j0));
            while (r + 2 <= bulk_last) {
                ++r; shift_q();
                fast_step<0>(r, vcnt0);
                ++r; shift_t();
                fast_step<1>(r, vcnt1);
            }
        }
        while (r < last_r) {
            ++r;
            if ((r - w) & 1) shift_t(); else shift_q();
            masked_step(r);
        }
    }
};

// Pairs the warp kernel takes: valid and narrow enough for 32*C slots.
__device__ __forceinline__ bool warp_takes(const DevBatch &B, int32_t pair) {
    const int32_t tl = B.t_len[pair], ql = B.q_len[pair];
    const int32_t w = effective_w(B.params.w, tl, ql);
    return w <= B.warp_w_max && (B.narrow_w_max <= 0 || w > B.narrow_w_max);
}

template <int C>
__global__ void __launch_bounds__(WARP_BLOCK_THREADS)
warp_align_kernel(const DevBatch *__restrict__ d_batch, int32_t use_fast, int32_t list) {
    const DevBatch B = *d_batch;
    const int lane = threadIdx.x & 31;
    const WorkList L = work_list(B, list);
    for (;;) {
        int32_t k = 0;
        if (lane == 0) k = L.begin + atomicAdd(L.head, 1);
        k = __shfl_sync(FULL, k, 0);
        if (k >= L.end) break;
        const int32_t pair = L.items ? L.items[k] : k;
        if (!L.items && (!pair_valid(B, pair) || !warp_takes(B, pair))) continue;
        WarpPair<C> wp;
        wp.run(B, pair, lane, use_fast != 0);
    }
    if (lane == 0) mark_step_end(B.counters);
}

template <int C>
cudaError_t launch_warp_c(const DevBatch *d_batch, int n_blocks, cudaStream_t s, int use_fast,
                          int list) {
    warp_align_kernel<C><<<n_blocks, WARP_BLOCK_THREADS, 0, s>>>(d_batch, use_fast, list);
    return cudaGetLastError();
}

template <int C>
int occupancy_warp_c() {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, warp_align_kernel<C>,
                                                      WARP_BLOCK_THREADS, 0) != cudaSuccess)
        return 1;
    return nb > 0 ? nb : 1;
}

}  // namespace agatha
