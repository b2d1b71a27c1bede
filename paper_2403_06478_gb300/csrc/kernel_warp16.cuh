// Batched persistent kernel on 16-bit packed lanes: one warp aligns one pair
// (or 2 or 4 warps share one pair's band, or each half warp aligns its own
// pair), two band slots per 32-bit register, so one integer instruction
// updates two cells of the anti-diagonal.
//
// Frame.  Anti-diagonal r holds the band cells t in [ceil((r-w)/2),
// floor((r+w)/2)].  This kernel numbers them by the slot j = t - B(r) with
// B(r) = floor((r - w) / 2):
//   (r - w) even: slots 0..w are band cells; E comes from slot j of r-1,
//                 F from slot j+1 of r-1, and the target window slides;
//   (r - w) odd:  slots 1..w are band cells (slot 0 is t - q = -w-1); E comes
//                 from slot j-1, F from slot j, and the query window slides;
//   the diagonal predecessor is always the same slot two anti-diagonals back.
// So the only slot outside the band inside [0, w] is slot 0 on odd
// anti-diagonals, which belongs to lane 0 at a fixed place.
//
// Packing: register p of a lane holds slot j0+p in its low half and slot
// j0+p+P in its high half (P = C/2).  Scores are stored as unsigned 16-bit
// values u = v - base + OFF with a per-warp int32 base:
//   - NEG (0x1000) stands for minus infinity;
//   - D = the largest change one anti-diagonal can make (max of a, b, q+e,
//     q2+e2).  At most every K anti-diagonals the warp rebases: base moves to
//     the current anti-diagonal maximum (stored at OFF) and the warp checks,
//     exactly, that every score of a band cell is at least (K+3)D above NEG.
//     Between rebases scores then stay in [NEG + 2D, OFF + (K+1)D], clear of
//     NEG and of 0xFFFF.  K is as large as a score spread of 32,768 inside
//     the band allows (570 anti-diagonals for D = 25).  A pair that fails the
//     check is handed to the int32 kernel, which recomputes it from the
//     start; no 16-bit result is written for it.
//   - Real scores never come near 0 or 0xFFFF, so packed 32-bit adds and
//     subtracts never carry or borrow across the two halves (a borrow out of a
//     slot beyond the band can only reach the high half, which is then beyond
//     the band as well).
//
// Per packed register (two cells) the bulk step issues: a shift and a mask of
// the step's mismatch word and one multiply-add for the substitution, one
// add-max, one three-input max and one max for H, one 16x2 add-max for each
// of the four gap states, and half a three-input max for the anti-diagonal
// maximum.  Slots outside the band keep their outgoing gap states at NEG
// through a per-slot mask, so nothing flows back into the band.
// The registers are updated in place: F-from-j+1 steps walk the registers
// upwards and E-from-j-1 steps downwards, so every old value is read before it
// is overwritten and no copies are needed.  Anti-diagonals where the band meets
// the table's edges run the same packed update with per-slot masks (the head
// of the table, where the virtual row and column enter, runs the bulk or the
// tail step wherever their values follow from the recurrence itself).
#pragma once

#include <climits>
#include <type_traits>

#include "kernel_warp.cuh"

namespace agatha {

constexpr uint32_t U_NEG = 0x1000u;     // minus infinity of the 16-bit lanes
constexpr int32_t U_SPREAD = 32768;     // score spread inside the band the lanes keep

// Anti-diagonals between rebases for a step change of at most D: as many as
// leave U_SPREAD between the lowest band score allowed and the rebased maximum.
__host__ __device__ inline int32_t rebase_interval(int32_t D) {
    int32_t k = (int32_t)(0xffff - U_NEG - U_SPREAD) / (2 * D) - 3;
    k = k < 16 ? 16 : (k > 4096 ? 4096 : k);
    return k & ~1;
}

__device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t b, uint32_t sel) {
    uint32_t d;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(sel));
    return d;
}
// Sign of each 16-bit half of (a - b) replicated over the half, computed
// where it is used: a mask that is cheaper to recompute than to keep in a
// register across the anti-diagonal loop.
__device__ __forceinline__ uint32_t half_sign_of_diff(uint32_t a, uint32_t b) {
    uint32_t d;
    asm volatile("{\n\t.reg .b32 t;\n\tsub.u32 t, %1, %2;\n\tprmt.b32 %0, t, 0, 0xbb99;\n\t}"
                 : "=r"(d) : "r"(a), "r"(b));
    return d;
}

// bits of x where m is set, bits of y elsewhere
__device__ __forceinline__ uint32_t mux(uint32_t m, uint32_t x, uint32_t y) {
    return (m & x) | (~m & y);
}

struct Cold16 {
    int32_t mqe, mqe_t, mte, mte_q, gscore;
    int32_t gt, gq;               // cell of the global maximum
    int32_t Dp, LOWCHK, kint;     // step bound, lowest allowed score, rebase interval
};

// What the K warps sharing one pair's band (K > 1) hand each other through
// shared memory after every anti-diagonal, double-buffered by its parity:
// the gap-state word a warp's edge lane publishes for the neighbouring warp
// (E/E2 of its last slot going up, or F/F2 of its first slot going down), the
// warp's anti-diagonal maximum, and overflow flags.
struct Xchg16 {
    uint32_t e0[2][4], e1[2][4];
    int32_t m[2][4];
    int32_t f[2][4];
    int32_t t[2];                 // cell (t) of the maximum, found by the warp holding it
    int32_t g[4];                 // flags of a group-wide vote
    int32_t pair;                 // the group's current pair
};

// DMREG: keep the dead-slot masks in registers (the larger register budget)
// instead of recomputing them at every use.  DEFER: a new maximum found by a
// bulk step is only located (its cell found) when that can matter: before the
// next Z-drop test and when the bulk loop ends; until then the H values of its
// anti-diagonal are kept, so a run of growing maxima costs one copy each
// instead of one search each.
// DIR: the traceback variant (kernel_tb.cuh).  The same steps, run to a given
// end anti-diagonal without the termination test, also write one direction
// byte per slot: register p's low and high halves give bytes 2p and 2p+1 of
// the lane's C bytes of the anti-diagonal's row (slots j0+p and j0+p+P).
//   bits 0-3  H differs from the diagonal input H(r-2)+s, from E, F, E2
//             (H took the first input it equals; F2 if it differs from all four)
//   bits 4-7  Eo, Fo, E2o, F2o leaving the cell extend the cell's own gap
//             state (strictly better than opening from H)
// Each bit is one 16x2 minimum of an exclusive or (0 or 1 per half).
// SCORE: the termination test and the result (the score path).  DIR with
// SCORE is the fused traceback variant: the score path itself writes the
// direction bytes of every anti-diagonal it computes, so the traceback needs
// no second pass over the band; without SCORE (run_dir) the end anti-diagonal
// is given and nothing else is tracked.
// K: warps sharing one pair's band (1, 2 or 4).  Warp k of the group holds
// slots 32kC .. 32(k+1)C - 1 of the frame; after every anti-diagonal the warps
// exchange their edge gap states and anti-diagonal maxima through shared
// memory and a named barrier, so that the termination test stays exact.
// FHEAD: the head runs on the bulk step where the pair allows it.  EDEFER:
// the edge steps defer their arg-max search like the bulk.  (The larger
// register budget only: the extra state does not fit the smaller one
// without spills.)
template <int C, bool DMREG, bool DEFER = false, bool DIR = false, bool SCORE = !DIR, int K = 1,
          bool FHEAD = false, bool EDEFER = false, int G = 32>
struct WarpPair16 {
    static_assert(C == 4 || C == 6 || C == 8 || C == 12 || C == 16 || C == 20 || C == 24,
                  "16-bit lanes use 4, 6, 8, 12, 16, 20 or 24 slots per lane");
    static_assert(K == 1 || K == 2 || K == 4, "1, 2 or 4 warps per pair");
    static_assert(K == 1 || !DIR, "the traceback variants run one warp per pair");
    static_assert(G == 32 || (G == 16 && K == 1 && !DIR), "half-warp pairs: one group, score only");
    static constexpr int P = C / 2;
    static constexpr int32_t NS = G * C * K;      // slots of the frame
    // G lanes per pair: the whole warp, or a half warp (two pairs per warp,
    // each half with its own mask for every warp-collective operation)
    __device__ __forceinline__ static uint32_t gmask() {
        if constexpr (G == 32) return FULL;
        else return 0xffffu << (threadIdx.x & 16);
    }
    // ballot over the pair's lanes, bit i for the pair's lane i
    __device__ __forceinline__ static uint32_t gballot(bool v) {
        const uint32_t b = __ballot_sync(gmask(), v);
        if constexpr (G == 32) return b;
        else return (b >> (threadIdx.x & 16)) & 0xffffu;
    }
    // a base window holds 2 bits per slot
    using Win = typename std::conditional<(2 * C > 32), uint64_t, uint32_t>::type;
    static constexpr Win WMASK = (Win)(((uint64_t)1 << (2 * C)) - 1);
    // mismatch bits of a step, one word per 8 registers: register p's
    // low-half slot p at bit 2(p mod 8), its high-half slot p+P at bit
    // 16+2(p mod 8), of lo for p < 8 and of hi for p >= 8 (C = 24 only)
    struct Comb { uint32_t lo, hi; };

    // each sequence as its own words: base k of the pair at index k + phase
    // of the words from tp (qp); reads outside [0, span) words give 0 (those
    // bases only reach cells outside the table)
    const uint32_t *tp, *qp;
    int32_t tspan, qspan;
    int32_t tlen, qlen, w, last_r, lane, j0;
    DevParams prm;
    int32_t oe, oe2;
    // packed band state.  H(r) overwrites H(r-2) in the array of its parity:
    // Hev holds H of the last anti-diagonal with (r - w) even, Hod of the last
    // odd one.  Gap states leaving the last anti-diagonal: Eo to (t+1,q), Fo
    // to (t,q+1), E2o/F2o the same for the second gap piece.
    uint32_t Hev[P], Hod[P], Eo[P], E2o[P], Fo[P], F2o[P];
    // slots beyond the band (j > w): local slots k0.. of this lane, held as
    // (k0 - 1) in both halves so that dead_mask() is one add and one prmt
    uint32_t DF2;
    uint32_t DMR[DMREG ? P : 1];   // DMREG: dead_mask(p), computed once per pair
    uint32_t Hsave[DEFER ? P : 1]; // DEFER: H of the pending maximum's anti-diagonal
    uint8_t *dtab;                 // DIR: this lane's bytes of anti-diagonal 0
    int32_t end_t, end_q;          // DIR and SCORE: where the traceback starts (-1: empty)
    int32_t pend_r, pend_m, pend_lm;   // its anti-diagonal (-3: none), maximum, lane maximum
    uint32_t pend_rb;              // lane bits of its band slots (~0: every slot of the bulk)
    bool in_head;                  // FHEAD: the pair loop is running head anti-diagonals
    // base windows (2 bits per slot): Tw field jl = T[B + j0 + jl],
    // Qw field jl = Q[r - B - j0 - jl]
    Win Tw, Qw;
    uint32_t Tpf, Qpf;
    int32_t wcnt;          // pairs of shifts left in Tpf and Qpf (one count for both)
    int32_t tpos, qpos;    // next prefetch position (bases, word-relative)
    // relative scores
    int32_t base, OFF, last_m;
    int32_t until_rebase;  // anti-diagonals left before the next rebase
    bool ovf;
    // packed constants
    uint32_t A2, OEp, DOEp, Ep, E2p, NEp, NE2p, NEGp, L0LO, L31HI;
    uint32_t NABs;                 // -(a + b) as a 32-bit multiplier of the mismatch bits
    // bookkeeping (uniform across the warp)
    int32_t gmax;
    int32_t zdropped;
    // state the bulk step never reads, kept in shared memory (written by lane
    // 0) so that it holds no registers through the bulk loop
    Cold16 &cold;
    // K > 1: this warp's place in the group, the group's exchange area and
    // named barrier, the edge words the neighbouring warp published for the
    // next anti-diagonal, and this warp's maximum at the last exchange
    Xchg16 *xch;
    int32_t wk, bar_id;
    uint32_t xe0, xe1;
    int32_t xm_w;
    int32_t pend_owner;            // K > 1: the warp holding the pending maximum

    __device__ explicit WarpPair16(Cold16 &c, Xchg16 *x = nullptr, int32_t wk_ = 0, int32_t bar = 0)
        : cold(c), xch(x), wk(wk_), bar_id(bar) {}

    // K > 1: barrier of the group's warps (orders their shared-memory traffic)
    __device__ __forceinline__ void group_sync() const {
        if constexpr (K == 4) {
            asm volatile("bar.sync 1, 128;" ::: "memory");
        } else if constexpr (K == 2) {
            if (bar_id == 1) asm volatile("bar.sync 1, 64;" ::: "memory");
            else asm volatile("bar.sync 2, 64;" ::: "memory");
        }
    }
    // the lane that publishes for the group (lane 0 of warp 0)
    __device__ __forceinline__ bool leader() const { return lane == 0 && (K == 1 || wk == 0); }
    // K > 1: true in every lane of the group if v is true in any lane of any warp
    __device__ __forceinline__ bool group_any(bool v) {
        const bool w_any = __any_sync(gmask(), v);
        if constexpr (K == 1) return w_any;
        if (lane == 0) xch->g[wk] = w_any ? 1 : 0;
        group_sync();
        int32_t a = 0;
#pragma unroll
        for (int k = 0; k < K; ++k) a |= xch->g[k];
        group_sync();
        return a != 0;
    }
    // K > 1: publish this warp's anti-diagonal maximum lm (lane maxima) and,
    // for the next anti-diagonal (odd one when ODDNEXT), the edge gap states
    // the neighbouring warp needs; with FLAG also the overflow flag.  Returns
    // the group's maximum; leaves the neighbour's edge words in xe0/xe1.
    template <bool ODDNEXT, bool FLAG>
    __device__ __forceinline__ int32_t exchange(int32_t r, int32_t lm) {
        const int b = r & 1;
        const int32_t mw = __reduce_max_sync(gmask(), lm);
        const bool fw = FLAG ? __any_sync(gmask(), ovf) : false;
        if (lane == 0) {
            xch->m[b][wk] = mw;
            if (FLAG) xch->f[b][wk] = fw ? 1 : 0;
        }
        if (ODDNEXT) {
            if (lane == 31) { xch->e0[b][wk] = Eo[P - 1]; xch->e1[b][wk] = E2o[P - 1]; }
        } else {
            if (lane == 0) { xch->e0[b][wk] = Fo[0]; xch->e1[b][wk] = F2o[0]; }
        }
        group_sync();
        int32_t m = xch->m[b][0];
        int32_t f = FLAG ? xch->f[b][0] : 0;
#pragma unroll
        for (int k = 1; k < K; ++k) {
            m = max(m, xch->m[b][k]);
            if (FLAG) f |= xch->f[b][k];
        }
        if (FLAG) ovf = f != 0;
        const int src = ODDNEXT ? wk - 1 : wk + 1;
        if (src >= 0 && src < K) { xe0 = xch->e0[b][src]; xe1 = xch->e1[b][src]; }
        xm_w = mw;
        return m;
    }
    // K > 1: the lowest warp whose maximum at the last exchange of r is m
    __device__ __forceinline__ int32_t owner_of(int32_t r, int32_t m) const {
        const int b = r & 1;
        int32_t o = K - 1;
#pragma unroll
        for (int k = K - 1; k >= 0; --k) o = xch->m[b][k] == m ? k : o;
        return o;
    }

    __device__ __forceinline__ int32_t to_true(int32_t u) const { return u - OFF + base; }
    __device__ __forceinline__ int32_t to_u(int32_t v) const { return v - base + OFF; }
    __device__ __forceinline__ int32_t frame(int32_t r) const { return floor_div2(r - w); }

    // ------------------------------------------------------------ windows
    // 16 bases from word-relative base index a (any a; outside the span: 0)
    __device__ __forceinline__ static uint32_t load_rel(const uint32_t *__restrict__ p, int32_t span,
                                                        int32_t a) {
        const int32_t wi = a >> 4;                     // floor for negative a too
        const uint32_t lo = (uint32_t)wi < (uint32_t)span ? __ldg(p + wi) : 0u;
        const uint32_t hi = (uint32_t)(wi + 1) < (uint32_t)span ? __ldg(p + wi + 1) : 0u;
        return __funnelshift_r(lo, hi, (uint32_t)(a & 15) * 2u);
    }
    __device__ __forceinline__ static uint64_t load_rel32(const uint32_t *__restrict__ p, int32_t span,
                                                          int32_t a) {
        return (uint64_t)load_rel(p, span, a) | ((uint64_t)load_rel(p, span, a + 16) << 32);
    }
    // tph/qph: the phase of the pair's first base in its first word
    __device__ __forceinline__ void init_windows(int32_t r, int32_t tph, int32_t qph) {
        const int32_t B = frame(r);
        const int32_t tb = B + j0 + tph;
        const int32_t qb = r - B - j0 + qph;
        if constexpr (C <= 16) {
            Tw = load_rel(tp, tspan, tb) & WMASK;
            Qw = rev2_32(load_rel(qp, qspan, qb - C + 1)) >> (2 * (16 - C));
        } else {
            Tw = load_rel32(tp, tspan, tb) & WMASK;
            Qw = rev2_64(load_rel32(qp, qspan, qb - C + 1)) >> (2 * (32 - C));
        }
        tpos = tb + C;
        qpos = qb + 1;
        Tpf = load_rel(tp, tspan, tpos);
        Qpf = load_rel(qp, qspan, qpos);
        // Every pair of anti-diagonals shifts T ((r - w) even) then Q, so one
        // count serves both words: T reloads on the shift that finds one pair
        // left, Q on the shift that ends the count.  When the first shift is
        // a Q shift, T's first word is used for 15 bases only (the 16th is
        // the first of its next load), which keeps the two in step.
        tpos += ((r + 1 - w) & 1) ? 15 : 16;
        qpos += 16;
        wcnt = 16;
    }
    __device__ __forceinline__ void shift_t_window() {
        Tw = (Tw >> 2) | ((Win)(Tpf & 3u) << (2 * C - 2));
        Tpf >>= 2;
    }
    __device__ __forceinline__ void shift_q_window() {
        Qw = ((Qw << 2) | (Win)(Qpf & 3u)) & WMASK;
        Qpf >>= 2;
    }
    __device__ __forceinline__ void reload_t() { Tpf = load_rel(tp, tspan, tpos); tpos += 16; }
    __device__ __forceinline__ void reload_q() { Qpf = load_rel(qp, qspan, qpos); qpos += 16; }
    __device__ __forceinline__ void shift_t() {
        shift_t_window();
        if (wcnt == 1) reload_t();
    }
    __device__ __forceinline__ void shift_q() {
        shift_q_window();
        if (--wcnt == 0) { reload_q(); wcnt = 16; }
    }
    // windows of anti-diagonal r from those of r-1
    __device__ __forceinline__ void advance(int32_t r) {
        if ((r - w) & 1) shift_q(); else shift_t();
    }
    __device__ __forceinline__ Comb packed_mismatch() const {
        const Win x = Tw ^ Qw;
        const Win nm = (x | (x >> 1)) & (Win)0x5555555555555555ull;    // slot jl at bit 2*jl
        if constexpr (C == 16) return {(uint32_t)nm, 0u};
        else if constexpr (C == 12) return {((uint32_t)nm & 0xfffu) | (((uint32_t)nm & 0xfff000u) << 4), 0u};
        else if constexpr (C == 8) return {((uint32_t)nm & 0xffu) | (((uint32_t)nm & 0xff00u) << 8), 0u};
        else if constexpr (C == 6) return {((uint32_t)nm & 0x3fu) | (((uint32_t)nm & 0xfc0u) << 10), 0u};
        else if constexpr (C == 4) return {((uint32_t)nm & 0xfu) | (((uint32_t)nm & 0xf0u) << 12), 0u};
        else if constexpr (C == 20) {
            // slots 0..9 and 10..19 (bits 0..18 and 20..38); registers 0..7
            // in lo, 8..9 in hi
            return {((uint32_t)nm & 0xffffu) | ((uint32_t)(nm >> 4) & 0xffff0000u),
                    ((uint32_t)(nm >> 16) & 0xfu) | ((uint32_t)(nm >> 20) & 0xf0000u)};
        }
        else {
            // slots 0..11 and 12..23; registers 0..7 in lo, 8..11 in hi
            const uint32_t a = (uint32_t)(nm & 0xffffffu), b = (uint32_t)(nm >> 24);
            return {prmt(a, b, 0x5410), prmt(a, b, 0x7632)};
        }
    }
    // 0xFFFF halves of register p from lane bits (low half p at bit p, high at 16+p)
    template <int PP>
    __device__ __forceinline__ static uint32_t half_mask(uint32_t bits) {
        return prmt(bits << (15 - PP), 0, 0xbb99);
    }
    // the same for a register index known only after unrolling
    __device__ __forceinline__ static uint32_t half_mask_rt(uint32_t bits, int p) {
        return prmt(bits << (15 - p), 0, 0xbb99);
    }
    // lane bits of the local slots [lo, hi] (empty if lo > hi)
    __device__ __forceinline__ static uint32_t range_bits(int32_t lo, int32_t hi) {
        lo = max(lo, 0);
        hi = min(hi, C - 1);
        if (lo > hi) return 0u;
        const uint32_t b = ((2u << hi) - 1u) & ~((1u << lo) - 1u);
        return (b & ((1u << P) - 1u)) | ((b >> P) << 16);
    }
    __device__ __forceinline__ static uint32_t slot_bit(int32_t jl) {
        if (jl < 0 || jl >= C) return 0u;
        return jl < P ? (1u << jl) : (1u << (16 + jl - P));
    }

    // 0xFFFF halves of register p whose slot lies beyond the band: the half
    // (k0 - 1 - slot) is negative exactly there (a borrow out of the low half
    // only reaches a high half that is beyond the band as well)
    __device__ __forceinline__ uint32_t dead_mask(int p) const {
        if constexpr (DMREG) return DMR[p];
        return half_sign_of_diff(DF2, (uint32_t)p | ((uint32_t)(p + P) << 16));
    }
    // the same plus slot 0 of lane 0, outside the band on odd anti-diagonals
    template <bool ODD>
    __device__ __forceinline__ uint32_t dead_mask_r(int p) const {
        return (ODD && p == 0) ? (dead_mask(0) | L0LO) : dead_mask(p);
    }

    // ------------------------------------------------------- Eq. 4-7 test
    __device__ __forceinline__ bool max_and_zdrop(int32_t m, int32_t tstar, int32_t r) {
        const int32_t qstar = r - tstar;
        if (m > gmax) {
            gmax = m;
            if (leader()) { cold.gt = tstar; cold.gq = qstar; }
            __syncwarp(gmask());
            return false;
        }
        const int32_t gt = cold.gt, gq = cold.gq;
        if (tstar >= gt && qstar >= gq && prm.zdrop >= 0) {
            int32_t l = (tstar - gt) - (qstar - gq);
            l = l < 0 ? -l : l;
            if (gmax - m > prm.zdrop + l * prm.e2) return true;
        }
        return false;
    }

    // Anti-diagonal maximum and termination rule.  lmax: 16x2 maximum of
    // H - q - e over the lane's band cells (others 0); Hn: the H values of r;
    // excl(p): 0xFFFF halves of slots that are not band cells.  Returns true
    // to stop.
    // Locate a pending maximum (DEFER): the same search as anti_diagonal_max
    // on the kept H values; sets the cell of the global maximum.
    __device__ __forceinline__ void locate_pending() {
        if constexpr (DEFER) {
            if (pend_r == -3) return;
            if (K > 1 && wk != pend_owner) {       // the warp holding it finds it
                group_sync();
                pend_r = -3;
                return;
            }
            const unsigned ball = gballot(pend_lm == pend_m);
            const int src = __ffs(ball) - 1;
            const uint32_t mh2 = (uint32_t)(pend_m + oe) * 0x10001u;
            const uint32_t x0 = ((pend_r - w) & 1) ? L0LO : 0u;   // slot 0 of lane 0 on odd ones
            uint32_t ne = 0;
#pragma unroll
            for (int p = 0; p < P; ++p)
                ne += __vminu2((Hsave[p] ^ mh2) | (p == 0 ? x0 : 0u) | ~half_mask_rt(pend_rb, p), 0x10001u) << p;
            const uint32_t eq = ~ne & ((((1u << P) - 1) << 16) | ((1u << P) - 1));
            const uint32_t lo_eq = eq & 0xffffu, hi_eq = eq >> 16;
            const int32_t jl = lo_eq ? __ffs(lo_eq) - 1 : P + __ffs(hi_eq) - 1;
            const int32_t lj = __shfl_sync(gmask(), jl, src, G);
            const int32_t tstar = frame(pend_r) + (wk * G + src) * C + lj;
            if (lane == 0) { cold.gt = tstar; cold.gq = pend_r - tstar; }
            __syncwarp(gmask());
            group_sync();
            pend_r = -3;
        }
    }

    // Head on the bulk step, when a virtual cell may hold the anti-diagonal
    // maximum: the maximum and the termination test over the band cells only.
    template <bool ODD>
    __device__ __forceinline__ bool head_band_max(int32_t r) {
        if (r < 0) return false;       // no band cell yet: nothing to test
        const uint32_t (&Hn)[P] = ODD ? Hod : Hev;
        const int32_t B = frame(r);
        const uint32_t rb = table_bits(r);
        uint32_t lmax = 0;
#pragma unroll
        for (int p = 0; p < P; ++p) lmax = __vmaxu2(lmax, half_mask_rt(rb, p) & (Hn[p] - OEp));
        const int32_t lm = (int32_t)max(lmax & 0xffffu, lmax >> 16);
        auto excl = [&](int p) { return ~half_mask_rt(rb, p); };
        return anti_diagonal_max<ODD, decltype(excl), false>(r, B, lm, 0, Hn, excl, rb);
    }

    // lm: the lane's maximum; m_grp (K > 1): the group's, from exchange();
    // rb: lane bits of the band slots (edge steps; the search excludes the rest).
    template <bool ODD, typename Excl, bool BULKSTEP = false>
    __device__ __forceinline__ bool anti_diagonal_max(int32_t r, int32_t B, int32_t lm, int32_t m_grp,
                                                      const uint32_t (&Hn)[P], Excl excl,
                                                      uint32_t rb = ~0u) {
        const int32_t m = K == 1 ? __reduce_max_sync(gmask(), lm) : m_grp;
        const int32_t mt = to_true(m + oe);
        last_m = m + oe;
        if constexpr (DEFER && (BULKSTEP || EDEFER)) {
            if (mt > gmax) {                   // keep it; locate it when needed
                gmax = mt;
#pragma unroll
                for (int p = 0; p < P; ++p) Hsave[p] = Hn[p];
                pend_r = r;
                pend_m = K == 1 ? m : xm_w;
                pend_lm = lm;
                pend_rb = rb;
                if constexpr (K > 1) pend_owner = owner_of(r, m);
                return false;
            }
            if (!(prm.zdrop >= 0 && gmax - mt > prm.zdrop)) return false;
            locate_pending();
        }
        if (mt > gmax || (prm.zdrop >= 0 && gmax - mt > prm.zdrop)) {
            // position only when it can matter: lowest slot of the first lane
            // (of the first warp) holding the maximum; bit p / 16+p of `ne` is
            // set where the low / high half of register p is not it
            int32_t tstar = 0;
            const int32_t owner = K == 1 ? 0 : owner_of(r, m);
            if (K == 1 || wk == owner) {
                const unsigned ball = gballot(lm == m);
                const int src = __ffs(ball) - 1;
                const uint32_t mh2 = (uint32_t)(m + oe) * 0x10001u;
                uint32_t ne = 0;
#pragma unroll
                for (int p = 0; p < P; ++p) ne += __vminu2((Hn[p] ^ mh2) | excl(p), 0x10001u) << p;
                const uint32_t eq = ~ne & ((((1u << P) - 1) << 16) | ((1u << P) - 1));
                const uint32_t lo_eq = eq & 0xffffu, hi_eq = eq >> 16;
                const int32_t jl = lo_eq ? __ffs(lo_eq) - 1 : P + __ffs(hi_eq) - 1;
                const int32_t lj = __shfl_sync(gmask(), jl, src, G);
                tstar = B + (wk * G + src) * C + lj;
                if (K > 1 && lane == 0) xch->t[r & 1] = tstar;
            }
            if constexpr (K > 1) {
                group_sync();
                tstar = xch->t[r & 1];
            }
            if (max_and_zdrop(mt, tstar, r)) { zdropped = 1; return true; }
        }
        return false;
    }

    // H of the band slot j (the same j in every lane) of the anti-diagonal
    // just computed, read from the lane that owns it.
    __device__ __forceinline__ int32_t slot_value(const uint32_t (&Hn)[P], int32_t j) const {
        const int32_t local = j % C;
        return __shfl_sync(gmask(), half_of(reg_select(Hn, local % P), local), (j / C) & (G - 1), G);
    }
    // Register pl of Hn (pl may differ between lanes): a select tree on the
    // bits of pl, P - 1 selects.
    __device__ __forceinline__ static uint32_t reg_select(const uint32_t (&Hn)[P], int32_t pl) {
        uint32_t v[P];
#pragma unroll
        for (int p = 0; p < P; ++p) v[p] = Hn[p];
#pragma unroll
        for (int b = 1; b < P; b <<= 1) {
            const bool hi = (pl & b) != 0;
#pragma unroll
            for (int p = 0; p + b < P; p += 2 * b) v[p] = hi ? v[p + b] : v[p];
        }
        return v[0];
    }
    __device__ __forceinline__ static int32_t half_of(uint32_t v, int32_t local) {
        return local >= P ? (int32_t)(v >> 16) : (int32_t)(v & 0xffffu);
    }
    // H of slots jt and jq (each the same in every lane) at once: every lane
    // selects the slot it owns (jt where it owns both) and each value is one
    // shuffle from its owner; a second pass only when one lane owns both and
    // they differ.
    __device__ __forceinline__ void slot_values(const uint32_t (&Hn)[P], int32_t jt, int32_t jq, int32_t &vt,
                                                int32_t &vq) const {
        const int32_t lt = (jt / C) & (G - 1), lq = (jq / C) & (G - 1);
        const int32_t j = lane == lt ? jt : jq;
        const int32_t local = j % C;
        const int32_t h = half_of(reg_select(Hn, local % P), local);
        vt = __shfl_sync(gmask(), h, lt, G);
        if (lt == lq && jt != jq) vq = slot_value(Hn, jq);
        else vq = __shfl_sync(gmask(), h, lq, G);
    }
    // K > 1: the warp of the group that holds frame slot j
    __device__ __forceinline__ static int32_t slot_warp(int32_t j) { return j / (G * C); }

    // Step modes.  BULK: every slot in [0, w] is a band cell of the table.
    // HEAD (r <= w + 1): the band meets the table's first row and column;
    // after the update every slot is set to what the recurrence defines
    // there: a band cell keeps its value, the virtual row/column cell
    // (-1, r+1) or (r+1, -1) gets H = -gap(r+2) (H(-1,-1) = 0 on r = -2),
    // anything else is minus infinity.  TAIL (r >= w + 2): the band may run
    // past the last row or column.  Cells there (t >= tlen or q >= qlen) feed
    // only cells past the end again, never a cell of the table, so they are
    // left as computed and only kept out of the maximum.
    enum : int { BULK = 0, HEAD = 1, TAIL = 2 };

    // One anti-diagonal on the packed registers, in place (H(r) replaces
    // H(r-2) in the array of its parity, the gap arrays turn from the states
    // leaving r-1 into those leaving r).  ODD: (r - w) odd, E from slot j-1
    // and F from slot j; else E from slot j and F from slot j+1.  F-from-j+1
    // steps walk the registers upwards and E-from-j-1 steps downwards, so
    // every old value is read before it is overwritten.
    template <bool ODD, int MODE>
    __device__ __forceinline__ bool step(int32_t r) {
        uint32_t (&Hd)[P] = ODD ? Hod : Hev;
        const int32_t B = frame(r);
        int32_t st = 0, en = -1;
        uint32_t rb = 0, vb = 0, VVp = 0;
        if constexpr (MODE != BULK) {
            if (r >= 0) {
                st = max(max(0, r - qlen + 1), ceil_div2(r - w));
                en = min(min(tlen - 1, r), floor_div2(r + w));
                if (st > en) { zdropped = 1; return true; }  // the band left the table
            }
            rb = range_bits(st - B - j0, en - B - j0);
        }
        if constexpr (MODE == HEAD) {
            if (r + 1 < qlen) vb |= slot_bit(-1 - B - j0);                 // (-1, r+1)
            if (r >= -1 && r + 1 < tlen) vb |= slot_bit(r + 1 - B - j0);  // (r+1, -1)
            const int32_t vv = to_u(r == -2 ? 0 : -gap_cost(prm, r + 2));
            if (__any_sync(gmask(), vb != 0u) && (vv < cold.LOWCHK || vv > 0xffff - cold.Dp)) ovf = true;
            VVp = (uint32_t)vv * 0x10001u;
        }
        uint32_t edge, edge2;
        if constexpr (ODD) {
            // E of slot 0 from the left lane's last slot (high half of its last
            // register); for lane 0 it would feed slot 0, outside the band here
            // (with K warps, lane 0 of a later warp takes the word the warp
            // below published)
            uint32_t eL = __shfl_up_sync(gmask(), Eo[P - 1], 1, G);
            uint32_t e2L = __shfl_up_sync(gmask(), E2o[P - 1], 1, G);
            if (K > 1 && wk > 0 && lane == 0) { eL = xe0; e2L = xe1; }
            edge = mux(L0LO, NEGp, prmt(eL, Eo[P - 1], 0x5432));
            edge2 = mux(L0LO, NEGp, prmt(e2L, E2o[P - 1], 0x5432));
        } else {
            // F of the last slot from the right lane's first slot (low half of
            // its register 0; with K warps, from the warp above for lane 31)
            uint32_t fR = __shfl_down_sync(gmask(), Fo[0], 1, G);
            uint32_t f2R = __shfl_down_sync(gmask(), F2o[0], 1, G);
            if (K > 1 && wk < K - 1 && lane == 31) { fR = xe0; f2R = xe1; }
            uint32_t inj = NEGp, inj2 = NEGp;
            if (MODE == HEAD && lane == G - 1 && (K == 1 || wk == K - 1)) {
                // beyond the last lane: slot NS of r-1, the virtual column
                // cell (t, -1) when q == -1 there
                const int32_t ts = frame(r - 1) + NS, qs = r - 1 - ts;
                if (qs == -1 && ts >= 0 && ts < tlen) {
                    const int32_t v = to_u(-gap_cost(prm, ts + 1));
                    if (v < cold.LOWCHK || v > 0xffff - cold.Dp) ovf = true;
                    inj = ((uint32_t)(v - oe) << 16) | (NEGp & 0xffffu);
                    inj2 = ((uint32_t)(v - oe2) << 16) | (NEGp & 0xffffu);
                }
            }
            edge = mux(L31HI, inj, prmt(Fo[0], fR, 0x5432));
            edge2 = mux(L31HI, inj2, prmt(F2o[0], f2R, 0x5432));
        }
        const Comb comb = packed_mismatch();
        uint32_t lmax = 0, pend = 0;
        uint32_t dbits[DIR ? P : 1];
#pragma unroll
        for (int i = 0; i < P; ++i) {
            const int p = ODD ? P - 1 - i : i;
            uint32_t Ein, E2in, Fin, F2in;
            if constexpr (ODD) {
                Ein = p ? Eo[p - 1] : edge;
                E2in = p ? E2o[p - 1] : edge2;
                Fin = Fo[p];
                F2in = F2o[p];
            } else {
                Ein = Eo[p];
                E2in = E2o[p];
                Fin = p < P - 1 ? Fo[p + 1] : edge;
                F2in = p < P - 1 ? F2o[p + 1] : edge2;
            }
            // substitution: H(r-2) + s = (H(r-2) - m (a+b)) + a per half, m = 1
            // where the bases differ.  The first part is one multiply-add of
            // the mismatch bits: no half borrows, since every score a later
            // cell of the table can read stays far above a + b (the same
            // argument as for the open terms below).
            const uint32_t mword = (C <= 16 || p < 8) ? comb.lo : comb.hi;
            const uint32_t mb = (mword >> (2 * (p & 7))) & 0x10001u;
            const uint32_t Hs = mb * NABs + Hd[p];
            const uint32_t s2 = A2;
            // H = max(H(r-2) + s, E, F, E2, F2): add-max, 3-input max, max
            const uint32_t H = __vmaxu2(__vimax3_u16x2(__viaddmax_u16x2(Hs, s2, Ein), Fin, E2in),
                                        F2in);
            if constexpr (DIR) {
                // 1 per half where H differs from the input (scores sit far
                // above 0, so the per-half add of s needs no further clamp)
                const uint32_t one = 0x10001u;
                const uint32_t hd = __viaddmax_u16x2(Hs, s2, 0u);
                dbits[p] = __vminu2(H ^ hd, one) + (__vminu2(H ^ Ein, one) << 1) +
                           (__vminu2(H ^ Fin, one) << 2) + (__vminu2(H ^ E2in, one) << 3);
            }
            uint32_t mx;                          // this register's share of the maximum
            if constexpr (MODE != HEAD) {
                const uint32_t dead = dead_mask_r<ODD>(p);
                const uint32_t hoe = mux(dead, NEGp, H - OEp);
                const uint32_t hoe2 = hoe - DOEp;
                // per-half add of -e (wraps within the half) then max: one op each
                Eo[p] = __viaddmax_u16x2(Ein, NEp, hoe);
                Fo[p] = __viaddmax_u16x2(Fin, NEp, hoe);
                E2o[p] = __viaddmax_u16x2(E2in, NE2p, hoe2);
                F2o[p] = __viaddmax_u16x2(F2in, NE2p, hoe2);
                Hd[p] = H;
                mx = MODE == BULK ? hoe : (half_mask_rt(rb, p) & hoe);
                if constexpr (DIR) dbits[p] += ext_bits(hoe, hoe2, p);
            } else {
                // H of the band cells; the virtual row/column cell gets its
                // exact value and every other slot minus infinity.  The gap
                // states then follow from this H: a virtual cell's inputs come
                // from slots at minus infinity, so it emits exactly
                // -gap(r+2) - q - e (- q2 - e2); the other slots off the table
                // emit at most NEG, or, past the table's end, values that only
                // reach cells past the end
                const uint32_t rm = half_mask_rt(rb, p);
                const uint32_t vm = half_mask_rt(vb, p);
                const uint32_t Hm = mux(rm, H, mux(vm, VVp, NEGp));
                const uint32_t hoe = Hm - OEp;
                const uint32_t hoe2 = hoe - DOEp;
                Eo[p] = __viaddmax_u16x2(Ein, NEp, hoe);
                Fo[p] = __viaddmax_u16x2(Fin, NEp, hoe);
                E2o[p] = __viaddmax_u16x2(E2in, NE2p, hoe2);
                F2o[p] = __viaddmax_u16x2(F2in, NE2p, hoe2);
                Hd[p] = Hm;
                mx = rm & hoe;
                if constexpr (DIR) dbits[p] += ext_bits(hoe, hoe2, p);
            }
            // running maximum, two registers per 3-input max
            if (i & 1) lmax = __vimax3_u16x2(lmax, pend, mx);
            else if (i == P - 1) lmax = __vmaxu2(lmax, mx);
            else pend = mx;
        }
        if constexpr (DIR && !SCORE) return dir_finish<ODD, MODE>(r, lmax, rb, vb, dbits);
        if constexpr (DIR && SCORE) {
            if (r >= 0) store_row(r, dbits);
        }
        const int32_t lm = (int32_t)max(lmax & 0xffffu, lmax >> 16);
        int32_t m_grp = 0;
        if constexpr (K > 1) m_grp = exchange<!ODD, MODE != BULK>(r, lm);
        if constexpr (MODE == BULK) {
            // slots beyond the band sit above every band slot of their lane, so
            // the lowest slot holding the maximum is a band slot; only slot 0 of
            // lane 0 (below the band on odd anti-diagonals) is excluded
            auto excl = [&](int p) { return (ODD && p == 0) ? L0LO : 0u; };
            return anti_diagonal_max<ODD, decltype(excl), true>(r, B, lm, m_grp, Hd, excl);
        } else {
            if (K == 1 ? __any_sync(gmask(), ovf) : ovf) { ovf = true; return true; }
            if (r < 0) return false;
            // best score on the last target row / the last query column (with
            // K warps, the warp holding the slot reads it)
            bool set_gs = false;
            int32_t gs = K_NEG_OUT;
            const int32_t jt = tlen - 1 - B, jq = r - qlen + 1 - B;
            const bool at_t = st <= tlen - 1 && tlen - 1 <= en && (K == 1 || slot_warp(jt) == wk);
            const bool at_q = st <= r - qlen + 1 && r - qlen + 1 <= en && (K == 1 || slot_warp(jq) == wk);
            if (at_t || at_q) {
                int32_t hv_t, hv_q;
                slot_values(Hd, at_t ? jt : jq, at_q ? jq : jt, hv_t, hv_q);
                if (at_t) {
                    const int32_t tv = to_true(hv_t);
                    if (tv > cold.mte && lane == 0) { cold.mte = tv; cold.mte_q = r - (tlen - 1); }
                    if (r == last_r) { gs = tv; set_gs = true; }   // kept unless Z-drop stops r
                }
                if (at_q) {
                    const int32_t qv = to_true(hv_q);
                    if (qv > cold.mqe && lane == 0) { cold.mqe = qv; cold.mqe_t = r - (qlen - 1); }
                }
            }
            __syncwarp(gmask());
            if (anti_diagonal_max<ODD>(r, B, lm, m_grp, Hd, [&](int p) { return ~half_mask_rt(rb, p); }, rb))
                return true;
            if (set_gs && lane == 0) cold.gscore = gs;
            if (--until_rebase <= 2) {
                // slots off the table (past its end, or holding NEG) are
                // reset; the virtual cells' values are kept
                if (MODE == TAIL) {
                    // (a tail step run in the head keeps the virtual cells)
                    const bool vh = FHEAD && in_head;
                    rebase(last_m, r, rb | (vh ? virtual_bits(r) : 0u),
                           table_bits(r - 1) | (vh ? virtual_bits(r - 1) : 0u));
                } else {
                    rebase(last_m, r, rb | vb, table_bits(r - 1) | virtual_bits(r - 1));
                }
            }
            return ovf;
        }
    }

    // DIR: bits 4-7 of register p's two bytes from the gap states just
    // written (a state that differs from the opening value extended)
    __device__ __forceinline__ uint32_t ext_bits(uint32_t hoe, uint32_t hoe2, int p) const {
        const uint32_t one = 0x10001u;
        return (__vminu2(Eo[p] ^ hoe, one) << 4) + (__vminu2(Fo[p] ^ hoe, one) << 5) +
               (__vminu2(E2o[p] ^ hoe2, one) << 6) + (__vminu2(F2o[p] ^ hoe2, one) << 7);
    }

    // DIR: the lane's C bytes of anti-diagonal r, one vector store
    __device__ __forceinline__ void store_row(int32_t r, const uint32_t (&db)[P]) const {
        uint32_t wd[C / 4];
#pragma unroll
        for (int k = 0; k < C / 4; ++k) wd[k] = prmt(db[2 * k], db[2 * k + 1], 0x6420);
        uint8_t *p = dtab + (int64_t)r * (32 * C);
        if constexpr (C % 16 == 0) {
#pragma unroll
            for (int k = 0; k < C / 16; ++k)
                reinterpret_cast<uint4 *>(p)[k] = make_uint4(wd[4 * k], wd[4 * k + 1], wd[4 * k + 2], wd[4 * k + 3]);
        } else if constexpr (C % 8 == 0) {
#pragma unroll
            for (int k = 0; k < C / 8; ++k) reinterpret_cast<uint2 *>(p)[k] = make_uint2(wd[2 * k], wd[2 * k + 1]);
        } else {
            *reinterpret_cast<uint32_t *>(p) = wd[0];
        }
    }

    // DIR without SCORE: end of a step.  Store the row, then what the rebase
    // needs: the anti-diagonal maximum (only when a rebase follows) and the
    // rebase.
    template <bool ODD, int MODE>
    __device__ __forceinline__ bool dir_finish(int32_t r, uint32_t lmax, uint32_t rb, uint32_t vb,
                                               const uint32_t (&db)[P]) {
        if (r >= 0) store_row(r, db);
        if constexpr (MODE == BULK) {
            // fast_pair rebases after the odd step of a pair
            if (ODD && until_rebase <= 4) {
                const int32_t lm = (int32_t)max(lmax & 0xffffu, lmax >> 16);
                last_m = __reduce_max_sync(gmask(), lm) + oe;
            }
            return false;
        } else {
            if (__any_sync(gmask(), ovf)) { ovf = true; return true; }
            if (r < 0) return false;
            if (--until_rebase <= 2) {
                const int32_t lm = (int32_t)max(lmax & 0xffffu, lmax >> 16);
                last_m = __reduce_max_sync(gmask(), lm) + oe;
                if (MODE == TAIL) rebase(last_m, r, rb, table_bits(r - 1));
                else rebase(last_m, r, rb | vb, table_bits(r - 1) | virtual_bits(r - 1));
            }
            return ovf;
        }
    }

    // Bulk anti-diagonals r ((r - w) even) and r+1; returns 0 to go on, else
    // k+1 when the extension stopped on r+k.
    // FHEAD, in the head: 3 (4) when a virtual cell may hold the maximum of
    // r (r + 1), the step's own decision undone; the caller decides again
    // over the band cells only.
    // The pair's two window shifts share one count test (after the Q shift).
    __device__ __forceinline__ int fast_pair(int32_t r) {
        shift_t_window();
        const bool s1 = step<false, BULK>(r);
        if (FHEAD && in_head && last_m == to_u(-gap_cost(prm, r + 2))) {
            zdropped = 0;
            if (wcnt == 1) reload_t();          // the T shift's own reload
            return 3;
        }
        if (s1) return 1;
        shift_q_window();
        if (--wcnt == 0) { reload_t(); reload_q(); wcnt = 16; }
        const bool s2 = step<true, BULK>(r + 1);
        if (FHEAD && in_head && last_m == to_u(-gap_cost(prm, r + 3))) { zdropped = 0; return 4; }
        if (s2) return 2;
        until_rebase -= 2;
        if (until_rebase <= 2) {
            if (FHEAD && in_head)          // cells beyond the virtual ones are neither reset nor checked
                rebase(last_m, r + 1, table_bits(r + 1) | virtual_bits(r + 1), table_bits(r) | virtual_bits(r));
            else
                rebase(last_m, r + 1);
            if (ovf) return 2;
        }
        return 0;
    }

    __device__ __forceinline__ bool head_step(int32_t r) {
        return ((r - w) & 1) ? step<true, HEAD>(r) : step<false, HEAD>(r);
    }
    __device__ __forceinline__ bool tail_step(int32_t r) {
        return ((r - w) & 1) ? step<true, TAIL>(r) : step<false, TAIL>(r);
    }

    // ---------------------------------------------------------------- rebase
    // Move base so that the anti-diagonal maximum m_u is stored at OFF; check
    // that every band score keeps (K+3)D of headroom above NEG; reset minus
    // infinity (anything at most NEG) and slots outside the band to NEG.
    // Both halves of x at once: halves of dm (0xFFFF) and halves at most NEG
    // become NEG; the others must be at least `low2` (else ovf) and move by
    // -delta, clamped to [NEG + 1, 0xFFFF] (sub: delta >= 0, by d2 = delta;
    // else by d2 = -delta upwards).
    template <bool SUB>
    __device__ __forceinline__ void rebase_reg(uint32_t &x, uint32_t dm, uint32_t d2, uint32_t low2) {
        const uint32_t reset = __vcmpleu2(x, NEGp) | dm;
        if (__vcmpltu2(x, low2) & ~reset) ovf = true;
        const uint32_t y = __vmaxu2(SUB ? __vsubus2(x, d2) : __vaddus2(x, d2), NEGp + 0x10001u);
        x = mux(reset, NEGp, y);
    }
    // r: the last anti-diagonal computed (its gap states are in Eo..)
    // in_r / in_r1: lane bits of the slots of anti-diagonals r / r-1 that are
    // cells of the table; the others (past the table's end in the tail) are
    // reset like the slots beyond the band and not checked.
    __device__ __forceinline__ void rebase(int32_t m_u, int32_t r, uint32_t in_r = ~0u,
                                           uint32_t in_r1 = ~0u) {
        until_rebase = cold.kint;
        const int32_t delta = m_u - OFF;
        const int32_t low = min(max(cold.LOWCHK - cold.Dp + delta, 0), 0xffff);
        const uint32_t low2 = (uint32_t)low * 0x10001u;
        const bool odd = ((r - w) & 1) != 0;
        const uint32_t in_ev = odd ? in_r1 : in_r, in_od = odd ? in_r : in_r1;
        if (delta >= 0) rebase_all<true>((uint32_t)min(delta, 0xffff) * 0x10001u, low2, odd, in_ev, in_od);
        else rebase_all<false>((uint32_t)min(-delta, 0xffff) * 0x10001u, low2, odd, in_ev, in_od);
        base += delta;
        ovf = group_any(ovf);
    }
    template <bool SUB>
    __device__ __forceinline__ void rebase_all(uint32_t d2, uint32_t low2, bool odd, uint32_t in_ev,
                                               uint32_t in_od) {
#pragma unroll
        for (int p = 0; p < P; ++p) {
            const uint32_t dm = dead_mask(p);
            const uint32_t dm_ev = dm | ~half_mask_rt(in_ev, p);
            const uint32_t dm_od = (p == 0 ? (dm | L0LO) : dm) | ~half_mask_rt(in_od, p);
            const uint32_t dm_r = odd ? dm_od : dm_ev;         // slots of anti-diagonal r
            rebase_reg<SUB>(Hev[p], dm_ev, d2, low2);
            rebase_reg<SUB>(Hod[p], dm_od, d2, low2);
            rebase_reg<SUB>(Eo[p], dm_r, d2, low2);
            rebase_reg<SUB>(E2o[p], dm_r, d2, low2);
            rebase_reg<SUB>(Fo[p], dm_r, d2, low2);
            rebase_reg<SUB>(F2o[p], dm_r, d2, low2);
        }
        if constexpr (K > 1) {
            // the edge words the neighbouring warp published before this
            // rebase move with the rest (the half the next anti-diagonal reads:
            // high for an odd one, low for an even one); the neighbour checks
            // its own copy, so these are only shifted
            const bool next_odd = !odd;
            const uint32_t keep = next_odd ? 0xffff0000u : 0x0000ffffu;
            rebase_edge<SUB>(xe0, keep, d2);
            rebase_edge<SUB>(xe1, keep, d2);
        }
    }
    template <bool SUB>
    __device__ __forceinline__ void rebase_edge(uint32_t &x, uint32_t keep, uint32_t d2) const {
        const uint32_t reset = __vcmpleu2(x, NEGp) | ~keep;
        const uint32_t y = __vmaxu2(SUB ? __vsubus2(x, d2) : __vaddus2(x, d2), NEGp + 0x10001u);
        x = mux(reset, NEGp, y);
    }
    // lane bits of the virtual row/column cells among the slots of anti-diagonal r
    __device__ __forceinline__ uint32_t virtual_bits(int32_t r) const {
        const int32_t B = frame(r);
        uint32_t vb = 0;
        if (r + 1 < qlen) vb |= slot_bit(-1 - B - j0);
        if (r >= -1 && r + 1 < tlen) vb |= slot_bit(r + 1 - B - j0);
        return vb;
    }
    // lane bits of the table's cells among the slots of anti-diagonal r
    __device__ __forceinline__ uint32_t table_bits(int32_t r) const {
        const int32_t st = max(max(0, r - qlen + 1), ceil_div2(r - w));
        const int32_t en = min(min(tlen - 1, r), floor_div2(r + w));
        const int32_t B = frame(r);
        return range_bits(st - B - j0, en - B - j0);
    }

    // Whether the head (anti-diagonals -1 .. w+1) can run on the bulk step:
    // the table reaches past it on both sides (no last row or column there,
    // no cell past the end), and the cells beyond the virtual row and column
    // stay within 16 bits and far below every other score: from minus
    // infinity they rise by at most a and fall by at most b every two
    // anti-diagonals, so after w+6 they sit within [NEG - b(w+6)/2 - q2 - e2,
    // NEG + a(w+6)/2], while the virtual cells and the band's maximum stay
    // above OFF - K D - gap(w+3) - a(w+3) (the maximum moves by at most D
    // per anti-diagonal between rebases).
    __device__ __forceinline__ bool head_on_bulk_step() const {
        if (min(tlen, qlen) <= w + 2 || w < 4) return false;
        return head_bounds_ok();
    }
    // A table that the head reaches past on neither side or one side only
    // (min(tlen, qlen) <= w + 2): the head up to w - 3 runs the tail step
    // instead (the same recurrence with the maximum taken over table cells
    // only, and the last row and column read), under the same bounds.
    __device__ __forceinline__ bool head_on_tail_step() const {
        if (min(tlen, qlen) > w + 2 || w < 8) return false;
        return head_bounds_ok();
    }
    __device__ __forceinline__ bool head_bounds_ok() const {
        const int64_t n = w + 6;
        const int64_t lo = (int64_t)U_NEG - (int64_t)prm.b * n / 2 - oe2;
        const int64_t hi = (int64_t)U_NEG + (int64_t)prm.a * n / 2;
        const int64_t floor_virt = (int64_t)OFF - (int64_t)cold.kint * cold.Dp - gap_cost(prm, w + 3) -
                                   (int64_t)prm.a * (w + 3);
        return lo > 2 * (int64_t)(prm.a + prm.b + oe2) && hi + 4 * (int64_t)cold.Dp < floor_virt;
    }

    // ------------------------------------------------------------------ pair
    // Returns false if the pair must be recomputed with int32 lanes.
    // DIR (fused): dt is the pair's direction table, one row per anti-diagonal
    // up to the last one the extension can reach.
    __device__ __forceinline__ bool run(const DevBatch &Bt, int32_t pair, int32_t lane_, bool use_fast,
                                        uint8_t *dt = nullptr) {
        prm = Bt.params;
        lane = lane_;
        tlen = Bt.t_len[pair]; qlen = Bt.q_len[pair];
        int32_t tph, qph;
        {
            const int64_t toff = Bt.t_off[pair], qoff = Bt.q_off[pair];
            const int64_t tw0 = toff >> 4, qw0 = qoff >> 4;
            tp = Bt.t_packed + tw0;
            qp = Bt.q_packed + qw0;
            tph = (int32_t)(toff & 15);
            qph = (int32_t)(qoff & 15);
            // the words the pair's bases occupy (inside the stream: checked by prep)
            tspan = (int32_t)min(Bt.t_words - tw0, (int64_t)((tph + tlen + 15) >> 4));
            qspan = (int32_t)min(Bt.q_words - qw0, (int64_t)((qph + qlen + 15) >> 4));
        }
        agatha_result *out = Bt.out + pair;
        if constexpr (DIR) { end_t = -1; end_q = -1; }
        if (tlen <= 0 || qlen <= 0) {
            if (leader()) write_empty_result(out);
            return true;
        }
        w = effective_w(prm.w, tlen, qlen);
        oe = prm.q + prm.e; oe2 = prm.q2 + prm.e2;
        j0 = (wk * G + lane) * C;
        last_r = tlen + qlen - 2;
        if constexpr (DIR) dtab = dt + j0;
        {
            const int32_t Dp = step_change_max(prm), kint = rebase_interval(Dp);
            until_rebase = kint;
            OFF = 0xffff - (kint + 3) * Dp;
            if (leader()) {
                cold.Dp = Dp;
                cold.kint = kint;
                cold.LOWCHK = (int32_t)U_NEG + (kint + 3) * Dp;
            }
        }
        base = 0;
        last_m = OFF;
        ovf = false;
        A2 = ((uint32_t)prm.a & 0xffffu) * 0x10001u;
        NABs = 0u - (uint32_t)(prm.a + prm.b);
        OEp = (uint32_t)oe * 0x10001u;
        DOEp = (uint32_t)(oe2 - oe) * 0x10001u;
        Ep = (uint32_t)prm.e * 0x10001u;
        E2p = (uint32_t)prm.e2 * 0x10001u;
        NEp = ((uint32_t)(-prm.e) & 0xffffu) * 0x10001u;
        NE2p = ((uint32_t)(-prm.e2) & 0xffffu) * 0x10001u;
        NEGp = U_NEG * 0x10001u;
        L0LO = (lane == 0 && wk == 0) ? 0x0000ffffu : 0u;
        L31HI = (lane == G - 1 && wk == K - 1) ? 0xffff0000u : 0u;
        xe0 = xe1 = NEGp;
#pragma unroll
        for (int p = 0; p < P; ++p) {
            Hev[p] = Hod[p] = Eo[p] = E2o[p] = Fo[p] = F2o[p] = NEGp;
        }
        {
            const int32_t k0 = min(max(w + 1 - j0, 0), C);     // first local slot beyond the band
            DF2 = (uint32_t)(k0 - 1) * 0x10001u;
            if constexpr (DMREG) {
#pragma unroll
                for (int p = 0; p < P; ++p)
                    DMR[p] = prmt(DF2 - ((uint32_t)p | ((uint32_t)(p + P) << 16)), 0, 0xbb99);
            }
        }
        gmax = 0;
        pend_r = -3;
        pend_rb = ~0u;
        if (leader()) {
            cold.mqe = K_NEG_OUT; cold.mqe_t = -1; cold.mte = K_NEG_OUT; cold.mte_q = -1;
            cold.gscore = K_NEG_OUT;
            cold.gt = -1; cold.gq = -1;
        }
        __syncwarp(gmask());
        group_sync();
        zdropped = 0;

        int32_t r = -2;
        init_windows(r, tph, qph);
        bool stop = head_step(r);
        const int32_t head_end = min(last_r, w + 1);
        // bulk: pairs starting at r = w + 2 ((r - w) even) while every band
        // cell of the pair is a real cell away from the last row and column
        const int32_t L = min(tlen, qlen);
        const int32_t bulk_last = 2 * L - 3 - w;
        int32_t limit = INT_MIN;          // the pair loop runs anti-diagonals up to here
        in_head = false;
        if (FHEAD && DEFER && K == 1 && use_fast && head_on_bulk_step()) {
            // The head on the bulk step, in the same pair loop as the bulk.
            // The virtual row (t = -1) and column (q = -1) then come out of
            // the recurrence itself, exactly, from the origin the first step
            // placed; cells beyond them (t < -1 or q < -1) never feed a cell
            // of the table or a virtual cell and stay far below both (checked
            // per pair by head_on_bulk_step).  The pair loop covers the head
            // anti-diagonals from the first with (r - w) even up to w - 3;
            // the masked step runs the others: r = w - 1, where the virtual
            // cells (-1, w) and (w, -1) sit in slot 0 and slot w + 1 outside
            // the band, r = w, which takes (w, -1) from beyond the frame when
            // w + 1 is its last slot, and the few around them.
            const int32_t ha = ((-1 - w) & 1) ? 0 : -1;
            while (!stop && r < ha - 1) {
                ++r;
                advance(r);
                stop = head_step(r);
            }
            in_head = true;
            limit = w - 3;
        } else if (FHEAD && DEFER && K == 1 && use_fast && head_on_tail_step()) {
            // The head of a short table: the virtual row and column again
            // come out of the recurrence (as on the bulk step above) up to
            // w - 3, where the tail step's maximum over table cells leaves
            // them out; the masked step runs the rest of the head.
            const int32_t ha = ((-1 - w) & 1) ? 0 : -1;
            while (!stop && r < ha - 1) {
                ++r;
                advance(r);
                stop = head_step(r);
            }
            in_head = true;
            const int32_t hz = min(w - 3, last_r);
            while (!stop && r < hz) {
                ++r;
                advance(r);
                stop = tail_step(r);
            }
            in_head = false;
            while (!stop && r < head_end) {
                ++r;
                advance(r);
                stop = head_step(r);
            }
            if (use_fast && !stop && r == w + 1) limit = bulk_last;
        } else {
            while (!stop && r < head_end) {
                ++r;
                advance(r);
                stop = head_step(r);
            }
            if (use_fast && !stop && r == w + 1) limit = bulk_last;
        }
        for (;;) {
            while (!stop && r + 2 <= limit) {
                const int st = fast_pair(r + 1);
                if (st >= 3) {
                    // a virtual cell may hold the maximum of r + st - 2: the
                    // maximum and the termination test over its band cells
                    r += st - 2;
                    until_rebase -= st - 2;
                    stop = ((r - w) & 1) ? head_band_max<true>(r) : head_band_max<false>(r);
                    break;
                }
                if (st) {
                    r += st;          // stopped (Z-drop or 16-bit overflow) on r+st
                    stop = true;
                    break;
                }
                r += 2;
            }
            if (FHEAD && in_head) {
                in_head = false;
                // the rest of the head on the masked step
                while (!stop && r < head_end) {
                    ++r;
                    advance(r);
                    stop = head_step(r);
                }
                if (!stop && r == w + 1) {
                    limit = bulk_last;
                    continue;
                }
                break;
            }
            locate_pending();
            break;
        }
        while (!stop && r < last_r) {     // r > w + 1 here
            ++r;
            advance(r);
            stop = tail_step(r);
        }
        if (ovf) return false;
        locate_pending();
        if constexpr (DIR) {
            // the traceback's start: the query end when reached, else the maximum
            const bool reach = !zdropped && cold.mqe != K_NEG_OUT && cold.mqe + prm.end_bonus > gmax;
            end_t = reach ? cold.mqe_t : cold.gt;
            end_q = reach ? qlen - 1 : cold.gq;
        }
        group_sync();           // K > 1: every warp's last writes to cold are in
        if (leader()) {
            agatha_result o;
            const int32_t mqe = cold.mqe;
            o.max = gmax; o.te = cold.gt; o.qe = cold.gq;
            o.gscore = cold.gscore; o.mqe = mqe; o.mqe_t = cold.mqe_t; o.mte = cold.mte;
            o.mte_q = cold.mte_q;
            // band cells of anti-diagonals 0 .. r (none on r when the band
            // left the table there)
            const int32_t st_r = max(max(0, r - qlen + 1), ceil_div2(r - w));
            const int32_t en_r = min(min(tlen - 1, r), floor_div2(r + w));
            o.cells = band_cells_through(tlen, qlen, w, st_r > en_r ? r - 1 : r);
            o.zdropped = (uint8_t)zdropped;
            o.reach_end = (uint8_t)(!zdropped && mqe != K_NEG_OUT && mqe + prm.end_bonus > gmax);
            o.lane16 = 1;
            for (int i = 0; i < 5; ++i) o.pad[i] = 0;
            *out = o;
        }
        return true;
    }

    // DIR: anti-diagonals 0..r_end with their direction bytes in
    // dt[r * 32C + lane byte]; no termination test.  Returns false if the
    // scores left the 16-bit range (the int32 kernel then takes the pair).
    __device__ __forceinline__ bool run_dir(const DevBatch &Bt, int32_t pair, int32_t lane_, int32_t r_end,
                                            uint8_t *dt) {
        static_assert(DIR, "run_dir needs the direction variant");
        prm = Bt.params;
        lane = lane_;
        tlen = Bt.t_len[pair]; qlen = Bt.q_len[pair];
        int32_t tph, qph;
        {
            const int64_t toff = Bt.t_off[pair], qoff = Bt.q_off[pair];
            const int64_t tw0 = toff >> 4, qw0 = qoff >> 4;
            tp = Bt.t_packed + tw0;
            qp = Bt.q_packed + qw0;
            tph = (int32_t)(toff & 15);
            qph = (int32_t)(qoff & 15);
            tspan = (int32_t)min(Bt.t_words - tw0, (int64_t)((tph + tlen + 15) >> 4));
            qspan = (int32_t)min(Bt.q_words - qw0, (int64_t)((qph + qlen + 15) >> 4));
        }
        w = effective_w(prm.w, tlen, qlen);
        oe = prm.q + prm.e; oe2 = prm.q2 + prm.e2;
        j0 = lane * C;
        last_r = r_end;
        dtab = dt + j0;
        {
            const int32_t Dp = step_change_max(prm), kint = rebase_interval(Dp);
            until_rebase = kint;
            OFF = 0xffff - (kint + 3) * Dp;
            if (lane == 0) {
                cold.Dp = Dp;
                cold.kint = kint;
                cold.LOWCHK = (int32_t)U_NEG + (kint + 3) * Dp;
            }
        }
        base = 0;
        last_m = OFF;
        ovf = false;
        A2 = ((uint32_t)prm.a & 0xffffu) * 0x10001u;
        NABs = 0u - (uint32_t)(prm.a + prm.b);
        OEp = (uint32_t)oe * 0x10001u;
        DOEp = (uint32_t)(oe2 - oe) * 0x10001u;
        Ep = (uint32_t)prm.e * 0x10001u;
        E2p = (uint32_t)prm.e2 * 0x10001u;
        NEp = ((uint32_t)(-prm.e) & 0xffffu) * 0x10001u;
        NE2p = ((uint32_t)(-prm.e2) & 0xffffu) * 0x10001u;
        NEGp = U_NEG * 0x10001u;
        L0LO = lane == 0 ? 0x0000ffffu : 0u;
        L31HI = lane == 31 ? 0xffff0000u : 0u;
#pragma unroll
        for (int p = 0; p < P; ++p) {
            Hev[p] = Hod[p] = Eo[p] = E2o[p] = Fo[p] = F2o[p] = NEGp;
        }
        {
            const int32_t k0 = min(max(w + 1 - j0, 0), C);
            DF2 = (uint32_t)(k0 - 1) * 0x10001u;
            if constexpr (DMREG) {
#pragma unroll
                for (int p = 0; p < P; ++p)
                    DMR[p] = prmt(DF2 - ((uint32_t)p | ((uint32_t)(p + P) << 16)), 0, 0xbb99);
            }
        }
        gmax = 0;
        pend_r = -3;
        __syncwarp(gmask());
        zdropped = 0;
        int32_t r = -2;
        init_windows(r, tph, qph);
        bool stop = head_step(r);
        const int32_t head_end = min(last_r, w + 1);
        while (!stop && r < head_end) {
            ++r;
            advance(r);
            stop = head_step(r);
        }
        const int32_t L = min(tlen, qlen);
        const int32_t bulk_last = min(2 * L - 3 - w, last_r);
        if (!stop && r == w + 1) {
            while (r + 2 <= bulk_last) {
                if (fast_pair(r + 1)) { stop = true; break; }    // only a 16-bit overflow stops it
                r += 2;
            }
        }
        while (!stop && r < last_r) {
            ++r;
            advance(r);
            stop = tail_step(r);
        }
        return !ovf;
    }
};

// G = 16: each half warp aligns its own pairs (two pairs per warp), taking
// them from the queue on its own.
template <int C, int MINB, int G = 32>
__global__ void __launch_bounds__(WARP_BLOCK_THREADS, MINB)
warp16_align_kernel(const DevBatch *__restrict__ d_batch, int32_t use_fast, int32_t list) {
    __shared__ Cold16 cold[WARP_BLOCK_THREADS / G];
    const DevBatch B = *d_batch;
    const int lane = threadIdx.x & (G - 1);
    const uint32_t gm = G == 32 ? FULL : 0xffffu << (threadIdx.x & 16);
    const WorkList L = work_list(B, list);
    // the larger register budget of each slot count: 4 blocks per SM for
    // 4 slots per lane, 2 for 20 and 24, 3 otherwise
    constexpr bool HIGH = C == 4 ? MINB == 4 : ((C == 24 || C == 20) ? MINB == 2 : MINB == 3);
    using Pair = WarpPair16<C, (MINB < 4 && C <= 16) || MINB < 3, true, false, true, 1, HIGH, HIGH, G>;
    if constexpr (G == 32) {
        for (;;) {
            int32_t k = 0;
            if (lane == 0) k = L.begin + atomicAdd(L.head, 1);
            k = __shfl_sync(gm, k, 0, G);
            if (k >= L.end) break;
            const int32_t pair = L.items ? L.items[k] : k;
            if (!L.items && (!pair_valid(B, pair) || !warp_takes(B, pair))) continue;
            Pair wp(cold[threadIdx.x / G]);
            if (!wp.run(B, pair, lane, use_fast != 0) && lane == 0) {
                const int32_t slot = atomicAdd(&B.counters[CTR_NOVF], 1);
                B.ovf_list[slot] = pair;
            }
        }
    } else {
        // The warp takes two neighbouring pairs of the longest-first queue at
        // once (about the same length), one per half, and both halves start
        // their next pairs together: the two then pass through the same step
        // variants at the same time for most of their anti-diagonals.
        for (;;) {
            int32_t k0 = 0;
            if ((threadIdx.x & 31) == 0) k0 = L.begin + atomicAdd(L.head, 2);
            k0 = __shfl_sync(FULL, k0, 0);
            if (k0 >= L.end) break;
            const int32_t k = k0 + (int32_t)((threadIdx.x >> 4) & 1);
            if (k < L.end) {
                const int32_t pair = L.items ? L.items[k] : k;
                if (L.items || (pair_valid(B, pair) && warp_takes(B, pair))) {
                    Pair wp(cold[threadIdx.x / G]);
                    if (!wp.run(B, pair, lane, use_fast != 0) && lane == 0) {
                        const int32_t slot = atomicAdd(&B.counters[CTR_NOVF], 1);
                        B.ovf_list[slot] = pair;
                    }
                }
            }
            __syncwarp();
        }
    }
    if (lane == 0) mark_step_end(B.counters);
}

// K warps of a block share one pair's band (K = 2: two pairs per block at a
// time, K = 4: one): for the longest pairs, whose anti-diagonals then take
// K times fewer steps of each warp (the paper's warps per task, Section 4.3,
// here grown instead of split).  The group's first warp takes the next pair
// from the queue and hands it to the others through shared memory.
template <int C, int K, int MINB>
__global__ void __launch_bounds__(WARP_BLOCK_THREADS, MINB)
warp16k_align_kernel(const DevBatch *__restrict__ d_batch, int32_t use_fast, int32_t list) {
    constexpr int G = WARP_BLOCK_THREADS / 32 / K;       // groups per block
    __shared__ Cold16 cold[G];
    __shared__ Xchg16 xch[G];
    const DevBatch B = *d_batch;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = warp / K, wk = warp % K;
    const int32_t bar = 1 + g;                           // named barrier of the group
    const WorkList L = work_list(B, list);
    for (;;) {
        WarpPair16<C, (MINB < 4 && C <= 16) || MINB < 3, true, false, true, K> wp(cold[g], &xch[g], wk, bar);
        if (wk == 0 && lane == 0) xch[g].pair = L.begin + atomicAdd(L.head, 1);
        wp.group_sync();
        const int32_t k = xch[g].pair;
        wp.group_sync();
        if (k >= L.end) break;
        const int32_t pair = L.items ? L.items[k] : k;
        if (!L.items && (!pair_valid(B, pair) || !warp_takes(B, pair))) continue;
        if (!wp.run(B, pair, lane, use_fast != 0) && lane == 0 && wk == 0) {
            const int32_t slot = atomicAdd(&B.counters[CTR_NOVF], 1);
            B.ovf_list[slot] = pair;
        }
    }
    if (lane == 0) mark_step_end(B.counters);
}

template <int C, int K, int MINB>
cudaError_t launch_warp16k_c(const DevBatch *d_batch, int n_blocks, cudaStream_t s, int use_fast,
                             int list) {
    warp16k_align_kernel<C, K, MINB><<<n_blocks, WARP_BLOCK_THREADS, 0, s>>>(d_batch, use_fast, list);
    return cudaGetLastError();
}

template <int C, int K, int MINB>
int occupancy_warp16k_c() {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, warp16k_align_kernel<C, K, MINB>,
                                                      WARP_BLOCK_THREADS, 0) != cudaSuccess)
        return 1;
    return nb > 0 ? nb : 1;
}

template <int C, int MINB, int G>
cudaError_t launch_warp16_c(const DevBatch *d_batch, int n_blocks, cudaStream_t s, int use_fast,
                            int list) {
    warp16_align_kernel<C, MINB, G><<<n_blocks, WARP_BLOCK_THREADS, 0, s>>>(d_batch, use_fast, list);
    return cudaGetLastError();
}

// The same launch at a given stream priority (lower is more urgent): the
// 24-slot launch ahead of the 20-slot one that runs beside it, whose blocks
// then take SMs only as the first one's blocks leave.
template <int C, int MINB>
cudaError_t launch_warp16_prio(const DevBatch *d_batch, int n_blocks, cudaStream_t s, int use_fast, int list,
                               int priority) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)n_blocks);
    cfg.blockDim = dim3(WARP_BLOCK_THREADS);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributePriority;
    attr[0].val.priority = priority;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, warp16_align_kernel<C, MINB, 32>, d_batch, use_fast, list);
}

template <int C, int MINB, int G>
int occupancy_warp16_c() {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, warp16_align_kernel<C, MINB, G>,
                                                      WARP_BLOCK_THREADS, 0) != cudaSuccess)
        return 1;
    return nb > 0 ? nb : 1;
}

}  // namespace agatha
