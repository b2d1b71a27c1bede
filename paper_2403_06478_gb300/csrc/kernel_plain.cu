// Plain comparison kernel: one thread block aligns one pair, pairs in input
// order, one launch per batch.  This is the straightforward GPU design the
// batched kernel is measured against (paper Section 3.1: exact guiding on the
// baseline design).  The band of the current anti-diagonal is spread over the
// block's threads; its state lives in shared memory (three H buffers and two
// buffers of each gap state), the anti-diagonal maximum is a block reduction
// and every anti-diagonal ends with one __syncthreads().
//
// The kernel also serves pairs whose band is too wide for the warp kernel
// (use_wide_list = 1): it then walks the list the prep kernels built.
#include <climits>

#include "agatha_dev.cuh"

namespace agatha {

constexpr int PLAIN_MAX_THREADS = 1024;
constexpr int PLAIN_SMEM_LIMIT = 200 * 1024;

// 64-bit key: larger H first, then smaller t.  Invalid entries are 0.
__device__ __forceinline__ uint64_t plain_key(int32_t H, int32_t t) {
    return ((uint64_t)((uint32_t)H ^ 0x80000000u) << 32) | (uint32_t)(0x7fffffff - t);
}
__device__ __forceinline__ int32_t key_H(uint64_t k) { return (int32_t)((uint32_t)(k >> 32) ^ 0x80000000u); }
__device__ __forceinline__ int32_t key_t(uint64_t k) { return 0x7fffffff - (int32_t)(uint32_t)k; }

__device__ __forceinline__ uint32_t base_at(const uint32_t *__restrict__ p, int64_t n_words,
                                            int64_t off, int32_t i) {
    const int64_t g = off + i;
    return (load_word(p, n_words, g >> 4) >> (2 * (uint32_t)(g & 15))) & 3u;
}

__global__ void __launch_bounds__(PLAIN_MAX_THREADS)
plain_align_kernel(const DevBatch *__restrict__ d_batch, int32_t slots, int32_t use_wide_list) {
    extern __shared__ uint64_t sm64[];
    const DevBatch Bt = *d_batch;
    const DevParams P = Bt.params;
    const int32_t stride = slots + 1;              // slot `slots` is a permanent -inf
    uint64_t *red = sm64;                          // [2][32] per-warp max keys
    int32_t *redte = (int32_t *)(red + 64);        // [2][2][32] last row / column candidates
    int32_t *sm = redte + 128;
    int32_t *Hb = sm;                              // 3 * stride
    int32_t *Eb = Hb + 3 * stride;                 // 2 * stride each
    int32_t *E2b = Eb + 2 * stride;
    int32_t *Fb = E2b + 2 * stride;
    int32_t *F2b = Fb + 2 * stride;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, wid = tid >> 5, nwarps = (nt + 31) >> 5;
    const int64_t n_items = use_wide_list ? (int64_t)Bt.counters[CTR_NWIDE] : Bt.n_pairs;

    for (int64_t item = blockIdx.x; item < n_items; item += gridDim.x) {
        const int32_t pair = use_wide_list ? Bt.wide_order[item] : (int32_t)item;
        const int32_t tlen = Bt.t_len[pair], qlen = Bt.q_len[pair];
        const int64_t toff = Bt.t_off[pair], qoff = Bt.q_off[pair];
        agatha_result *out = Bt.out + pair;
        if (tlen <= 0 || qlen <= 0) {
            if (tid == 0) write_empty_result(out);
            continue;
        }
        const int32_t w = effective_w(P.w, tlen, qlen);
        if (w + 1 > slots) {                       // cannot happen for a valid launch
            if (tid == 0) atomicExch(&Bt.counters[CTR_ERR], DEV_ERR_BAD_PAIR);
            continue;
        }
        const int32_t oe = P.q + P.e, oe2 = P.q2 + P.e2;
        const int32_t last_r = tlen + qlen - 2;
        for (int i = tid; i < 3 * stride + 8 * stride; i += nt) sm[i] = K_NEG;
        __syncthreads();
        int32_t gmax = 0, gt = -1, gq = -1;
        int32_t mqe = K_NEG_OUT, mqe_t = -1, mte = K_NEG_OUT, mte_q = -1, gscore = K_NEG_OUT;
        int64_t cells = 0;
        int32_t zdropped = 0;

        for (int32_t r = -2; r <= last_r; ++r) {
            const int32_t B = ceil_div2(r - w);
            const int32_t d = (r - w) & 1;
            if (r >= 0) {
                const int32_t st = max(max(0, r - qlen + 1), B);
                const int32_t en = min(min(tlen - 1, r), floor_div2(r + w));
                if (st > en) { zdropped = 1; break; }
                cells += en - st + 1;
            }
            const int cur3 = (r + 3) % 3, prv2 = (r + 1) % 3;
            const int cur2 = r & 1, prv = (r - 1) & 1;
            int32_t *Hc = Hb + cur3 * stride;
            const int32_t *Hd = Hb + prv2 * stride;
            int32_t *Ec = Eb + cur2 * stride, *E2c = E2b + cur2 * stride;
            int32_t *Fc = Fb + cur2 * stride, *F2c = F2b + cur2 * stride;
            const int32_t *Ep = Eb + prv * stride, *E2p = E2b + prv * stride;
            const int32_t *Fp = Fb + prv * stride, *F2p = F2b + prv * stride;
            // E input of slot 0 on even steps: cell (B-1, r-B) of r-1
            int32_t injE = K_NEG, injE2 = K_NEG;
            if (B - 1 == -1 && r - B < qlen) {
                const int32_t qs = r - B;
                const int32_t v = (qs == -1) ? 0 : -gap_cost(P, qs + 1);
                injE = v - oe; injE2 = v - oe2;
            }
            uint64_t best = 0;
            int32_t te_c = INT_MIN, qe_c = INT_MIN;
            for (int32_t j = tid; j <= w; j += nt) {
                const int32_t t = B + j, q = r - t;
                const int32_t Ein = d ? Ep[j] : (j ? Ep[j - 1] : injE);
                const int32_t E2in = d ? E2p[j] : (j ? E2p[j - 1] : injE2);
                const int32_t Fin = d ? Fp[j + 1] : Fp[j];
                const int32_t F2in = d ? F2p[j + 1] : F2p[j];
                const int32_t k = t - q;
                const bool real = t >= 0 && q >= 0 && t < tlen && q < qlen && k <= w && -k <= w;
                int32_t H, ne, nf, ne2, nf2;
                if (real) {
                    const uint32_t tb = base_at(Bt.t_packed, Bt.t_words, toff, t);
                    const uint32_t qb = base_at(Bt.q_packed, Bt.q_words, qoff, q);
                    const int32_t s = tb == qb ? P.a : -P.b;
                    H = max(max(Hd[j] + s, Ein), max(max(Fin, E2in), F2in));
                    ne = max(H - oe, Ein - P.e);
                    nf = max(H - oe, Fin - P.e);
                    ne2 = max(H - oe2, E2in - P.e2);
                    nf2 = max(H - oe2, F2in - P.e2);
                    const uint64_t key = plain_key(H, t);
                    best = key > best ? key : best;
                    if (t == tlen - 1) te_c = H;
                    if (q == qlen - 1) qe_c = H;
                } else if ((t == -1 && q >= -1 && q < qlen) || (q == -1 && t >= 0 && t < tlen)) {
                    H = (t == -1 && q == -1) ? 0 : -gap_cost(P, (t == -1 ? q : t) + 1);
                    ne = nf = H - oe;
                    ne2 = nf2 = H - oe2;
                } else {
                    H = ne = nf = ne2 = nf2 = K_NEG;
                }
                Hc[j] = H; Ec[j] = ne; E2c[j] = ne2; Fc[j] = nf; F2c[j] = nf2;
            }
            // block reduction of the anti-diagonal maximum (double-buffered)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const uint64_t other = __shfl_xor_sync(0xffffffffu, best, o);
                best = other > best ? other : best;
                te_c = max(te_c, __shfl_xor_sync(0xffffffffu, te_c, o));
                qe_c = max(qe_c, __shfl_xor_sync(0xffffffffu, qe_c, o));
            }
            uint64_t *rb = red + (r & 1) * 32;
            int32_t *rte = redte + (r & 1) * 64;
            int32_t *rqe = rte + 32;
            if (lane == 0) { rb[wid] = best; rte[wid] = te_c; rqe[wid] = qe_c; }
            __syncthreads();
            if (r < 0) continue;
            uint64_t m = 0;
            int32_t te_v = INT_MIN, qe_v = INT_MIN;
            for (int i = 0; i < nwarps; ++i) {
                m = rb[i] > m ? rb[i] : m;
                te_v = max(te_v, rte[i]);
                qe_v = max(qe_v, rqe[i]);
            }
            if (te_v != INT_MIN && te_v > mte) { mte = te_v; mte_q = r - (tlen - 1); }
            if (qe_v != INT_MIN && qe_v > mqe) { mqe = qe_v; mqe_t = r - (qlen - 1); }
            const int32_t mH = key_H(m), mt = key_t(m), mq = r - mt;
            if (mH > gmax) {
                gmax = mH; gt = mt; gq = mq;
            } else if (mt >= gt && mq >= gq && P.zdrop >= 0) {
                int32_t l = (mt - gt) - (mq - gq);
                l = l < 0 ? -l : l;
                if (gmax - mH > P.zdrop + l * P.e2) { zdropped = 1; break; }
            }
            if (r == last_r && te_v != INT_MIN) gscore = te_v;
        }
        if (tid == 0) {
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
        __syncthreads();
    }
    if (threadIdx.x == 0) mark_step_end(Bt.counters);
}

static size_t plain_smem_bytes(int32_t slots) {
    const size_t stride = (size_t)slots + 1;
    return 64 * sizeof(uint64_t) + 128 * sizeof(int32_t) + 11 * stride * sizeof(int32_t);
}

int plain_kernel_max_w() {
    int32_t lo = 1, hi = 1 << 20;
    while (lo < hi) {
        const int32_t mid = (lo + hi + 1) / 2;
        if (plain_smem_bytes(mid + 1) <= (size_t)PLAIN_SMEM_LIMIT) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Raise the kernel's dynamic shared memory limit (once per device, outside
// any stream capture).
cudaError_t plain_kernel_prepare() {
    return cudaFuncSetAttribute(plain_align_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)PLAIN_SMEM_LIMIT + 4096);
}

cudaError_t launch_plain_kernel(const DevBatch *d_batch, int64_t n_blocks, int32_t w_max,
                                int use_wide_list, cudaStream_t s) {
    const int32_t slots = w_max + 1;
    const size_t smem = plain_smem_bytes(slots);
    if (smem > (size_t)PLAIN_SMEM_LIMIT) return cudaErrorInvalidValue;
    int threads = ((slots + 31) / 32) * 32;
    if (threads > PLAIN_MAX_THREADS) threads = PLAIN_MAX_THREADS;
    if (threads < 64) threads = 64;
    if (n_blocks <= 0) return cudaSuccess;
    if (n_blocks > (1 << 30)) n_blocks = 1 << 30;
    plain_align_kernel<<<(unsigned)n_blocks, threads, smem, s>>>(d_batch, slots, use_wide_list);
    return cudaGetLastError();
}

}  // namespace agatha
