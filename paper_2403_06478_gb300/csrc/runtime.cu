// Host runtime behind the C ABI: context, device buffers, batch validation,
// kernel selection, CUDA-graph replay and result copy-back.
#include <algorithm>
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include "agatha_dev.cuh"
#include "runtime.h"

using namespace agatha;

// ------------------------------------------------------------------ errors

const char *agatha_strerror(int code) {
    switch (code) {
        case AGATHA_OK: return "ok";
        case AGATHA_EINVAL: return "invalid argument";
        case AGATHA_ENOMEM: return "out of memory or over budget";
        case AGATHA_ECUDA: return "CUDA runtime error";
        case AGATHA_ETIMEDOUT: return "timed out";
        case AGATHA_EAGAIN: return "not ready";
        case AGATHA_ECANCELED: return "cancelled";
        case AGATHA_EDEVICE: return "device reported an error";
        case AGATHA_ENOTSUP: return "not supported";
        case AGATHA_ERANGE: return "output buffer too small";
        default: return "unknown error";
    }
}

int32_t agatha_version(void) { return 100; }

namespace agatha {

int set_error(agatha_ctx *ctx, int code, const char *fmt, ...) {
    if (ctx) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof(buf), fmt, ap);
        va_end(ap);
        std::lock_guard<std::mutex> g(ctx->err_mu);
        ctx->last_error = buf;
    }
    return code;
}

int cuda_fail(agatha_ctx *ctx, cudaError_t e, const char *what) {
    return set_error(ctx, AGATHA_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

// Grow a buffer to at least `need` bytes.  The caller has made sure no
// device work still uses the old allocation.
int DevBuf::ensure(agatha_ctx *ctx, Ledger &ledger, size_t need) {
    if (need <= cap) return AGATHA_OK;
    size_t want = std::max(need, cap + cap / 2);
    want = (want + 255) & ~(size_t)255;
    need = (need + 255) & ~(size_t)255;
    if (ledger.budget > 0 && ledger.held - (int64_t)cap + (int64_t)want > ledger.budget) {
        want = need;
        if (ledger.held - (int64_t)cap + (int64_t)want > ledger.budget)
            return set_error(ctx, AGATHA_ENOMEM, "device buffer of %zu bytes exceeds the budget", need);
    }
    release(ledger);
    cudaError_t e = cudaMalloc(&ptr, want);
    if (e != cudaSuccess) {
        ptr = nullptr;
        cudaGetLastError();
        return set_error(ctx, AGATHA_ENOMEM, "cudaMalloc(%zu): %s", want, cudaGetErrorString(e));
    }
    cap = want;
    ledger.held += (int64_t)want;
    return AGATHA_OK;
}

void DevBuf::release(Ledger &ledger) {
    if (ptr) {
        cudaFree(ptr);
        ledger.held -= (int64_t)cap;
    }
    ptr = nullptr;
    cap = 0;
}

// ------------------------------------------------------------- parameters

int normalise_params(const agatha_params *in, DevParams *out) {
    if (!in) return AGATHA_EINVAL;
    if (in->a < 0 || in->b < 0 || in->q < 0 || in->e < 0 || in->q2 < 0 || in->e2 < 0)
        return AGATHA_EINVAL;
    if (in->w == 0) return AGATHA_EINVAL;
    if (in->a > (1 << 16) || in->b > (1 << 16) || in->q > (1 << 20) || in->e > (1 << 16) ||
        in->q2 > (1 << 20) || in->e2 > (1 << 16) || in->end_bonus > (1 << 20) ||
        in->end_bonus < -(1 << 20) || in->zdrop > (1 << 27))
        return AGATHA_EINVAL;
    DevParams p;
    p.a = in->a; p.b = in->b; p.q = in->q; p.e = in->e; p.q2 = in->q2; p.e2 = in->e2;
    p.w = in->w < 0 ? -1 : in->w;
    p.zdrop = in->zdrop; p.end_bonus = in->end_bonus;
    if (p.q2 <= p.q || p.e2 >= p.e) { p.q2 = p.q; p.e2 = p.e; }
    *out = p;
    return AGATHA_OK;
}

static int64_t score_unit(const DevParams &p) {
    return (int64_t)p.a + p.b + p.q + p.e + p.q2 + p.e2 + (p.end_bonus > 0 ? p.end_bonus : 0);
}

// Host-side check of a host batch; fills the widest effective band.
int validate_host_batch(agatha_ctx *ctx, const agatha_batch *b, const DevParams &p,
                        BatchShape *shape) {
    if (!b || b->n_pairs < 0 || b->n_pairs > (int64_t)INT32_MAX - 1)
        return set_error(ctx, AGATHA_EINVAL, "bad batch or n_pairs");
    shape->n = b->n_pairs;
    shape->max_w_warp = 0;
    shape->max_w_all = 0;
    shape->max_len = 0;
    if (b->n_pairs == 0) return AGATHA_OK;
    if (!b->q_len || !b->t_len || !b->q_off || !b->t_off)
        return set_error(ctx, AGATHA_EINVAL, "null batch array");
    if (b->q_words < 0 || b->t_words < 0) return set_error(ctx, AGATHA_EINVAL, "negative stream size");
    if ((b->q_words > 0 && !b->q_packed) || (b->t_words > 0 && !b->t_packed))
        return set_error(ctx, AGATHA_EINVAL, "null packed stream");
    const int64_t unit = score_unit(p);
    for (int64_t i = 0; i < b->n_pairs; ++i) {
        const int32_t tl = b->t_len[i], ql = b->q_len[i];
        const int64_t to = b->t_off[i], qo = b->q_off[i];
        if (tl < 0 || ql < 0 || tl >= (1 << 24) || ql >= (1 << 24))
            return set_error(ctx, AGATHA_EINVAL, "pair %lld: bad length", (long long)i);
        if (to < 0 || qo < 0 || to + tl > b->t_words * 16 || qo + ql > b->q_words * 16)
            return set_error(ctx, AGATHA_EINVAL, "pair %lld: sequence outside its stream", (long long)i);
        if (unit * ((int64_t)tl + ql + 2) >= ((int64_t)1 << 28))
            return set_error(ctx, AGATHA_EINVAL, "pair %lld: scores could overflow int32", (long long)i);
        shape->max_len = std::max<int64_t>(shape->max_len, std::max(tl, ql));
        if (tl > 0 && ql > 0)
            shape->max_w_all = std::max(shape->max_w_all, effective_w(p.w, tl, ql));
    }
    return AGATHA_OK;
}

int pick_slots_per_lane(int32_t w) {
    const int cs[] = {4, 8, 16, 24, 32};
    for (int c : cs)
        if (32 * c - 1 >= w) return c;
    return 32;
}

static cudaError_t launch_warp(int C, const DevBatch *d, int blocks, cudaStream_t s, int fast,
                               int list) {
    switch (C) {
        case 4: return launch_warp_c<4>(d, blocks, s, fast, list);
        case 8: return launch_warp_c<8>(d, blocks, s, fast, list);
        case 16: return launch_warp_c<16>(d, blocks, s, fast, list);
        case 24: return launch_warp_c<24>(d, blocks, s, fast, list);
        default: return launch_warp_c<32>(d, blocks, s, fast, list);
    }
}

// 16-bit kernel with C slots per lane; high: the larger register budget
// (one resident block per SM fewer).
static cudaError_t launch_warp16(int C, int high, const DevBatch *d, int blocks, cudaStream_t s,
                                 int fast, int list) {
    switch (C * 2 + high) {
        case 8: return launch_warp16_c<4, 6>(d, blocks, s, fast, list);
        case 9: return launch_warp16_c<4, 4>(d, blocks, s, fast, list);
        case 16: return launch_warp16_c<8, 4>(d, blocks, s, fast, list);
        case 17: return launch_warp16_c<8, 3>(d, blocks, s, fast, list);
        case 32: return launch_warp16_c<16, 4>(d, blocks, s, fast, list);
        case 33: return launch_warp16_c<16, 3>(d, blocks, s, fast, list);
        case 48: return launch_warp16_c<24, 3>(d, blocks, s, fast, list);
        default: return launch_warp16_c<24, 2>(d, blocks, s, fast, list);
    }
}

// 16-bit kernel with two pairs per warp (16 lanes each) for the band of the
// C16-slot kernel: 8 slots per lane for the 4-slot band; none for wider ones.
static cudaError_t launch_warp16h(int C16, const DevBatch *d, int blocks, cudaStream_t s, int fast,
                                  int list) {
    if (C16 == 4) return launch_warp16_c<8, 3, 16>(d, blocks, s, fast, list);
    return cudaErrorInvalidValue;
}
int warp16h_occupancy(int C16) { return C16 == 4 ? occupancy_warp16_c<8, 3, 16>() : 0; }

// 16-bit kernel with K warps per pair, for the band of the C16-slot kernel:
// 2 warps of 8 or 12 slots per lane, 4 warps of 4 or 6.
static cudaError_t launch_warp16k(int C16, int K, const DevBatch *d, int blocks, cudaStream_t s,
                                  int fast, int list) {
    switch (C16 * 8 + K) {
        case 16 * 8 + 2: return launch_warp16k_c<8, 2, 4>(d, blocks, s, fast, list);
        case 24 * 8 + 2: return launch_warp16k_c<12, 2, 4>(d, blocks, s, fast, list);
        case 16 * 8 + 4: return launch_warp16k_c<4, 4, 6>(d, blocks, s, fast, list);
        case 24 * 8 + 4: return launch_warp16k_c<6, 4, 4>(d, blocks, s, fast, list);
        default: return cudaErrorInvalidValue;
    }
}

// Resident blocks per SM of that kernel; 0 where none exists for C16.
int warp16k_occupancy(int C16, int K) {
    switch (C16 * 8 + K) {
        case 16 * 8 + 2: return occupancy_warp16k_c<8, 2, 4>();
        case 24 * 8 + 2: return occupancy_warp16k_c<12, 2, 4>();
        case 16 * 8 + 4: return occupancy_warp16k_c<4, 4, 6>();
        case 24 * 8 + 4: return occupancy_warp16k_c<6, 4, 4>();
        default: return 0;
    }
}

cudaError_t launch_overflow_int32(const Slot *sl, const LaunchPlan &lp, cudaStream_t s) {
    return launch_warp(lp.C, sl->d_desc, lp.warp_blocks, s, lp.fast, WARP_LIST_OVERFLOW);
}

int warp16_occupancy(int C, int high) {
    switch (C * 2 + high) {
        case 8: return occupancy_warp16_c<4, 6>();
        case 9: return occupancy_warp16_c<4, 4>();
        case 16: return occupancy_warp16_c<8, 4>();
        case 17: return occupancy_warp16_c<8, 3>();
        case 32: return occupancy_warp16_c<16, 4>();
        case 33: return occupancy_warp16_c<16, 3>();
        case 48: return occupancy_warp16_c<24, 3>();
        default: return occupancy_warp16_c<24, 2>();
    }
}

// Slots per lane of the 16-bit kernel for a band of half-width w (0: none).
int pick_slots16(int32_t w) {
    if (w <= 32 * 4 - 1) return 4;
    if (w <= 32 * 8 - 1) return 8;
    if (w <= 32 * 16 - 1) return 16;
    if (w <= 32 * 24 - 1) return 24;
    return 0;
}

int warp_occupancy(int C) {
    switch (C) {
        case 4: return occupancy_warp_c<4>();
        case 8: return occupancy_warp_c<8>();
        case 16: return occupancy_warp_c<16>();
        case 24: return occupancy_warp_c<24>();
        default: return occupancy_warp_c<32>();
    }
}

// Enqueue the device work of one batch whose descriptor is already in the
// slot, in two parts: part 0 = validation and ordering, part 1 = the
// alignment kernels.  Each part is captured into its own CUDA graph (unless
// the caller asked otherwise) so timing events can sit between them.  The
// kernels find every batch buffer through the descriptor, so a graph stays
// valid when those buffers move; it bakes in only the slot's descriptor,
// counters and histogram, which never move.
static cudaError_t enqueue_part(agatha_ctx *ctx, Slot *sl, const LaunchPlan &lp, int part,
                                cudaStream_t s) {
    cudaError_t e = cudaSuccess;
    const DevBatch *d = sl->d_desc;
    if (part == 0) {
        e = cudaMemsetAsync(sl->counters.ptr, 0, CTR_COUNT * sizeof(int32_t), s);
        if (e != cudaSuccess) return e;
        if (!lp.plain) {
            e = cudaMemsetAsync(sl->hist.ptr, 0, 256 * sizeof(int64_t), s);
            if (e != cudaSuccess) return e;
        }
        // the plain path only validates (no sort); the batched path also orders
        return launch_prep(d, lp.n, lp.plain ? 0 : lp.sort, s, ctx->n_sm);
    }
    if (lp.plain) return launch_plain_kernel(d, lp.plain_blocks, lp.plain_w, 0, s);
    bool any16 = false;
    if (!lp.split) {
        if (lp.lane16 && lp.narrow_w > 0) {
            // the 24-slot launch and, beside it on a branch, the 20-slot one
            // over the pairs whose band fits 640 slots (the shortest); the
            // first at the higher priority, so that its blocks take the SMs
            // and the second's fill them as the first's leave
            if ((e = cudaEventRecord(sl->fork, s)) != cudaSuccess) return e;
            if ((e = cudaStreamWaitEvent(sl->aux[0], sl->fork, 0)) != cudaSuccess) return e;
            e = lp.regs_high ? launch_warp16_prio<24, 2>(d, lp.warp16_blocks[1], s, lp.fast, WARP_LIST_MAIN,
                                                         ctx->prio_greatest)
                             : launch_warp16_prio<24, 3>(d, lp.warp16_blocks[0], s, lp.fast, WARP_LIST_MAIN,
                                                         ctx->prio_greatest);
            if (e != cudaSuccess) return e;
            if ((e = launch_warp16_prio<20, 2>(d, lp.narrow_blocks, sl->aux[0], lp.fast, WARP_LIST_NARROW,
                                               ctx->prio_least)) != cudaSuccess)
                return e;
            if ((e = cudaEventRecord(sl->join[0], sl->aux[0])) != cudaSuccess) return e;
            if ((e = cudaStreamWaitEvent(s, sl->join[0], 0)) != cudaSuccess) return e;
            any16 = true;
        } else if (lp.lane16 && lp.half) {
            e = launch_warp16h(lp.C16, d, lp.warp16h_blocks, s, lp.fast, WARP_LIST_MAIN);
            any16 = true;
        } else if (lp.lane16 && lp.groupk > 1) {
            e = launch_warp16k(lp.C16, lp.groupk, d, lp.warp16k_blocks[lp.groupk == 4], s, lp.fast,
                               WARP_LIST_MAIN);
            any16 = true;
        } else if (lp.lane16) {
            e = launch_warp16(lp.C16, lp.regs_high, d, lp.warp16_blocks[lp.regs_high], s, lp.fast,
                              WARP_LIST_MAIN);
            any16 = true;
        } else {
            e = launch_warp(lp.C, d, lp.warp_blocks, s, lp.fast, WARP_LIST_MAIN);
        }
        if (e != cudaSuccess) return e;
    } else {
        // one launch per length class, each on its own branch so that the next
        // class's blocks take SMs as the longer class's blocks drain
        if ((e = cudaEventRecord(sl->fork, s)) != cudaSuccess) return e;
        for (int c = 0; c < N_CLASSES; ++c) {
            cudaStream_t sc = sl->aux[c];
            if ((e = cudaStreamWaitEvent(sc, sl->fork, 0)) != cudaSuccess) return e;
            const int v = lp.cls_var[c];
            if (v == VAR_32) {
                e = launch_warp(lp.C, d, lp.warp_blocks, sc, lp.fast, WARP_LIST_CLASS + c);
            } else if (v == VAR_16_HALF) {
                e = launch_warp16h(lp.C16, d, lp.warp16h_blocks, sc, lp.fast, WARP_LIST_CLASS + c);
                any16 = true;
            } else if (v == VAR_16_K2 || v == VAR_16_K4) {
                const int K = variant_warps(v);
                e = launch_warp16k(lp.C16, K, d, lp.warp16k_blocks[K == 4], sc, lp.fast, WARP_LIST_CLASS + c);
                any16 = true;
            } else {
                e = launch_warp16(lp.C16, v == VAR_16_HIGHREG, d, lp.warp16_blocks[v == VAR_16_HIGHREG],
                                  sc, lp.fast, WARP_LIST_CLASS + c);
                any16 = true;
            }
            if (e != cudaSuccess) return e;
            if ((e = cudaEventRecord(sl->join[c], sc)) != cudaSuccess) return e;
            if ((e = cudaStreamWaitEvent(s, sl->join[c], 0)) != cudaSuccess) return e;
        }
    }
    // pairs whose scores left the 16-bit range, recomputed on int32 lanes
    if (any16 && (e = launch_warp(lp.C, d, lp.warp_blocks, s, lp.fast, WARP_LIST_OVERFLOW)) != cudaSuccess)
        return e;
    if (lp.wide_w > 0) e = launch_plain_kernel(d, (int64_t)ctx->n_sm * 2, lp.wide_w, 1, s);
    return e;
}

static cudaError_t launch_part(agatha_ctx *ctx, Slot *sl, const LaunchPlan &lp, int part,
                               cudaStream_t s) {
    if (!lp.use_graph) return enqueue_part(ctx, sl, lp, part, s);
    const auto key = std::make_tuple(part, lp.key());
    auto it = sl->graphs.find(key);
    if (it == sl->graphs.end()) {
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return e;
        cudaError_t e1 = enqueue_part(ctx, sl, lp, part, s);
        e = cudaStreamEndCapture(s, &g);
        if (e1 != cudaSuccess) { if (g) cudaGraphDestroy(g); return e1; }
        if (e != cudaSuccess) return e;
        cudaGraphExec_t ge = nullptr;
        e = cudaGraphInstantiate(&ge, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return e;
        it = sl->graphs.emplace(key, ge).first;
    }
    return cudaGraphLaunch(it->second, s);
}

cudaError_t slot_run(agatha_ctx *ctx, Slot *sl, const LaunchPlan &lp, cudaStream_t s,
                     cudaEvent_t ev0, cudaEvent_t ev1) {
    cudaError_t e = launch_part(ctx, sl, lp, 0, s);
    if (e != cudaSuccess) return e;
    if (ev0 && (e = cudaEventRecord(ev0, s)) != cudaSuccess) return e;
    if ((e = launch_part(ctx, sl, lp, 1, s)) != cudaSuccess) return e;
    if (ev1) e = cudaEventRecord(ev1, s);
    return e;
}

int slot_init(agatha_ctx *ctx, Ledger &ledger, Slot *sl) {
    int rc;
    if ((rc = sl->counters.ensure(ctx, ledger, CTR_COUNT * sizeof(int32_t))) ||
        (rc = sl->hist.ensure(ctx, ledger, 256 * sizeof(int64_t))) ||
        (rc = sl->desc.ensure(ctx, ledger, sizeof(DevBatch))))
        return rc;
    sl->d_desc = (DevBatch *)sl->desc.ptr;
    for (int c = 0; c < N_CLASSES; ++c)
        if (cudaStreamCreateWithFlags(&sl->aux[c], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl->join[c], cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            return set_error(ctx, AGATHA_ECUDA, "slot streams");
        }
    if (cudaEventCreateWithFlags(&sl->fork, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        return set_error(ctx, AGATHA_ECUDA, "slot events");
    }
    if (cudaMallocHost(&sl->h_desc, sizeof(DevBatch)) != cudaSuccess ||
        cudaMallocHost(&sl->h_counters, CTR_COUNT * sizeof(int32_t)) != cudaSuccess) {
        cudaGetLastError();
        return set_error(ctx, AGATHA_ENOMEM, "pinned host staging");
    }
    return AGATHA_OK;
}

void slot_release(Ledger &ledger, Slot *sl) {
    for (auto &kv : sl->graphs) cudaGraphExecDestroy(kv.second);
    sl->graphs.clear();
    DevBuf *bufs[] = {&sl->q_packed, &sl->t_packed, &sl->q_off, &sl->t_off, &sl->q_len, &sl->t_len,
                      &sl->out, &sl->order, &sl->wide_order, &sl->ovf_list, &sl->counters, &sl->hist,
                      &sl->desc};
    for (DevBuf *b : bufs) b->release(ledger);
    if (sl->h_desc) cudaFreeHost(sl->h_desc);
    if (sl->h_counters) cudaFreeHost(sl->h_counters);
    for (int c = 0; c < N_CLASSES; ++c) {
        if (sl->aux[c]) cudaStreamDestroy(sl->aux[c]);
        if (sl->join[c]) cudaEventDestroy(sl->join[c]);
        sl->aux[c] = nullptr;
        sl->join[c] = nullptr;
    }
    if (sl->fork) cudaEventDestroy(sl->fork);
    sl->fork = nullptr;
    sl->h_desc = nullptr;
    sl->h_counters = nullptr;
    sl->d_desc = nullptr;
}

int slot_ensure(agatha_ctx *ctx, Ledger &ledger, Slot *sl, int64_t n, int64_t q_words,
                int64_t t_words, bool copy_inputs) {
    const int64_t n1 = std::max<int64_t>(n, 1);
    struct Need { DevBuf *b; size_t bytes; };
    std::vector<Need> needs = {{&sl->order, (size_t)n1 * 4}, {&sl->wide_order, (size_t)n1 * 4},
                               {&sl->ovf_list, (size_t)n1 * 4}};
    if (copy_inputs) {
        needs.push_back({&sl->q_packed, (size_t)std::max<int64_t>(q_words, 1) * 4});
        needs.push_back({&sl->t_packed, (size_t)std::max<int64_t>(t_words, 1) * 4});
        needs.push_back({&sl->q_off, (size_t)n1 * 8});
        needs.push_back({&sl->t_off, (size_t)n1 * 8});
        needs.push_back({&sl->q_len, (size_t)n1 * 4});
        needs.push_back({&sl->t_len, (size_t)n1 * 4});
        needs.push_back({&sl->out, (size_t)n1 * sizeof(agatha_result)});
    }
    bool grow = false;
    for (const Need &x : needs) grow |= x.bytes > x.b->cap;
    if (!grow) return AGATHA_OK;
    // the previous batch of this slot may still read the buffers being replaced
    if (sl->last_stream) cudaStreamSynchronize(sl->last_stream);
    int rc;
    for (const Need &x : needs)
        if ((rc = x.b->ensure(ctx, ledger, x.bytes))) return rc;
    return AGATHA_OK;
}

// Build the launch plan of a batch: which kernels, grids and graph key.
int make_plan(agatha_ctx *ctx, const DevParams &p, const BatchShape &shape, uint32_t flags,
              LaunchPlan *lp) {
    lp->n = shape.n;
    lp->plain = (flags & AGATHA_PLAIN) != 0;
    lp->sort = (flags & AGATHA_NO_SORT) ? 0 : 1;
    lp->fast = (flags & AGATHA_EDGE_PATH_ONLY) ? 0 : 1;
    lp->use_graph = (flags & (AGATHA_NO_GRAPH | AGATHA_PLAIN)) ? 0 : 1;
    const int32_t pmax = plain_kernel_max_w();
    if (lp->plain) {
        lp->C = 0;
        lp->plain_w = std::max<int32_t>(shape.max_w_all, 1);
        if (lp->plain_w > pmax)
            return set_error(ctx, AGATHA_ENOTSUP, "band of %d cells is wider than the plain kernel's %d",
                             lp->plain_w, pmax);
        lp->plain_blocks = std::max<int64_t>(shape.n, 1);
        lp->warp_blocks = 0;
        lp->wide_w = 0;
        lp->warp_w_max = 0;
        return AGATHA_OK;
    }
    lp->C = pick_slots_per_lane(shape.max_w_all);
    lp->warp_w_max = 32 * lp->C - 1;
    lp->wide_w = shape.max_w_all > lp->warp_w_max ? shape.max_w_all : 0;
    if (lp->wide_w > pmax)
        return set_error(ctx, AGATHA_ENOTSUP, "band of %d cells is wider than supported (%d)",
                         lp->wide_w, pmax);
    const int occ = warp_occupancy(lp->C);
    lp->warp_blocks = ctx->n_sm * occ;
    // 16-bit packed lanes when the band fits and one anti-diagonal changes a
    // score by at most 255 (the 16-bit kernel then still rebases at least
    // every 50 anti-diagonals)
    lp->C16 = pick_slots16(shape.max_w_all);
    lp->lane16 = !(flags & AGATHA_FORCE32) && lp->C16 > 0 && step_change_max(p) <= STEP16_MAX && !lp->wide_w;
    lp->regs_high = (flags & AGATHA_REGS_HIGH) ? 1 : 0;
    lp->split = 0;
    lp->groupk = 1;
    lp->half = 0;
    lp->warp16h_blocks = 0;
    if (lp->lane16) {
        lp->warp_w_max = 32 * lp->C16 - 1;
        lp->warp16_blocks[0] = ctx->n_sm * warp16_occupancy(lp->C16, 0);
        lp->warp16_blocks[1] = ctx->n_sm * warp16_occupancy(lp->C16, 1);
        lp->warp16k_blocks[0] = ctx->n_sm * warp16k_occupancy(lp->C16, 2);
        lp->warp16k_blocks[1] = ctx->n_sm * warp16k_occupancy(lp->C16, 4);
        const int K = (flags & AGATHA_WARPS4) ? 4 : ((flags & AGATHA_WARPS2) ? 2 : 1);
        if (K > 1 && (flags & AGATHA_HALF_WARP))
            return set_error(ctx, AGATHA_EINVAL, "two pairs per warp and several warps per pair");
        if (K > 1) {
            if (!lp->warp16k_blocks[K == 4])
                return set_error(ctx, AGATHA_ENOTSUP, "%d warps per pair need a band of 256 to 767", K);
            lp->groupk = K;
        }
        lp->warp16h_blocks = ctx->n_sm * warp16h_occupancy(lp->C16);
        if (flags & AGATHA_HALF_WARP) {
            if (!lp->warp16h_blocks)
                return set_error(ctx, AGATHA_ENOTSUP, "two pairs per warp need a band of at most 127");
            lp->half = 1;
        }
    }
    lp->plain_w = 0;
    lp->plain_blocks = 0;
    return AGATHA_OK;
}

// Frame per pair: on a single launch of the 24-slot 16-bit kernel with one
// warp per pair over the ordered queue, the pairs whose own band fits a
// 640-slot frame (w_eff <= 638) take the 20-slot kernel instead, after it
// (AGATHA_ONE_FRAME keeps every pair on the batch's frame).
void apply_narrow(agatha_ctx *ctx, LaunchPlan *lp, uint32_t flags) {
    lp->narrow_w = 0;
    lp->narrow_blocks = 0;
    if ((flags & AGATHA_ONE_FRAME) || !lp->lane16 || lp->plain || !lp->sort || lp->split || lp->groupk != 1 ||
        lp->half || lp->wide_w || lp->C16 != 24)
        return;
    const int occ = occupancy_warp16_c<20, 2>();
    if (occ <= 0) return;
    lp->narrow_w = 32 * 20 - 2;
    lp->narrow_blocks = ctx->n_sm * occ;
}

void fill_desc(const Slot *sl, DevBatch *d, const DevParams &p, const LaunchPlan &lp, void *order,
               void *wide_order, void *ovf_list) {
    d->order = (lp.sort && !lp.plain) ? (int32_t *)order : nullptr;
    d->counters = (int32_t *)sl->counters.ptr;
    d->wide_order = (int32_t *)wide_order;
    d->bucket_hist = (int64_t *)sl->hist.ptr;
    d->ovf_list = (int32_t *)ovf_list;
    d->h0 = nullptr;
    d->params = p;
    d->warp_w_max = lp.plain ? INT32_MAX : lp.warp_w_max;
    d->narrow_w_max = lp.plain ? 0 : lp.narrow_w;
}

}  // namespace agatha

// ------------------------------------------------------------------ ABI

extern "C" int agatha_check_params(const agatha_params *params, agatha_params *normalised) {
    DevParams p;
    int rc = normalise_params(params, &p);
    if (rc) return rc;
    if (normalised) {
        normalised->a = p.a; normalised->b = p.b; normalised->q = p.q; normalised->e = p.e;
        normalised->q2 = p.q2; normalised->e2 = p.e2; normalised->w = p.w;
        normalised->zdrop = p.zdrop; normalised->end_bonus = p.end_bonus;
    }
    return AGATHA_OK;
}

extern "C" int agatha_init(agatha_ctx **out, const agatha_config *cfg) {
    if (!out) return AGATHA_EINVAL;
    *out = nullptr;
    agatha_config c;
    std::memset(&c, 0, sizeof(c));
    if (cfg) c = *cfg;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess) { cudaGetLastError(); return AGATHA_ECUDA; }
    if (c.device < 0 || c.device >= ndev) return AGATHA_EINVAL;
    agatha_ctx *ctx = new (std::nothrow) agatha_ctx();
    if (!ctx) return AGATHA_ENOMEM;
    ctx->device = c.device;
    ctx->ledger.budget = c.mem_budget_bytes;
    if (c.tune_cache_path) ctx->tune_cache_path = c.tune_cache_path;
    if ((e = cudaSetDevice(c.device)) != cudaSuccess) { delete ctx; return AGATHA_ECUDA; }
    cudaDeviceProp prop;
    if ((e = cudaGetDeviceProperties(&prop, c.device)) != cudaSuccess) { delete ctx; return AGATHA_ECUDA; }
    ctx->n_sm = prop.multiProcessorCount;
    ctx->cc_major = prop.major;
    ctx->cc_minor = prop.minor;
    if (cudaDeviceGetStreamPriorityRange(&ctx->prio_least, &ctx->prio_greatest) != cudaSuccess) {
        cudaGetLastError();
        ctx->prio_least = ctx->prio_greatest = 0;
    }
    if ((e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking)) != cudaSuccess) {
        delete ctx;
        return AGATHA_ECUDA;
    }
    int rc = slot_init(ctx, ctx->ledger, &ctx->main);
    if (rc) {
        agatha_destroy(ctx);
        return rc;
    }
    ctx->autotune = (c.flags & AGATHA_CFG_AUTOTUNE) != 0;
    tune_load(ctx);
    if (c.flags & AGATHA_CFG_TIMING) {
        ctx->timing = true;
        if (cudaEventCreate(&ctx->ev_k0) != cudaSuccess || cudaEventCreate(&ctx->ev_k1) != cudaSuccess) {
            agatha_destroy(ctx);
            return AGATHA_ECUDA;
        }
    }
    if ((e = plain_kernel_prepare()) != cudaSuccess) {
        agatha_destroy(ctx);
        return AGATHA_ECUDA;
    }
    if (c.max_pairs > 0) slot_ensure(ctx, ctx->ledger, &ctx->main, c.max_pairs, 0, 0, true);
    *out = ctx;
    return AGATHA_OK;
}

extern "C" void agatha_destroy(agatha_ctx *ctx) {
    if (!ctx) return;
    agatha_serve_stop(ctx, 0);
    serve_free(ctx);
    cudaSetDevice(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    slot_release(ctx->ledger, &ctx->main);
    ctx->tb.release(ctx->ledger);
    ctx->local_h0.release(ctx->ledger);
    if (ctx->ev_tb0) cudaEventDestroy(ctx->ev_tb0);
    if (ctx->ev_tb1) cudaEventDestroy(ctx->ev_tb1);
    if (ctx->tune_ev0) cudaEventDestroy(ctx->tune_ev0);
    if (ctx->tune_ev1) cudaEventDestroy(ctx->tune_ev1);
    if (ctx->ev_k0) cudaEventDestroy(ctx->ev_k0);
    if (ctx->ev_k1) cudaEventDestroy(ctx->ev_k1);
    if (ctx->stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
}

extern "C" const char *agatha_last_error(agatha_ctx *ctx) {
    if (!ctx) return "no context";
    std::lock_guard<std::mutex> g(ctx->err_mu);
    ctx->last_error_copy = ctx->last_error;
    return ctx->last_error_copy.c_str();
}

namespace agatha {

// Copy one batch (host arrays) or point at it (device arrays) and write the
// descriptor of the context's slot for plan lp (ctx->mu held).
int stage_batch(agatha_ctx *ctx, const agatha_batch *batch, const DevParams &p, agatha_result *out,
                uint32_t flags, cudaStream_t s, const LaunchPlan &lp, const int32_t *d_h0) {
    const bool dev = (flags & AGATHA_DEVICE_PTRS) != 0;
    const int64_t n = batch->n_pairs;
    cudaError_t e;
    int rc;
    Slot *sl = &ctx->main;
    if ((rc = slot_ensure(ctx, ctx->ledger, sl, n, batch->q_words, batch->t_words, !dev))) return rc;

    DevBatch *d = sl->h_desc;
    // the previous call's descriptor upload must be finished before it is rewritten
    cudaStreamSynchronize(sl->last_stream ? sl->last_stream : s);
    if (!dev) {
        const int64_t qw = batch->q_words, tw = batch->t_words;
        if (qw > 0 && (e = cudaMemcpyAsync(sl->q_packed.ptr, batch->q_packed, qw * 4,
                                           cudaMemcpyHostToDevice, s)) != cudaSuccess)
            return cuda_fail(ctx, e, "copy q_packed");
        if (tw > 0 && (e = cudaMemcpyAsync(sl->t_packed.ptr, batch->t_packed, tw * 4,
                                           cudaMemcpyHostToDevice, s)) != cudaSuccess)
            return cuda_fail(ctx, e, "copy t_packed");
        if ((e = cudaMemcpyAsync(sl->q_off.ptr, batch->q_off, n * 8, cudaMemcpyHostToDevice, s)) ||
            (e = cudaMemcpyAsync(sl->t_off.ptr, batch->t_off, n * 8, cudaMemcpyHostToDevice, s)) ||
            (e = cudaMemcpyAsync(sl->q_len.ptr, batch->q_len, n * 4, cudaMemcpyHostToDevice, s)) ||
            (e = cudaMemcpyAsync(sl->t_len.ptr, batch->t_len, n * 4, cudaMemcpyHostToDevice, s)))
            return cuda_fail(ctx, e, "copy batch arrays");
        d->q_packed = (const uint32_t *)sl->q_packed.ptr;
        d->t_packed = (const uint32_t *)sl->t_packed.ptr;
        d->q_off = (const int64_t *)sl->q_off.ptr;
        d->t_off = (const int64_t *)sl->t_off.ptr;
        d->q_len = (const int32_t *)sl->q_len.ptr;
        d->t_len = (const int32_t *)sl->t_len.ptr;
        d->out = (agatha_result *)sl->out.ptr;
    } else {
        d->q_packed = batch->q_packed;
        d->t_packed = batch->t_packed;
        d->q_off = batch->q_off;
        d->t_off = batch->t_off;
        d->q_len = batch->q_len;
        d->t_len = batch->t_len;
        d->out = out;
    }
    d->q_words = batch->q_words;
    d->t_words = batch->t_words;
    d->n_pairs = n;
    fill_desc(sl, d, p, lp, sl->order.ptr, sl->wide_order.ptr, sl->ovf_list.ptr);
    d->h0 = d_h0;
    if ((e = cudaMemcpyAsync(sl->d_desc, d, sizeof(DevBatch), cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return cuda_fail(ctx, e, "copy descriptor");
    sl->last_stream = s;
    return AGATHA_OK;
}

// Stage one batch on the context's slot and run it with plan lp (ctx->mu held).
int run_planned(agatha_ctx *ctx, const agatha_batch *batch, const DevParams &p, agatha_result *out,
                uint32_t flags, cudaStream_t s, const LaunchPlan &lp, cudaEvent_t ev0, cudaEvent_t ev1) {
    const bool dev = (flags & AGATHA_DEVICE_PTRS) != 0;
    const int64_t n = batch->n_pairs;
    cudaError_t e;
    int rc;
    Slot *sl = &ctx->main;
    if ((rc = stage_batch(ctx, batch, p, out, flags, s, lp))) return rc;
    if ((e = slot_run(ctx, sl, lp, s, ev0, ev1)) != cudaSuccess) return cuda_fail(ctx, e, "launch");
    if ((e = cudaMemcpyAsync(sl->h_counters, sl->counters.ptr, CTR_COUNT * sizeof(int32_t),
                             cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return cuda_fail(ctx, e, "copy counters");
    if (!dev) {
        if ((e = cudaMemcpyAsync(out, sl->out.ptr, n * sizeof(agatha_result), cudaMemcpyDeviceToHost,
                                 s)) != cudaSuccess)
            return cuda_fail(ctx, e, "copy results");
    }
    if (flags & AGATHA_ASYNC) return AGATHA_OK;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(ctx, e, "synchronize");
    if (sl->h_counters[CTR_ERR] != DEV_ERR_NONE)
        return set_error(ctx, AGATHA_EINVAL, "a pair has a bad length, offset or score range");
    return AGATHA_OK;
}

}  // namespace agatha

extern "C" int agatha_align_batch(agatha_ctx *ctx, const agatha_batch *batch,
                                  const agatha_params *params, agatha_result *out, uint32_t flags,
                                  void *stream) {
    if (!ctx || !batch || !params) return AGATHA_EINVAL;
    std::lock_guard<std::mutex> lock(ctx->mu);
    NvtxRange range("agatha_align_batch");
    DevParams p;
    if (normalise_params(params, &p)) return set_error(ctx, AGATHA_EINVAL, "bad scoring parameters");
    if (batch->n_pairs < 0) return set_error(ctx, AGATHA_EINVAL, "negative n_pairs");
    if (batch->n_pairs > 0 && !out) return set_error(ctx, AGATHA_EINVAL, "null out");
    const bool dev = (flags & AGATHA_DEVICE_PTRS) != 0;
    if ((flags & AGATHA_ASYNC) && !dev) return set_error(ctx, AGATHA_EINVAL, "ASYNC needs DEVICE_PTRS");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
    cudaStream_t s = stream ? (cudaStream_t)stream : ctx->stream;
    const int64_t n = batch->n_pairs;
    if (n == 0) return AGATHA_OK;

    BatchShape shape;
    if (!dev) {
        int rc = validate_host_batch(ctx, batch, p, &shape);
        if (rc) return rc;
    } else {
        shape.n = n;
        shape.max_len = 0;
        // lengths live on the device: plan for the widest band the parameters allow
        shape.max_w_all = p.w >= 0 ? p.w : 32 * 32 - 1;
        shape.max_w_warp = shape.max_w_all;
        if (batch->q_words < 0 || batch->t_words < 0)
            return set_error(ctx, AGATHA_EINVAL, "negative stream size");
    }
    LaunchPlan lp;
    int rc = make_plan(ctx, p, shape, flags, &lp);
    if (rc) return rc;
    if (dev && p.w < 0 && !lp.plain) {
        // unbanded device batch: pairs wider than the warp kernel go to the block kernel
        lp.wide_w = plain_kernel_max_w();
    }
    if ((rc = tune_apply(ctx, batch, p, flags, s, &lp))) return rc;
    apply_narrow(ctx, &lp, flags);
    rc = run_planned(ctx, batch, p, out, flags, s, lp, ctx->timing ? ctx->ev_k0 : nullptr,
                     ctx->timing ? ctx->ev_k1 : nullptr);
    if (rc == AGATHA_OK) ctx->timed_once = true;
    return rc;
}

extern "C" int agatha_last_kernel_ms(agatha_ctx *ctx, float *ms) {
    if (!ctx || !ms) return AGATHA_EINVAL;
    if (!ctx->timing) return AGATHA_ENOTSUP;
    if (!ctx->timed_once) return AGATHA_EAGAIN;
    cudaError_t e = cudaEventSynchronize(ctx->ev_k1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, ctx->ev_k0, ctx->ev_k1);
    return e == cudaSuccess ? AGATHA_OK : cuda_fail(ctx, e, "kernel timing");
}

extern "C" int64_t agatha_band_cells(int32_t tlen, int32_t qlen, int32_t w) {
    if (tlen <= 0 || qlen <= 0) return 0;
    const int32_t we = effective_w(w, tlen, qlen);
    int64_t total = 0;
    for (int32_t t = 0; t < tlen; ++t) {
        const int32_t lo = std::max(0, t - we), hi = std::min(qlen - 1, t + we);
        if (hi >= lo) total += hi - lo + 1;
    }
    return total;
}

// ------------------------------------------------------------------ packing

static int pack_range(const uint8_t *codes, int64_t lo_word, int64_t hi_word, int64_t n, uint32_t *out,
                      bool ascii) {
    static const int8_t lut_init[256] = {0};
    (void)lut_init;
    int8_t lut[256];
    for (int i = 0; i < 256; ++i) lut[i] = -1;
    if (ascii) {
        lut['A'] = lut['a'] = 0; lut['C'] = lut['c'] = 1; lut['G'] = lut['g'] = 2; lut['T'] = lut['t'] = 3;
    } else {
        lut[0] = 0; lut[1] = 1; lut[2] = 2; lut[3] = 3;
    }
    int bad = 0;
    for (int64_t wi = lo_word; wi < hi_word; ++wi) {
        uint32_t word = 0;
        const int64_t base = wi * 16;
        const int64_t cnt = std::min<int64_t>(16, n - base);
        for (int64_t k = 0; k < cnt; ++k) {
            const int8_t c = lut[codes[base + k]];
            bad |= (c < 0);
            word |= (uint32_t)(c & 3) << (2 * k);
        }
        out[wi] = word;
    }
    return bad ? AGATHA_EINVAL : AGATHA_OK;
}

static int pack_impl(const uint8_t *codes, int64_t n, uint32_t *out, bool ascii) {
    if (n < 0 || (n > 0 && (!codes || !out))) return AGATHA_EINVAL;
    const int64_t words = (n + 15) / 16;
    const int64_t per = 1 << 20;
    if (words <= per) return pack_range(codes, 0, words, n, out, ascii);
    unsigned nt = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    std::vector<std::thread> th;
    std::atomic<int> rc{AGATHA_OK};
    const int64_t chunk = (words + nt - 1) / nt;
    for (unsigned i = 0; i < nt; ++i) {
        const int64_t lo = i * chunk, hi = std::min(words, lo + chunk);
        if (lo >= hi) break;
        th.emplace_back([=, &rc] {
            if (pack_range(codes, lo, hi, n, out, ascii)) rc = AGATHA_EINVAL;
        });
    }
    for (auto &t : th) t.join();
    return rc.load();
}

extern "C" int agatha_pack_codes(const uint8_t *codes, int64_t n, uint32_t *out) {
    return pack_impl(codes, n, out, false);
}

extern "C" int agatha_pack_ascii(const char *ascii, int64_t n, uint32_t *out) {
    return pack_impl((const uint8_t *)ascii, n, out, true);
}
