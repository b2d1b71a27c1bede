// Traceback entry point: the CIGAR of each extension of a host batch.
//
// 1. The score path runs as in agatha_align_batch (same plan, tuning and
//    results); it leaves the batch staged on the device.
// 2. Each pair's end cell follows from its result: the query end when the
//    extension reached it, else the cell of the maximum.  Pairs with an end
//    cell become traceback items, ordered by predicted work (anti-diagonals
//    up to the end x band width), longest first.
// 3. A direction table takes (r_end + 1) x 32C bytes per pair (C: slots per
//    lane of the warp kernel for the batch's widest band).  Items run in
//    waves whose tables fit the device memory this call may use; each wave
//    is one persistent launch of a traceback kernel (kernel_tb.cuh): the
//    16-bit one when the score path may use 16-bit lanes, else (and for the
//    pairs whose scores leave the 16-bit range, found from the run counts)
//    the int32 one.
// 4. The run counts come back to the host, which lays the CIGARs out in
//    input order; a gather kernel reverses each pair's runs into one dense
//    device array, copied to the caller's buffer in one transfer.
#include <algorithm>
#include <numeric>
#include <vector>

#include "runtime.h"

namespace agatha {

__global__ void cigar_gather_kernel(const TbItem *__restrict__ items, int32_t n_items,
                                    const int32_t *__restrict__ n_cigar,
                                    const int64_t *__restrict__ dst_off,
                                    const uint32_t *__restrict__ ops, uint32_t *__restrict__ dense) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t n_warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t k = warp; k < n_items; k += n_warps) {
        const TbItem it = items[k];
        const int32_t n = n_cigar[it.pair];
        const uint32_t *src = ops + it.ops_off;
        uint32_t *dst = dense + dst_off[it.pair];
        for (int32_t i = lane; i < n; i += 32) dst[i] = src[n - 1 - i];
    }
}

cudaError_t launch_cigar_gather(const TbItem *items, int32_t n_items, const int32_t *n_cigar,
                                const int64_t *dst_off, const uint32_t *ops, uint32_t *dense,
                                int n_blocks, cudaStream_t s) {
    cigar_gather_kernel<<<n_blocks, 256, 0, s>>>(items, n_items, n_cigar, dst_off, ops, dense);
    return cudaGetLastError();
}

namespace {

cudaError_t launch_tb(int C, const DevBatch *d, const TbItem *items, int32_t n, int32_t *head,
                      uint8_t *dir, uint32_t *ops, int32_t *ncig, int blocks, cudaStream_t s) {
    switch (C) {
        case 4: return launch_tb_c<4>(d, items, n, head, dir, ops, ncig, blocks, s);
        case 8: return launch_tb_c<8>(d, items, n, head, dir, ops, ncig, blocks, s);
        case 16: return launch_tb_c<16>(d, items, n, head, dir, ops, ncig, blocks, s);
        case 24: return launch_tb_c<24>(d, items, n, head, dir, ops, ncig, blocks, s);
        default: return launch_tb_c<32>(d, items, n, head, dir, ops, ncig, blocks, s);
    }
}

int tb_occupancy(int C) {
    switch (C) {
        case 4: return occupancy_tb_c<4>();
        case 8: return occupancy_tb_c<8>();
        case 16: return occupancy_tb_c<16>();
        case 24: return occupancy_tb_c<24>();
        default: return occupancy_tb_c<32>();
    }
}

// 16-bit traceback kernel for C16 slots per lane (4, 8, 16 or 24)
cudaError_t launch_tb16(int C, const DevBatch *d, const TbItem *items, int32_t n, int32_t *head,
                        uint8_t *dir, uint32_t *ops, int32_t *ncig, int blocks, cudaStream_t s) {
    switch (C) {
        case 4: return launch_tb16_c<4, 6>(d, items, n, head, dir, ops, ncig, blocks, s);
        case 8: return launch_tb16_c<8, 4>(d, items, n, head, dir, ops, ncig, blocks, s);
        case 16: return launch_tb16_c<16, 3>(d, items, n, head, dir, ops, ncig, blocks, s);
        default: return launch_tb16_c<24, 2>(d, items, n, head, dir, ops, ncig, blocks, s);
    }
}

// fused score path and traceback on 16-bit lanes
cudaError_t launch_tbf16(int C, const DevBatch *d, const TbItem *items, int32_t n, int32_t *head,
                         uint8_t *dir, uint32_t *ops, int32_t *ncig, int blocks, cudaStream_t s) {
    switch (C) {
        case 4: return launch_tbf16_c<4, 6>(d, items, n, head, dir, ops, ncig, blocks, s);
        case 8: return launch_tbf16_c<8, 4>(d, items, n, head, dir, ops, ncig, blocks, s);
        case 16: return launch_tbf16_c<16, 3>(d, items, n, head, dir, ops, ncig, blocks, s);
        default: return launch_tbf16_c<24, 2>(d, items, n, head, dir, ops, ncig, blocks, s);
    }
}

int tbf16_occupancy(int C) {
    switch (C) {
        case 4: return occupancy_tbf16_c<4, 6>();
        case 8: return occupancy_tbf16_c<8, 4>();
        case 16: return occupancy_tbf16_c<16, 3>();
        default: return occupancy_tbf16_c<24, 2>();
    }
}

int tb16_occupancy(int C) {
    switch (C) {
        case 4: return occupancy_tb16_c<4, 6>();
        case 8: return occupancy_tb16_c<8, 4>();
        case 16: return occupancy_tb16_c<16, 3>();
        default: return occupancy_tb16_c<24, 2>();
    }
}

// Grow a buffer to exactly `need` bytes (no headroom: direction tables are
// tens of GB).  The previous call's work on it has finished.
int ensure_exact(agatha_ctx *ctx, DevBuf &b, size_t need) {
    need = (std::max<size_t>(need, 1) + 255) & ~(size_t)255;
    if (need <= b.cap) return AGATHA_OK;
    b.release(ctx->ledger);
    if (ctx->ledger.budget > 0 && ctx->ledger.held + (int64_t)need > ctx->ledger.budget)
        return set_error(ctx, AGATHA_ENOMEM, "traceback buffer of %zu bytes exceeds the budget", need);
    const cudaError_t e = cudaMalloc(&b.ptr, need);
    if (e != cudaSuccess) {
        b.ptr = nullptr;
        cudaGetLastError();
        return set_error(ctx, AGATHA_ENOMEM, "cudaMalloc(%zu): %s", need, cudaGetErrorString(e));
    }
    b.cap = need;
    ctx->ledger.held += (int64_t)need;
    return AGATHA_OK;
}

// Largest direction table this call may hold: what is left of the budget, or
// most of the device's free memory (a few GB kept back for everything else).
int64_t dir_bytes_available(agatha_ctx *ctx) {
    const int64_t mine = (int64_t)ctx->tb.dir.cap;
    if (ctx->ledger.budget > 0) return ctx->ledger.budget - (ctx->ledger.held - mine);
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        cudaGetLastError();
        return mine;
    }
    const int64_t keep = std::min<int64_t>((int64_t)total_b / 16, (int64_t)4 << 30);
    return mine + std::max<int64_t>(0, (int64_t)free_b - keep);
}

}  // namespace
}  // namespace agatha

using namespace agatha;

extern "C" int agatha_align_cigar(agatha_ctx *ctx, const agatha_batch *batch, const agatha_params *params,
                                  agatha_result *out, int64_t *cigar_off, uint32_t *cigar,
                                  int64_t cigar_cap, uint32_t flags, void *stream) {
    if (!ctx || !batch || !params || !cigar_off) return AGATHA_EINVAL;
    if (flags & (AGATHA_DEVICE_PTRS | AGATHA_ASYNC))
        return set_error(ctx, AGATHA_ENOTSUP, "the traceback takes host buffers only");
    std::lock_guard<std::mutex> lock(ctx->mu);
    NvtxRange range("agatha_align_cigar");
    DevParams p;
    if (normalise_params(params, &p)) return set_error(ctx, AGATHA_EINVAL, "bad scoring parameters");
    const int64_t n = batch->n_pairs;
    if (n < 0) return set_error(ctx, AGATHA_EINVAL, "negative n_pairs");
    if (n > 0 && !out) return set_error(ctx, AGATHA_EINVAL, "null out");
    if (cigar_cap < 0 || (cigar_cap > 0 && !cigar)) return set_error(ctx, AGATHA_EINVAL, "bad cigar buffer");
    cigar_off[0] = 0;
    if (n == 0) return AGATHA_OK;
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
    cudaStream_t s = stream ? (cudaStream_t)stream : ctx->stream;

    BatchShape shape;
    int rc = validate_host_batch(ctx, batch, p, &shape);
    if (rc) return rc;
    if (shape.max_w_all > 32 * 32 - 1)
        return set_error(ctx, AGATHA_ENOTSUP, "traceback takes bands up to 1023 cells (this batch: %d)",
                         shape.max_w_all);

    // 1. plan: the fused kernel (score path and traceback in one pass, on
    //    16-bit lanes) unless the scoring or the flags rule 16-bit lanes out
    //    or ask for the two-pass form
    LaunchPlan lp;
    if ((rc = make_plan(ctx, p, shape, flags, &lp))) return rc;
    const int C32 = pick_slots_per_lane(std::max<int32_t>(shape.max_w_all, 1));
    const int C16 = pick_slots16(std::max<int32_t>(shape.max_w_all, 1));
    const bool use16 = C16 > 0 && step_change_max(p) <= STEP16_MAX && !(flags & AGATHA_FORCE32);
    const bool fused = use16 && lp.lane16 && !lp.wide_w && !(flags & (AGATHA_PLAIN | AGATHA_TB_TWO_PASS));
    Slot *sl = &ctx->main;
    if (fused) {
        if ((rc = stage_batch(ctx, batch, p, out, flags, s, lp))) return rc;
        if ((e = cudaMemsetAsync(sl->counters.ptr, 0, CTR_COUNT * sizeof(int32_t), s)))
            return cuda_fail(ctx, e, "clear counters");
    } else {
        // the score path first: its results give each pair's end cell
        if ((rc = tune_apply(ctx, batch, p, flags, s, &lp))) return rc;
        if ((rc = run_planned(ctx, batch, p, out, flags, s, lp, ctx->timing ? ctx->ev_k0 : nullptr,
                              ctx->timing ? ctx->ev_k1 : nullptr)))
            return rc;
        ctx->timed_once = true;
    }

    // 2. items, longest predicted work first.  A fused item covers every
    //    anti-diagonal of its pair (its end is found on the way); a two-pass
    //    item ends at its end cell.
    std::vector<TbItem> items;
    items.reserve((size_t)n);
    for (int64_t i = 0; i < n; ++i) {
        const int32_t tl = batch->t_len[i], ql = batch->q_len[i];
        if (tl <= 0 || ql <= 0) continue;
        int32_t et = tl - 1, eq = ql - 1;
        if (!fused) {
            const agatha_result &r = out[i];
            et = r.reach_end ? r.mqe_t : r.te;
            eq = r.reach_end ? ql - 1 : r.qe;
            if (et < 0 || eq < 0) continue;             // the maximum is the origin: empty CIGAR
        }
        TbItem it;
        it.pair = (int32_t)i; it.end_t = et; it.end_q = eq; it.pad = 0;
        it.dir_off = 0; it.ops_off = 0;
        items.push_back(it);
    }
    const int64_t n_items = (int64_t)items.size();
    {
        std::vector<int64_t> key((size_t)n_items);
        for (int64_t k = 0; k < n_items; ++k) {
            const TbItem &it = items[k];
            const int32_t w = effective_w(p.w, batch->t_len[it.pair], batch->q_len[it.pair]);
            key[k] = ((int64_t)it.end_t + it.end_q + 1) * (w + 1);
        }
        std::vector<int64_t> ord((size_t)n_items);
        std::iota(ord.begin(), ord.end(), 0);
        std::stable_sort(ord.begin(), ord.end(), [&](int64_t a, int64_t b) { return key[a] > key[b]; });
        std::vector<TbItem> sorted((size_t)n_items);
        for (int64_t k = 0; k < n_items; ++k) sorted[k] = items[ord[k]];
        items.swap(sorted);
    }
    int64_t ops_total = 0;
    for (TbItem &it : items) {
        it.ops_off = ops_total;
        ops_total += (int64_t)it.end_t + it.end_q + 2;
    }

    // 3. buffers, then waves of each kernel
    TbBufs &tb = ctx->tb;
    // (the dense copy of the runs is sized here too, to its bound, so that the
    // direction tables may take whatever is left)
    if ((rc = ensure_exact(ctx, tb.items, (size_t)std::max<int64_t>(2 * n_items, 1) * sizeof(TbItem))) ||
        (rc = ensure_exact(ctx, tb.ops, (size_t)std::max<int64_t>(ops_total, 1) * 4)) ||
        (rc = ensure_exact(ctx, tb.dense, (size_t)std::max<int64_t>(ops_total, 1) * 4)) ||
        (rc = ensure_exact(ctx, tb.n_cigar, (size_t)n * 4)) ||
        (rc = ensure_exact(ctx, tb.heads, (size_t)std::max<int64_t>(2 * n_items, 1) * 4)) ||
        (rc = ensure_exact(ctx, tb.dst_off, (size_t)(n + 1) * 8)))
        return rc;
    if ((e = cudaMemsetAsync(tb.heads.ptr, 0, (size_t)std::max<int64_t>(2 * n_items, 1) * 4, s)) ||
        (e = cudaMemsetAsync(tb.n_cigar.ptr, 0, (size_t)n * 4, s)))
        return cuda_fail(ctx, e, "clear traceback counters");
    if (ctx->timing && !ctx->ev_tb0 &&
        (cudaEventCreate(&ctx->ev_tb0) != cudaSuccess || cudaEventCreate(&ctx->ev_tb1) != cudaSuccess)) {
        cudaGetLastError();
        return set_error(ctx, AGATHA_ECUDA, "traceback timing events");
    }
    ctx->tb_ms = 0.f;
    int64_t item_base = 0, head_base = 0;     // where this kind's items / queue heads start
    enum { K_INT32 = 0, K_16 = 1, K_FUSED = 2 };
    // one kind of kernel over `list`: waves whose tables fit, each one launch
    auto run_kind = [&](std::vector<TbItem> &list, int kind) -> int {
        if (list.empty()) return AGATHA_OK;
        NvtxRange waves(kind == K_FUSED ? "traceback waves (fused)" :
                        (kind == K_16 ? "traceback waves (16-bit)" : "traceback waves (int32)"));
        const int C = kind == K_INT32 ? C32 : C16;
        const int64_t row = 32 * C;
        int64_t total = 0, largest = 0;
        for (const TbItem &it : list) {
            const int64_t bytes = ((int64_t)it.end_t + it.end_q + 1) * row;
            total += bytes;
            largest = std::max(largest, bytes);
        }
        int64_t cap = std::min(total, dir_bytes_available(ctx));
        if (cap < largest)
            return set_error(ctx, AGATHA_ENOMEM, "a direction table of %lld bytes does not fit in %lld",
                             (long long)largest, (long long)cap);
        int r2 = ensure_exact(ctx, tb.dir, (size_t)cap);
        if (r2) return r2;
        cap = std::max<int64_t>(cap, (int64_t)tb.dir.cap);
        std::vector<int64_t> begin;
        int64_t used = cap;                      // forces a new wave at the first item
        for (size_t k = 0; k < list.size(); ++k) {
            const int64_t bytes = ((int64_t)list[k].end_t + list[k].end_q + 1) * row;
            if (used + bytes > cap) {
                begin.push_back((int64_t)k);
                used = 0;
            }
            list[k].dir_off = used;
            used += bytes;
        }
        begin.push_back((int64_t)list.size());
        TbItem *d_items = (TbItem *)tb.items.ptr + item_base;
        cudaError_t e2 = cudaMemcpyAsync(d_items, list.data(), list.size() * sizeof(TbItem),
                                         cudaMemcpyHostToDevice, s);
        if (e2 != cudaSuccess) return cuda_fail(ctx, e2, "copy traceback items");
        if (ctx->timing && (e2 = cudaEventRecord(ctx->ev_tb0, s)) != cudaSuccess) return cuda_fail(ctx, e2, "event");
        const int occ = kind == K_INT32 ? tb_occupancy(C) : (kind == K_16 ? tb16_occupancy(C) : tbf16_occupancy(C));
        const int resident = ctx->n_sm * occ;
        for (size_t wv = 0; wv + 1 < begin.size(); ++wv) {
            const int64_t b = begin[wv], cnt = begin[wv + 1] - b;
            const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(resident, (cnt + 3) / 4));
            int32_t *head = (int32_t *)tb.heads.ptr + head_base + (int64_t)wv;
            uint8_t *dir = (uint8_t *)tb.dir.ptr;
            uint32_t *ops = (uint32_t *)tb.ops.ptr;
            int32_t *ncg = (int32_t *)tb.n_cigar.ptr;
            if (kind == K_FUSED) e2 = launch_tbf16(C, sl->d_desc, d_items + b, (int32_t)cnt, head, dir, ops, ncg, blocks, s);
            else if (kind == K_16) e2 = launch_tb16(C, sl->d_desc, d_items + b, (int32_t)cnt, head, dir, ops, ncg, blocks, s);
            else e2 = launch_tb(C, sl->d_desc, d_items + b, (int32_t)cnt, head, dir, ops, ncg, blocks, s);
            if (e2 != cudaSuccess) return cuda_fail(ctx, e2, "traceback launch");
        }
        if (ctx->timing && (e2 = cudaEventRecord(ctx->ev_tb1, s)) != cudaSuccess) return cuda_fail(ctx, e2, "event");
        if ((e2 = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(ctx, e2, "traceback");
        if (ctx->timing) {
            float ms = 0.f;
            if ((e2 = cudaEventElapsedTime(&ms, ctx->ev_tb0, ctx->ev_tb1)) != cudaSuccess)
                return cuda_fail(ctx, e2, "traceback timing");
            ctx->tb_ms += ms;
        }
        item_base += (int64_t)list.size();
        head_base += (int64_t)begin.size() - 1;
        (kind == K_INT32 ? ctx->tb_info.pairs32 : ctx->tb_info.pairs16) += (int64_t)list.size();
        if (kind == K_FUSED) ctx->tb_info.fused += (int64_t)list.size();
        ctx->tb_info.waves += (int64_t)begin.size() - 1;
        return AGATHA_OK;
    };
    ctx->tb_info = agatha_tb_info{0, 0, 0, 0};
    std::vector<int32_t> ncig((size_t)n);
    std::vector<TbItem> rest;
    if (fused) {
        if ((rc = run_kind(items, K_FUSED))) return rc;
        // pairs handed back (scores left the 16-bit range): the int32 score
        // kernel over the hand-back list, bracketed as the score kernels
        if (ctx->timing && (e = cudaEventRecord(ctx->ev_k0, s))) return cuda_fail(ctx, e, "event");
        if ((e = launch_overflow_int32(sl, lp, s))) return cuda_fail(ctx, e, "launch");
        if (ctx->timing && (e = cudaEventRecord(ctx->ev_k1, s))) return cuda_fail(ctx, e, "event");
        ctx->timed_once = true;
        if ((e = cudaMemcpyAsync(out, sl->out.ptr, (size_t)n * sizeof(agatha_result), cudaMemcpyDeviceToHost, s)) ||
            (e = cudaMemcpyAsync(ncig.data(), tb.n_cigar.ptr, (size_t)n * 4, cudaMemcpyDeviceToHost, s)) ||
            (e = cudaStreamSynchronize(s)))
            return cuda_fail(ctx, e, "copy results");
        // pairs with an empty sequence are no items: their result is the
        // empty one the score kernels write
        for (int64_t i = 0; i < n; ++i) {
            if (batch->t_len[i] > 0 && batch->q_len[i] > 0) continue;
            agatha_result &o = out[i];
            o.max = 0; o.qe = -1; o.te = -1;
            o.gscore = AGATHA_NEG_INF; o.mqe = AGATHA_NEG_INF; o.mte = AGATHA_NEG_INF;
            o.mqe_t = -1; o.mte_q = -1;
            o.cells = 0;
            o.zdropped = 0; o.reach_end = 0; o.lane16 = 0;
            for (int k = 0; k < 5; ++k) o.pad[k] = 0;
        }
        // handed-back pairs: an int32 two-pass traceback from their end cells,
        // or no runs when the maximum is the origin
        bool empty_path = false;
        for (const TbItem &it0 : items) {
            if (ncig[it0.pair] >= 0) continue;
            const agatha_result &r = out[it0.pair];
            TbItem it = it0;
            it.end_t = r.reach_end ? r.mqe_t : r.te;
            it.end_q = r.reach_end ? batch->q_len[it.pair] - 1 : r.qe;
            if (it.end_t < 0 || it.end_q < 0) {
                ncig[it0.pair] = 0;
                empty_path = true;
                continue;
            }
            rest.push_back(it);
        }
        if (empty_path && (e = cudaMemcpyAsync(tb.n_cigar.ptr, ncig.data(), (size_t)n * 4,
                                               cudaMemcpyHostToDevice, s)))
            return cuda_fail(ctx, e, "run counts");
        if ((rc = run_kind(rest, K_INT32))) return rc;
    } else if (use16) {
        if ((rc = run_kind(items, K_16))) return rc;
        if ((e = cudaMemcpy(ncig.data(), tb.n_cigar.ptr, (size_t)n * 4, cudaMemcpyDeviceToHost)))
            return cuda_fail(ctx, e, "traceback run counts");
        for (const TbItem &it : items)
            if (ncig[it.pair] < 0) rest.push_back(it);      // scores left the 16-bit range
        if ((rc = run_kind(rest, K_INT32))) return rc;
    } else {
        rest = items;
        if ((rc = run_kind(rest, K_INT32))) return rc;
    }

    // 4. layout in input order, gather, copy back
    NvtxRange gather("CIGAR gather and copy");
    if ((e = cudaMemcpyAsync(ncig.data(), tb.n_cigar.ptr, (size_t)n * 4, cudaMemcpyDeviceToHost, s)) ||
        (e = cudaStreamSynchronize(s)))
        return cuda_fail(ctx, e, "traceback run counts");
    ctx->tb_timed = ctx->timing;
    for (int64_t i = 0; i < n; ++i) cigar_off[i + 1] = cigar_off[i] + ncig[i];
    const int64_t total = cigar_off[n];
    if (total > cigar_cap)
        return set_error(ctx, AGATHA_ERANGE, "CIGARs need %lld runs, the buffer holds %lld",
                         (long long)total, (long long)cigar_cap);
    if (total == 0) return AGATHA_OK;
    if ((rc = ensure_exact(ctx, tb.dense, (size_t)total * 4))) return rc;
    if ((e = cudaMemcpyAsync(tb.dst_off.ptr, cigar_off, (size_t)(n + 1) * 8, cudaMemcpyHostToDevice, s)))
        return cuda_fail(ctx, e, "copy CIGAR offsets");
    // the gather walks the 16-bit kernel's items: every item (its n_cigar
    // is final now), or the int32 list when the 16-bit kernel did not run
    const TbItem *d_items = (const TbItem *)tb.items.ptr;
    const int gblocks = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)ctx->n_sm * 8, (n_items + 7) / 8));
    if ((e = launch_cigar_gather(d_items, (int32_t)n_items, (const int32_t *)tb.n_cigar.ptr,
                                 (const int64_t *)tb.dst_off.ptr, (const uint32_t *)tb.ops.ptr,
                                 (uint32_t *)tb.dense.ptr, gblocks, s)))
        return cuda_fail(ctx, e, "CIGAR gather");
    if ((e = cudaMemcpyAsync(cigar, tb.dense.ptr, (size_t)total * 4, cudaMemcpyDeviceToHost, s)) ||
        (e = cudaStreamSynchronize(s)))
        return cuda_fail(ctx, e, "copy CIGARs");
    return AGATHA_OK;
}

extern "C" int agatha_last_traceback_info(agatha_ctx *ctx, agatha_tb_info *info) {
    if (!ctx || !info) return AGATHA_EINVAL;
    std::lock_guard<std::mutex> lock(ctx->mu);
    *info = ctx->tb_info;
    return AGATHA_OK;
}

extern "C" int agatha_last_traceback_ms(agatha_ctx *ctx, float *ms) {
    if (!ctx || !ms) return AGATHA_EINVAL;
    if (!ctx->timing) return AGATHA_ENOTSUP;
    if (!ctx->tb_timed) return AGATHA_EAGAIN;
    *ms = ctx->tb_ms;
    return AGATHA_OK;
}
