// agatha_align_batch_local: the BWA-MEM variant of the extension (local,
// from an initial score, row-by-row termination) through the batched path:
// validation and longest-first ordering by the prep kernels, then one warp
// per pair (kernel_local.cu).
#include <algorithm>
#include <cstring>
#include <mutex>

#include "agatha_dev.cuh"
#include "runtime.h"

using namespace agatha;

extern "C" int agatha_align_batch_local(agatha_ctx *ctx, const agatha_batch *batch,
                                        const agatha_params *params, const int32_t *h0,
                                        agatha_result *out, uint32_t flags, void *stream) {
    if (!ctx || !batch || !params) return AGATHA_EINVAL;
    std::lock_guard<std::mutex> lock(ctx->mu);
    NvtxRange range("agatha_align_batch_local");
    DevParams p;
    if (normalise_params(params, &p)) return set_error(ctx, AGATHA_EINVAL, "bad scoring parameters");
    if (p.w < 0) return set_error(ctx, AGATHA_ENOTSUP, "the local extension needs a band (w >= 1)");
    if (p.w > 32 * 16 - 1) return set_error(ctx, AGATHA_ENOTSUP, "band of %d is wider than 511", p.w);
    if (flags & AGATHA_PLAIN) return set_error(ctx, AGATHA_ENOTSUP, "no plain kernel for the local extension");
    if (batch->n_pairs < 0) return set_error(ctx, AGATHA_EINVAL, "negative n_pairs");
    const int64_t n = batch->n_pairs;
    if (n > 0 && (!out || !h0)) return set_error(ctx, AGATHA_EINVAL, "null out or h0");
    const bool dev = (flags & AGATHA_DEVICE_PTRS) != 0;
    if ((flags & AGATHA_ASYNC) && !dev) return set_error(ctx, AGATHA_EINVAL, "ASYNC needs DEVICE_PTRS");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
    cudaStream_t s = stream ? (cudaStream_t)stream : ctx->stream;
    if (n == 0) return AGATHA_OK;

    BatchShape shape;
    if (!dev) {
        int rc = validate_host_batch(ctx, batch, p, &shape);
        if (rc) return rc;
        for (int64_t i = 0; i < n; ++i)
            if (h0[i] < 1 || h0[i] > LOCAL_H0_MAX)
                return set_error(ctx, AGATHA_EINVAL, "pair %lld: initial score %d outside [1, %d]",
                                 (long long)i, h0[i], LOCAL_H0_MAX);
    } else {
        if (batch->q_words < 0 || batch->t_words < 0)
            return set_error(ctx, AGATHA_EINVAL, "negative stream size");
        shape.n = n;
        shape.max_len = 0;
        shape.max_w_all = p.w;
        shape.max_w_warp = p.w;
    }
    LaunchPlan lp;
    lp.n = n;
    lp.plain = 0;
    lp.sort = (flags & AGATHA_NO_SORT) ? 0 : 1;
    lp.fast = 0;
    lp.use_graph = 0;
    lp.C = pick_slots_per_lane(std::max<int32_t>(shape.max_w_all, 1));
    lp.warp_w_max = 32 * lp.C - 1;
    lp.lane16 = 0;
    lp.wide_w = 0;

    int rc;
    const int32_t *d_h0 = h0;
    if (!dev) {
        if ((rc = ctx->local_h0.ensure(ctx, ctx->ledger, (size_t)n * sizeof(int32_t)))) return rc;
        // the previous call may still read the old initial scores
        cudaStreamSynchronize(ctx->main.last_stream ? ctx->main.last_stream : s);
        if ((e = cudaMemcpyAsync(ctx->local_h0.ptr, h0, (size_t)n * sizeof(int32_t), cudaMemcpyHostToDevice,
                                 s)) != cudaSuccess)
            return cuda_fail(ctx, e, "copy h0");
        d_h0 = (const int32_t *)ctx->local_h0.ptr;
    }
    if ((rc = stage_batch(ctx, batch, p, out, flags, s, lp, d_h0))) return rc;
    Slot *sl = &ctx->main;
    const DevBatch *d = sl->d_desc;
    if ((e = cudaMemsetAsync(sl->counters.ptr, 0, CTR_COUNT * sizeof(int32_t), s)) != cudaSuccess ||
        (e = cudaMemsetAsync(sl->hist.ptr, 0, 256 * sizeof(int64_t), s)) != cudaSuccess ||
        (e = launch_prep(d, n, lp.sort, s, ctx->n_sm)) != cudaSuccess)
        return cuda_fail(ctx, e, "prep");
    if (ctx->timing && (e = cudaEventRecord(ctx->ev_k0, s)) != cudaSuccess) return cuda_fail(ctx, e, "event");
    if ((e = launch_local(lp.C, d, ctx->n_sm * local_occupancy(lp.C), s)) != cudaSuccess)
        return cuda_fail(ctx, e, "launch local");
    if (ctx->timing && (e = cudaEventRecord(ctx->ev_k1, s)) != cudaSuccess) return cuda_fail(ctx, e, "event");
    if ((e = cudaMemcpyAsync(sl->h_counters, sl->counters.ptr, CTR_COUNT * sizeof(int32_t),
                             cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return cuda_fail(ctx, e, "copy counters");
    if (!dev && (e = cudaMemcpyAsync(out, sl->out.ptr, (size_t)n * sizeof(agatha_result), cudaMemcpyDeviceToHost,
                                     s)) != cudaSuccess)
        return cuda_fail(ctx, e, "copy results");
    if (flags & AGATHA_ASYNC) return AGATHA_OK;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(ctx, e, "synchronize");
    if (ctx->timing) ctx->timed_once = true;
    if (sl->h_counters[CTR_ERR] != DEV_ERR_NONE)
        return set_error(ctx, AGATHA_EINVAL, "a pair has a bad length, offset, score range or initial score");
    return AGATHA_OK;
}
