// Autotuner: which kernel variant runs each length class of the ordered queue.
//
// The paper picks its slice width and subwarp size by sweeping them on its
// datasets (Sections 5.5 and 5.7).  Here the knobs are those of the warp
// kernels: 16-bit packed lanes or int32 lanes, the register budget of the
// 16-bit kernel (fewer resident warps, more registers each), and how many
// warps share one pair's band (1, 2 or 4: lanes per pair, for the classes of
// long pairs, whose anti-diagonals then take fewer steps of each warp).  They are
// chosen per length class, by measurement, the first time a host batch
// arrives for a scoring and band width: the pairs of each class (up to 4096,
// spread over the class) are aligned with every variant and the fastest one
// kept (a variant other than the default must win by 2% on these samples).
// The batch itself (up to 131072 of its pairs) is then timed as one launch of
// each 16-bit variant (and of int32 lanes if a class preferred them) and, if
// the classes disagree, as one launch per class; the fastest plan is kept
// (with a 1% margin, on the whole batch, for anything but one launch of the
// default variant).
// Every variant computes the same exact results, so the choice only moves
// time.  Choices are kept per context and, with a cache path, in a text file
// (one line per key: the key, the four class variants and the split flag).
#include <algorithm>
#include <cstdio>
#include <fstream>
#include <sstream>
#include <string>
#include <vector>

#include "runtime.h"

namespace agatha {

namespace {

constexpr int64_t kTuneMaxPairs = 4096;       // per class, to pick its variant
constexpr int64_t kTuneSplitPairs = 131072;   // of the whole batch, to decide the plan

std::string tune_key(const agatha_ctx *ctx, const DevParams &p, int C16) {
    char buf[256];
    std::snprintf(buf, sizeof(buf), "sm%d_cc%d%d_a%d_b%d_q%d_e%d_q2%d_e2%d_w%d_z%d_c%d", ctx->n_sm,
                  ctx->cc_major, ctx->cc_minor, p.a, p.b, p.q, p.e, p.q2, p.e2, p.w, p.zdrop, C16);
    return buf;
}

// (ctx->tune_mu held)
void tune_save(agatha_ctx *ctx) {
    if (ctx->tune_cache_path.empty()) return;
    const std::string tmp = ctx->tune_cache_path + ".tmp";
    {
        std::ofstream f(tmp, std::ios::trunc);
        if (!f) return;
        for (const auto &kv : ctx->tune_table) {
            f << kv.first;
            for (int8_t v : kv.second.var) f << ' ' << (int)v;
            f << ' ' << (int)kv.second.split << '\n';
        }
    }
    std::rename(tmp.c_str(), ctx->tune_cache_path.c_str());
}

// Median kernel time of three runs of a sub-batch under plan vp (after one
// untimed run).
int time_plan(agatha_ctx *ctx, const agatha_batch &sb, const DevParams &p, uint32_t flags,
              cudaStream_t s, LaunchPlan vp, std::vector<agatha_result> &res, float *ms) {
    vp.n = sb.n_pairs;
    vp.use_graph = 0;
    const uint32_t f = flags & ~(uint32_t)(AGATHA_DEVICE_PTRS | AGATHA_ASYNC);
    int rc = run_planned(ctx, &sb, p, res.data(), f, s, vp, nullptr, nullptr);
    if (rc) return rc;
    float t[3];
    for (float &x : t) {
        rc = run_planned(ctx, &sb, p, res.data(), f, s, vp, ctx->tune_ev0, ctx->tune_ev1);
        if (rc) return rc;
        const cudaError_t e = cudaEventElapsedTime(&x, ctx->tune_ev0, ctx->tune_ev1);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "tuning timer");
    }
    std::sort(t, t + 3);
    *ms = t[1];
    return AGATHA_OK;
}

LaunchPlan single_variant(LaunchPlan vp, int variant) {
    vp.split = 0;
    vp.lane16 = variant != VAR_32;
    vp.regs_high = variant == VAR_16_HIGHREG;
    vp.groupk = variant_warps(variant);
    vp.half = variant == VAR_16_HALF;
    return vp;
}

// Whether this plan can run a variant (the 2- and 4-warp kernels exist for
// the 16- and 24-slot bands only, two pairs per warp for the 4-slot band).
bool variant_available(const LaunchPlan &lp, int v) {
    if (v == VAR_16_HALF) return lp.warp16h_blocks > 0;
    const int K = variant_warps(v);
    return K == 1 || lp.warp16k_blocks[K == 4] > 0;
}

// A sub-batch of at most `cap` of the given pairs, spread over them.
struct SubBatch {
    std::vector<int64_t> qo, to;
    std::vector<int32_t> ql, tl;
    agatha_batch b;
    SubBatch(const agatha_batch *src, const std::vector<int64_t> &m, int64_t cap) {
        const int64_t k = std::min<int64_t>((int64_t)m.size(), cap);
        qo.resize(k); to.resize(k); ql.resize(k); tl.resize(k);
        for (int64_t j = 0; j < k; ++j) {
            const int64_t i = m[(size_t)(j * (int64_t)m.size() / k)];
            qo[j] = src->q_off[i]; to[j] = src->t_off[i]; ql[j] = src->q_len[i]; tl[j] = src->t_len[i];
        }
        b = *src;
        b.n_pairs = k;
        b.q_off = qo.data(); b.t_off = to.data(); b.q_len = ql.data(); b.t_len = tl.data();
    }
};

// A variant other than the default must win by this much to be taken: on a
// class's sample, and on the whole batch (repeatable to well under 1%).
constexpr float kMargin = 0.98f;
constexpr float kMarginBatch = 0.99f;

int tune_run(agatha_ctx *ctx, const agatha_batch *b, const DevParams &p, uint32_t flags, cudaStream_t s,
             const LaunchPlan &lp, TuneChoice *choice) {
    NvtxRange range("autotune");
    if (!ctx->tune_ev0 && (cudaEventCreate(&ctx->tune_ev0) != cudaSuccess ||
                           cudaEventCreate(&ctx->tune_ev1) != cudaSuccess)) {
        cudaGetLastError();
        return set_error(ctx, AGATHA_ECUDA, "tuning events");
    }
    std::vector<std::vector<int64_t>> members(N_CLASSES);
    std::vector<int64_t> all;
    for (int64_t i = 0; i < b->n_pairs; ++i) {
        const int32_t tl = b->t_len[i], ql = b->q_len[i];
        if (tl <= 0 || ql <= 0) continue;
        const int32_t w = effective_w(p.w, tl, ql);
        if (w > lp.warp_w_max) continue;             // aligned by the block kernel
        members[class_of_cells(predicted_cells(tl, ql, w))].push_back(i);
        all.push_back(i);
    }
    std::vector<agatha_result> res(std::min<int64_t>(std::max<int64_t>((int64_t)all.size(), 1), kTuneSplitPairs));
    if (all.empty()) return AGATHA_OK;                 // nothing the warp kernels take
    // 1. each length class on its own (up to kTuneMaxPairs of it): the
    //    fastest variant per class
    TuneChoice per;
    bool wins[N_VARIANTS] = {true, false, false, false, false};
    for (int c = 0; c < N_CLASSES; ++c) {
        per.var[c] = VAR_16;
        if (members[c].empty()) continue;
        SubBatch sb(b, members[c], kTuneMaxPairs);
        float t[N_VARIANTS];
        for (int v = 0; v < N_VARIANTS; ++v) {
            t[v] = 0.f;
            // warps sharing a pair only for the classes of long pairs
            if (!variant_available(lp, v) || (variant_warps(v) > 1 && c > 1)) continue;
            const int rc = time_plan(ctx, sb.b, p, flags, s, single_variant(lp, v), res, &t[v]);
            if (rc) return rc;
        }
        for (int v = 1; v < N_VARIANTS; ++v)
            if (t[v] > 0.f && t[v] < kMargin * t[per.var[c]]) per.var[c] = (int8_t)v;
        wins[per.var[c]] = true;
    }
    choice->split = 0;
    for (int c = 0; c < N_CLASSES; ++c) choice->var[c] = VAR_16;
    // 2. the batch itself (up to kTuneSplitPairs of it) as one launch of each
    //    16-bit variant (samples of a class can hide a few percent that the
    //    whole batch shows) and of int32 lanes if a class preferred them, and
    //    as one launch per class; the fastest plan is kept
    wins[VAR_16_HIGHREG] = true;
    SubBatch whole(b, all, kTuneSplitPairs);
    float best = 0.f;
    int best_v = VAR_16;
    for (int v = 0; v < N_VARIANTS; ++v) {
        if (!wins[v] || variant_warps(v) > 1) continue;    // the long classes' choice, not the batch's
        float t = 0.f;
        const int rc = time_plan(ctx, whole.b, p, flags, s, single_variant(lp, v), res, &t);
        if (rc) return rc;
        if (v == VAR_16) best = t;
        else if (t < kMarginBatch * best) { best = t; best_v = v; }
    }
    for (int c = 0; c < N_CLASSES; ++c) choice->var[c] = (int8_t)best_v;
    bool mixed = false;
    for (int c = 1; c < N_CLASSES; ++c) mixed |= per.var[c] != per.var[0];
    if (mixed) {
        // one launch per class costs its own tails
        LaunchPlan split = lp;
        split.split = 1;
        for (int c = 0; c < N_CLASSES; ++c) split.cls_var[c] = per.var[c];
        float t_split = 0.f;
        const int rc = time_plan(ctx, whole.b, p, flags, s, split, res, &t_split);
        if (rc) return rc;
        if (t_split < kMarginBatch * best) {
            *choice = per;
            choice->split = 1;
        }
    }
    return AGATHA_OK;
}

}  // namespace

void tune_load(agatha_ctx *ctx) {
    if (ctx->tune_cache_path.empty()) return;
    std::ifstream f(ctx->tune_cache_path);
    std::string line;
    while (f && std::getline(f, line)) {
        std::istringstream is(line);
        std::string key;
        TuneChoice v;
        bool ok = (bool)(is >> key);
        for (int c = 0; ok && c < N_CLASSES; ++c) {
            int x = -1;
            ok = (bool)(is >> x) && x >= 0 && x < N_VARIANTS;
            v.var[c] = (int8_t)x;
        }
        int sp = -1;
        ok = ok && (bool)(is >> sp) && (sp == 0 || sp == 1);
        v.split = (int8_t)sp;
        if (ok) ctx->tune_table[key] = v;        // malformed lines are ignored
    }
}

int tune_apply(agatha_ctx *ctx, const agatha_batch *batch, const DevParams &p, uint32_t flags,
               cudaStream_t s, LaunchPlan *lp) {
    const uint32_t off = AGATHA_NO_TUNE | AGATHA_PLAIN | AGATHA_FORCE32 | AGATHA_NO_SORT | AGATHA_REGS_HIGH |
                         AGATHA_WARPS2 | AGATHA_WARPS4 | AGATHA_HALF_WARP;
    if (!ctx->autotune || (flags & off) || lp->plain || !lp->lane16 || !lp->sort) return AGATHA_OK;
    const std::string key = tune_key(ctx, p, lp->C16);
    TuneChoice choice;
    bool found;
    {
        std::lock_guard<std::mutex> g(ctx->tune_mu);
        auto it = ctx->tune_table.find(key);
        found = it != ctx->tune_table.end();
        if (found) choice = it->second;
    }
    if (!found) {
        // lengths on the device (or a serving launch): the default plan
        if ((flags & AGATHA_DEVICE_PTRS) || !batch) return AGATHA_OK;
        const int rc = tune_run(ctx, batch, p, flags, s, *lp, &choice);
        if (rc) return rc;
        std::lock_guard<std::mutex> g(ctx->tune_mu);
        ctx->tune_table[key] = choice;
        tune_save(ctx);
    }
    if (!choice.split) {                        // one launch of one variant
        const int v = choice.var[0];
        if (!variant_available(*lp, v)) return AGATHA_OK;
        lp->lane16 = v != VAR_32;
        lp->regs_high = v == VAR_16_HIGHREG;
        lp->groupk = variant_warps(v);
        lp->half = v == VAR_16_HALF;
        return AGATHA_OK;
    }
    for (int c = 0; c < N_CLASSES; ++c)
        if (!variant_available(*lp, choice.var[c])) return AGATHA_OK;
    lp->split = 1;
    for (int c = 0; c < N_CLASSES; ++c) lp->cls_var[c] = choice.var[c];
    return AGATHA_OK;
}

}  // namespace agatha

using namespace agatha;

extern "C" int agatha_tune_variants(agatha_ctx *ctx, const agatha_params *params, int32_t w_max,
                                    int32_t *variants) {
    if (!ctx || !params || !variants) return AGATHA_EINVAL;
    DevParams p;
    if (normalise_params(params, &p)) return AGATHA_EINVAL;
    const int32_t w = w_max < 0 ? 32 * 32 - 1 : w_max;
    const int C16 = pick_slots16(w);
    if (C16 == 0 || step_change_max(p) > STEP16_MAX) return AGATHA_ENOTSUP;
    std::lock_guard<std::mutex> lock(ctx->tune_mu);
    auto it = ctx->tune_table.find(tune_key(ctx, p, C16));
    if (it == ctx->tune_table.end()) return AGATHA_EAGAIN;
    for (int c = 0; c < N_CLASSES; ++c) variants[c] = it->second.var[c];
    variants[N_CLASSES] = it->second.split;
    return AGATHA_OK;
}
