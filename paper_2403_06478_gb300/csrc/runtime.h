// Host-side internals of the library (not part of the C ABI).
#pragma once

#include <array>
#include <condition_variable>
#include <cstdint>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <tuple>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "agatha.h"
#include "agatha_dev.cuh"

struct ServeState;

namespace agatha {

// An NVTX range for the lifetime of a scope: API calls and their phases show
// up by name in profiler timelines (header-only NVTX 3; free without a tool).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// Device bytes a context's own buffers hold, against its budget.
struct Ledger {
    int64_t budget = 0;            // 0: no limit
    int64_t held = 0;
};

struct DevBuf {
    void *ptr = nullptr;
    size_t cap = 0;
    int ensure(agatha_ctx *ctx, Ledger &ledger, size_t need);
    void release(Ledger &ledger);
};

struct BatchShape {
    int64_t n = 0;
    int64_t max_len = 0;
    int32_t max_w_all = 0;    // widest effective band of any non-empty pair
    int32_t max_w_warp = 0;
};

using PlanKey = std::array<int32_t, 12>;

// Kernel variant of a length class: 16-bit lanes (one warp per pair, at
// either register budget, or 2 / 4 warps sharing a pair's band) or int32 lanes.
// VAR_16_HALF: two pairs per warp, 16 lanes of 8 slots each (bands up to 127).
enum : int8_t {
    VAR_16 = 0, VAR_16_HIGHREG = 1, VAR_32 = 2, VAR_16_K2 = 3, VAR_16_K4 = 4, VAR_16_HALF = 5, N_VARIANTS = 6
};
inline int variant_warps(int v) { return v == VAR_16_K2 ? 2 : (v == VAR_16_K4 ? 4 : 1); }

// What the autotuner keeps per key: the variant of each length class and
// whether one launch per class beat a single launch.
struct TuneChoice {
    int8_t var[N_CLASSES] = {VAR_16, VAR_16, VAR_16, VAR_16};
    int8_t split = 0;
};

struct LaunchPlan {
    int64_t n = 0;
    int plain = 0, sort = 1, fast = 1, use_graph = 1;
    int C = 16;                 // slots per lane of the int32 kernel
    int32_t warp_w_max = 0;
    int warp_blocks = 0;
    int lane16 = 0, C16 = 0;    // 16-bit lanes allowed; their slots per lane
    int regs_high = 0;          // 16-bit kernel at its larger register budget
    int warp16_blocks[2] = {0, 0};   // grid of the 16-bit kernel per budget
    int groupk = 1;             // warps per pair of the single launch (1, 2, 4)
    int warp16k_blocks[2] = {0, 0};  // grids of the 2- and 4-warp kernels (0: none)
    int half = 0;               // the single launch runs two pairs per warp
    int warp16h_blocks = 0;     // grid of that kernel (0: none for this band)
    int32_t narrow_w = 0;       // > 0: pairs whose band is at most this run on
                                // the 20-slot frame, beside the 24-slot launch
    int narrow_blocks = 0;      // grid of that kernel
    int split = 0;              // one launch per length class, variant cls_var[c]
    int8_t cls_var[N_CLASSES] = {VAR_16, VAR_16, VAR_16, VAR_16};
    int32_t wide_w = 0;         // > 0: pairs wider than the warp kernel exist
    int32_t plain_w = 0;
    int64_t plain_blocks = 0;
    PlanKey key() const {
        return {plain, C, C16 * lane16, regs_high, sort, fast, wide_w, warp_blocks, split,
                split ? cls_var[0] | (cls_var[1] << 4) | (cls_var[2] << 8) | (cls_var[3] << 12) : 0,
                split ? 1 : groupk, (split ? 0 : half) | (narrow_w > 0 ? 2 : 0)};
    }
};

// Everything one batch needs on the device: input copies (host batches),
// results, scheduling scratch, the descriptor the kernels read, and the
// CUDA graphs captured for this slot (they bake in the slot's addresses).
struct Slot {
    DevBuf q_packed, t_packed, q_off, t_off, q_len, t_len, out, order, wide_order, ovf_list,
        counters, hist, desc;
    DevBatch *d_desc = nullptr;
    DevBatch *h_desc = nullptr;       // pinned staging of the descriptor
    cudaStream_t aux[N_CLASSES] = {}; // branches of the per-class launches
    cudaEvent_t fork = nullptr, join[N_CLASSES] = {};
    int32_t *h_counters = nullptr;    // pinned copy of the counters after a batch
    cudaStream_t last_stream = nullptr;
    std::map<std::tuple<int, PlanKey>, cudaGraphExec_t> graphs;
};

// Device buffers of the traceback path (tb.cu), kept for later calls.
struct TbBufs {
    DevBuf dir, ops, items, n_cigar, heads, dst_off, dense;
    void release(Ledger &ledger) {
        DevBuf *b[] = {&dir, &ops, &items, &n_cigar, &heads, &dst_off, &dense};
        for (DevBuf *x : b) x->release(ledger);
    }
};

int set_error(agatha_ctx *ctx, int code, const char *fmt, ...);
int cuda_fail(agatha_ctx *ctx, cudaError_t e, const char *what);
int normalise_params(const agatha_params *in, DevParams *out);
int validate_host_batch(agatha_ctx *ctx, const agatha_batch *b, const DevParams &p, BatchShape *shape);
int pick_slots_per_lane(int32_t w);
int pick_slots16(int32_t w);
int warp_occupancy(int C);
int warp16_occupancy(int C, int high);
int warp16h_occupancy(int C16);   // two pairs per warp; 0 where none exists
void apply_narrow(agatha_ctx *ctx, LaunchPlan *lp, uint32_t flags);
int warp16k_occupancy(int C16, int K);

int slot_init(agatha_ctx *ctx, Ledger &ledger, Slot *s);
void slot_release(Ledger &ledger, Slot *s);
int slot_ensure(agatha_ctx *ctx, Ledger &ledger, Slot *s, int64_t n, int64_t q_words,
                int64_t t_words, bool copy_inputs);
int make_plan(agatha_ctx *ctx, const DevParams &p, const BatchShape &shape, uint32_t flags,
              LaunchPlan *lp);
// Fill the scheduling fields of a descriptor; order/wide_order/ovf_list are
// device arrays of n_pairs int32 each.
void fill_desc(const Slot *s, DevBatch *d, const DevParams &p, const LaunchPlan &lp, void *order,
               void *wide_order, void *ovf_list);
// Enqueue validation, ordering and the alignment kernels of the batch whose
// descriptor is in s->d_desc; ev0/ev1 (may be null) bracket the kernels.
cudaError_t slot_run(agatha_ctx *ctx, Slot *s, const LaunchPlan &lp, cudaStream_t st,
                     cudaEvent_t ev0, cudaEvent_t ev1);
// Stop and free the context's server, if any (serve.cu).
void serve_free(agatha_ctx *ctx);

// Copy (host arrays) or reference (device arrays) one batch on the context's
// own slot and write its descriptor for plan lp, without launching anything.
int stage_batch(agatha_ctx *ctx, const agatha_batch *batch, const DevParams &p, agatha_result *out,
                uint32_t flags, cudaStream_t s, const LaunchPlan &lp, const int32_t *d_h0 = nullptr);
// The int32 kernel over the 16-bit kernels' hand-back list of the slot's batch.
cudaError_t launch_overflow_int32(const Slot *sl, const LaunchPlan &lp, cudaStream_t s);
// Stage one batch on the context's own slot and run it with plan lp; ev0/ev1
// (may be null) bracket the alignment kernels.  ctx->mu must be held.
int run_planned(agatha_ctx *ctx, const agatha_batch *batch, const DevParams &p, agatha_result *out,
                uint32_t flags, cudaStream_t s, const LaunchPlan &lp, cudaEvent_t ev0, cudaEvent_t ev1);

// Autotuner (tune.cu): read the cache file; turn lp into per-class launches
// with the tuned variants, measuring them first if this key is new and the
// batch is on the host.
void tune_load(agatha_ctx *ctx);
int tune_apply(agatha_ctx *ctx, const agatha_batch *batch, const DevParams &p, uint32_t flags,
               cudaStream_t s, LaunchPlan *lp);

}  // namespace agatha

struct agatha_ctx {
    int device = 0;
    int n_sm = 0;
    int cc_major = 0, cc_minor = 0;
    int prio_least = 0, prio_greatest = 0;   // the device's stream priority range
    cudaStream_t stream = nullptr;
    agatha::Ledger ledger;
    std::string tune_cache_path;
    std::mutex mu;                     // serialises align_batch calls
    std::mutex err_mu;
    std::string last_error, last_error_copy;
    agatha::Slot main;                 // buffers of agatha_align_batch
    ServeState *serve = nullptr;
    bool timing = false;               // AGATHA_CFG_TIMING
    bool timed_once = false;
    cudaEvent_t ev_k0 = nullptr, ev_k1 = nullptr;
    bool autotune = false;             // AGATHA_CFG_AUTOTUNE
    std::mutex tune_mu;                // guards tune_table (align_batch and the server read it)
    std::map<std::string, agatha::TuneChoice> tune_table;
    cudaEvent_t tune_ev0 = nullptr, tune_ev1 = nullptr;
    agatha::TbBufs tb;                 // traceback buffers (agatha_align_cigar)
    agatha::DevBuf local_h0;           // initial scores of agatha_align_batch_local (host batches)
    cudaEvent_t ev_tb0 = nullptr, ev_tb1 = nullptr;
    bool tb_timed = false;
    float tb_ms = 0.f;                 // traceback kernels of the last call
    agatha_tb_info tb_info = {0, 0, 0, 0};
};
