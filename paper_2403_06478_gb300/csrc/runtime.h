// Host-side internals of the library (not part of the C ABI).
#pragma once

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

#include "agatha.h"
#include "agatha_dev.cuh"

struct ServeState;

namespace agatha {

struct DevBuf {
    void *ptr = nullptr;
    size_t cap = 0;
    int ensure(agatha_ctx *ctx, size_t need);
    void release();
};

struct BatchShape {
    int64_t n = 0;
    int64_t max_len = 0;
    int32_t max_w_all = 0;    // widest effective band of any non-empty pair
    int32_t max_w_warp = 0;
};

struct LaunchPlan {
    int64_t n = 0;
    int plain = 0, sort = 1, fast = 1, use_graph = 1;
    int C = 16;
    int32_t warp_w_max = 0;
    int warp_blocks = 0;
    int lane16 = 0, C16 = 0, warp16_blocks = 0;
    int32_t wide_w = 0;         // > 0: pairs wider than the warp kernel exist
    int32_t plain_w = 0;
    int64_t plain_blocks = 0;
    std::tuple<int, int, int, int, int32_t, int> key() const {
        return std::make_tuple(plain, C + 100 * C16 * lane16, sort, fast, wide_w, warp_blocks);
    }
};

int set_error(agatha_ctx *ctx, int code, const char *fmt, ...);
int cuda_fail(agatha_ctx *ctx, cudaError_t e, const char *what);
int normalise_params(const agatha_params *in, DevParams *out);
int validate_host_batch(agatha_ctx *ctx, const agatha_batch *b, const DevParams &p, BatchShape *shape);
int pick_slots_per_lane(int32_t w);
int warp_occupancy(int C);

}  // namespace agatha

struct agatha_ctx {
    int device = 0;
    int n_sm = 0;
    int cc_major = 0, cc_minor = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t last_desc_stream = nullptr;
    int64_t mem_budget = 0;
    int64_t mem_held = 0;
    int64_t fail_alloc_after = -1;     // test hook: fail the n-th next allocation
    std::string tune_cache_path;
    std::mutex mu;                     // serialises align_batch calls
    std::mutex err_mu;
    std::string last_error, last_error_copy;
    agatha::DevBuf q_packed, t_packed, q_off, t_off, q_len, t_len, out, order, wide_order,
        ovf_list, counters, hist, desc;
    agatha::DevBatch *d_desc = nullptr;
    agatha::DevBatch *h_desc = nullptr;
    int32_t *h_counters = nullptr;
    bool graphs_stale = false;
    std::map<std::tuple<int, std::tuple<int, int, int, int, int32_t, int>>, cudaGraphExec_t> graphs;
    ServeState *serve = nullptr;
    bool timing = false;               // AGATHA_CFG_TIMING
    bool timed_once = false;
    cudaEvent_t ev_k0 = nullptr, ev_k1 = nullptr;
};
