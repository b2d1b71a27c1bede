// Serving loop: continuous batching of alignment requests on one device.
//
// Requests arrive one by one (a read's candidate extensions, say) with host
// buffers.  Submission validates a request, copies the sequence words its
// pairs touch into server-owned memory and queues it.  One scheduler thread
// per server turns the queue into device launches:
//
//  * Merging.  Whenever a launch slot is free, the queued requests that share
//    the head request's (normalised) scoring are concatenated into one batch,
//    up to max_batch_pairs pairs; the device orders the merged pairs by
//    predicted work like any other batch (Section 4.5 model), so short and
//    long requests share one persistent-kernel queue.  Results do not depend
//    on what a pair is batched with: every pair is aligned independently.
//  * Admission.  Every launch takes one block of a device arena whose size is
//    the memory budget, so the bytes admitted requests hold can never exceed
//    it.  A request that alone needs more than the arena is refused at
//    submission (AGATHA_ENOMEM); a batch that does not fit now waits for a
//    running launch to give its block back.
//  * Overlap.  Up to max_inflight launches are on the device at once, each on
//    its own stream with its own descriptor, counters and captured graphs, so
//    the next batch's upload and ordering run under the previous batch's tail.
//    Completion is signalled by a host function enqueued after the result
//    copy; the scheduler then scatters results into the callers' buffers.
//
// Lock order: the scheduler never holds the server mutex while it calls the
// CUDA runtime, and the completion host function takes only that mutex, so a
// CUDA call that waits for a host function cannot wait on the scheduler.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "runtime.h"

using namespace agatha;

namespace {

using Clock = std::chrono::steady_clock;

constexpr int64_t kDefaultBudget = (int64_t)1 << 30;
constexpr int32_t kDefaultInflight = 2;
constexpr int32_t kDefaultBatchPairs = 8192;
constexpr int32_t kMaxInflight = 16;

inline int64_t round256(int64_t b) { return (std::max<int64_t>(b, 1) + 255) & ~(int64_t)255; }

// Byte layout of one launch, the same in pinned host staging (inputs) and in
// its device block: inputs first, so one copy uploads them all.
struct Layout {
    int64_t q_packed = 0, t_packed = 0, q_off = 0, t_off = 0, q_len = 0, t_len = 0;
    int64_t in_end = 0, out = 0, order = 0, wide = 0, ovf = 0, total = 0;
};

Layout make_layout(int64_t n, int64_t q_words, int64_t t_words) {
    Layout L;
    int64_t o = 0;
    auto take = [&](int64_t bytes) { const int64_t r = o; o += round256(bytes); return r; };
    const int64_t n1 = std::max<int64_t>(n, 1);
    L.q_packed = take(q_words * 4);
    L.t_packed = take(t_words * 4);
    L.q_off = take(n1 * 8);
    L.t_off = take(n1 * 8);
    L.q_len = take(n1 * 4);
    L.t_len = take(n1 * 4);
    L.in_end = o;
    L.out = take(n1 * (int64_t)sizeof(agatha_result));
    L.order = take(n1 * 4);
    L.wide = take(n1 * 4);
    L.ovf = take(n1 * 4);
    L.total = o;
    return L;
}

// First-fit allocator over the device arena, 256-byte granules, free blocks
// coalesced on release.
class Arena {
public:
    void reset(int64_t size) {
        free_.clear();
        if (size > 0) free_[0] = size;
        size_ = size;
        used_ = 0;
    }
    int64_t alloc(int64_t bytes) {
        bytes = round256(bytes);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < bytes) continue;
            const int64_t off = it->first, rest = it->second - bytes;
            free_.erase(it);
            if (rest > 0) free_[off + bytes] = rest;
            used_ += bytes;
            return off;
        }
        return -1;
    }
    void release(int64_t off, int64_t bytes) {
        bytes = round256(bytes);
        used_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto next = std::next(it);
        if (next != free_.end() && it->first + it->second == next->first) {
            it->second += next->second;
            free_.erase(next);
        }
        if (it != free_.begin()) {
            auto prev = std::prev(it);
            if (prev->first + prev->second == it->first) {
                prev->second += it->second;
                free_.erase(it);
            }
        }
    }
    int64_t size() const { return size_; }
    int64_t used() const { return used_; }

private:
    std::map<int64_t, int64_t> free_;
    int64_t size_ = 0, used_ = 0;
};

struct Pinned {
    void *p = nullptr;
    size_t cap = 0;
    bool ensure(size_t need) {
        if (need <= cap) return true;
        size_t want = std::max(need, cap + cap / 2);
        if (p) cudaFreeHost(p);
        p = nullptr;
        cap = 0;
        if (cudaMallocHost(&p, want) != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
            return false;
        }
        cap = want;
        return true;
    }
    void release() {
        if (p) cudaFreeHost(p);
        p = nullptr;
        cap = 0;
    }
};

bool same_params(const DevParams &x, const DevParams &y) {
    return x.a == y.a && x.b == y.b && x.q == y.q && x.e == y.e && x.q2 == y.q2 && x.e2 == y.e2 &&
           x.w == y.w && x.zdrop == y.zdrop && x.end_bonus == y.end_bonus;
}

struct Request {
    uint64_t id = 0;
    DevParams p;
    int64_t n = 0;
    int32_t max_w = 0;                 // widest effective band of its pairs
    std::vector<uint32_t> q_words, t_words;   // only the words its pairs touch
    std::vector<int64_t> q_off, t_off;        // offsets into those
    std::vector<int32_t> q_len, t_len;
    agatha_result *out = nullptr;
    Clock::time_point t_submit;
    int status = AGATHA_EAGAIN;
};
using ReqPtr = std::shared_ptr<Request>;

struct ServeSlot {
    Slot slot;                          // descriptor, counters, histogram, graphs
    cudaStream_t stream = nullptr;
    Pinned h_in, h_out;
    std::vector<ReqPtr> reqs;
    int64_t n = 0;
    int64_t block_off = -1, block_bytes = 0;
    Layout L;
    bool busy = false;
    bool done = false;                  // set by the completion host function
    bool failed = false;
    Clock::time_point t_launch;
    struct ServeState *owner = nullptr;
};

}  // namespace

struct ServeState {
    agatha_ctx *ctx = nullptr;
    agatha_serve_config cfg{};
    Ledger ledger;                      // slot scratch (descriptor, counters, histogram)
    void *arena_base = nullptr;
    Arena arena;
    std::vector<std::unique_ptr<ServeSlot>> slots;

    std::mutex mu;
    std::condition_variable cv;         // scheduler wake-up: submit, completion, stop
    std::condition_variable done_cv;    // a ticket changed state
    std::deque<ReqPtr> queue;
    std::unordered_map<uint64_t, ReqPtr> tickets;
    uint64_t next_id = 1;
    bool running = false, stop_requested = false, drain = false;
    std::thread thread;

    // statistics (under mu)
    int64_t requests_done = 0, pairs_done = 0, cells_done = 0, launches = 0;
    int64_t peak_bytes = 0;
    int n_busy = 0, max_busy = 0;
    double busy_seconds = 0;
    Clock::time_point busy_since;
    std::vector<double> latencies_ms;
    // device-clock span (ns) of every finished launch's kernels
    std::vector<std::pair<uint64_t, uint64_t>> dev_spans;
};

namespace {

void CUDART_CB on_slot_done(void *arg) {
    ServeSlot *s = (ServeSlot *)arg;
    ServeState *S = s->owner;
    std::lock_guard<std::mutex> g(S->mu);
    s->done = true;
    S->cv.notify_all();
}

// Copy a request's pairs into server memory: only the words each pair
// touches, with offsets rewritten into the copy.
void gather_stream(const uint32_t *packed, const int64_t *off, const int32_t *len, int64_t n,
                   std::vector<uint32_t> &words, std::vector<int64_t> &new_off) {
    words.clear();
    new_off.resize(n);
    for (int64_t i = 0; i < n; ++i) {
        if (len[i] <= 0) {
            new_off[i] = 0;
            continue;
        }
        const int64_t w0 = off[i] / 16, w1 = (off[i] + len[i] + 15) / 16;
        new_off[i] = (int64_t)words.size() * 16 + off[i] % 16;
        words.insert(words.end(), packed + w0, packed + w1);
    }
}

void finish_requests(ServeState *S, ServeSlot *s, int status) {
    const auto now = Clock::now();
    const agatha_result *res = (const agatha_result *)s->h_out.p;
    int64_t at = 0;
    for (const ReqPtr &r : s->reqs) {
        if (status == AGATHA_OK) {
            std::memcpy(r->out, res + at, (size_t)r->n * sizeof(agatha_result));
            for (int64_t i = 0; i < r->n; ++i) S->cells_done += res[at + i].cells;
            S->pairs_done += r->n;
            S->requests_done += 1;
            S->latencies_ms.push_back(std::chrono::duration<double, std::milli>(now - r->t_submit).count());
        }
        at += r->n;
        r->status = status;
        // the ticket outlives the launch; its input copy does not
        std::vector<uint32_t>().swap(r->q_words);
        std::vector<uint32_t>().swap(r->t_words);
        std::vector<int64_t>().swap(r->q_off);
        std::vector<int64_t>().swap(r->t_off);
        std::vector<int32_t>().swap(r->q_len);
        std::vector<int32_t>().swap(r->t_len);
    }
    s->reqs.clear();
    S->done_cv.notify_all();
}

// Retire a finished launch: results to the callers, block back to the arena.
// Called with S->mu held; makes no CUDA call.
void reap(ServeState *S, ServeSlot *s) {
    int status = AGATHA_OK;
    if (s->failed) status = AGATHA_ECUDA;
    else if (s->slot.h_counters[CTR_ERR] != DEV_ERR_NONE) status = AGATHA_EDEVICE;
    if (!s->failed) {
        uint64_t t0 = 0, t1 = 0;
        std::memcpy(&t0, s->slot.h_counters + CTR_T_BEGIN, sizeof(t0));
        std::memcpy(&t1, s->slot.h_counters + CTR_T_END, sizeof(t1));
        if (t0 > 0 && t1 >= t0) S->dev_spans.emplace_back(t0, t1);
    }
    finish_requests(S, s, status);
    S->arena.release(s->block_off, s->block_bytes);
    s->block_off = -1;
    s->busy = false;
    s->done = false;
    s->failed = false;
    if (--S->n_busy == 0)
        S->busy_seconds += std::chrono::duration<double>(Clock::now() - S->busy_since).count();
}

// Stage, upload and launch one merged batch on a slot.  Called WITHOUT the
// server mutex.  Returns a CUDA error; on error nothing stays enqueued that
// would signal completion.
cudaError_t launch_slot(ServeState *S, ServeSlot *s, const DevParams &p, int32_t max_w) {
    NvtxRange range("serve launch");
    agatha_ctx *ctx = S->ctx;
    int64_t n = 0, qw = 0, tw = 0;
    for (const ReqPtr &r : s->reqs) {
        n += r->n;
        qw += (int64_t)r->q_words.size();
        tw += (int64_t)r->t_words.size();
    }
    const Layout &L = s->L;
    if (!s->h_in.ensure((size_t)L.in_end) || !s->h_out.ensure((size_t)std::max<int64_t>(n, 1) * sizeof(agatha_result)))
        return cudaErrorMemoryAllocation;
    unsigned char *h = (unsigned char *)s->h_in.p;
    uint32_t *hq = (uint32_t *)(h + L.q_packed), *ht = (uint32_t *)(h + L.t_packed);
    int64_t *hqo = (int64_t *)(h + L.q_off), *hto = (int64_t *)(h + L.t_off);
    int32_t *hql = (int32_t *)(h + L.q_len), *htl = (int32_t *)(h + L.t_len);
    int64_t at = 0, qb = 0, tb = 0;
    for (const ReqPtr &r : s->reqs) {
        std::copy(r->q_words.begin(), r->q_words.end(), hq + qb);
        std::copy(r->t_words.begin(), r->t_words.end(), ht + tb);
        for (int64_t i = 0; i < r->n; ++i) {
            hqo[at + i] = r->q_off[i] + qb * 16;
            hto[at + i] = r->t_off[i] + tb * 16;
        }
        std::copy(r->q_len.begin(), r->q_len.end(), hql + at);
        std::copy(r->t_len.begin(), r->t_len.end(), htl + at);
        at += r->n;
        qb += (int64_t)r->q_words.size();
        tb += (int64_t)r->t_words.size();
    }
    unsigned char *d = (unsigned char *)S->arena_base + s->block_off;
    cudaStream_t st = s->stream;

    BatchShape shape;
    shape.n = n;
    shape.max_w_all = std::max<int32_t>(max_w, 1);
    shape.max_w_warp = shape.max_w_all;
    LaunchPlan lp;
    const uint32_t lf = S->cfg.launch_flags;
    if (make_plan(ctx, p, shape, lf & AGATHA_REGS_HIGH, &lp) != AGATHA_OK) return cudaErrorInvalidValue;
    if (lf) {
        // the server's own plan: several warps per pair where the band has that
        // kernel, one warp per pair elsewhere
        const int K = (lf & AGATHA_WARPS4) ? 4 : ((lf & AGATHA_WARPS2) ? 2 : 1);
        if (K > 1 && lp.lane16 && lp.warp16k_blocks[K == 4] > 0) lp.groupk = K;
    } else {
        // the plan the context's autotuner chose for this scoring, if any (no measuring here)
        if (tune_apply(ctx, nullptr, p, AGATHA_DEVICE_PTRS, st, &lp) != AGATHA_OK) return cudaErrorInvalidValue;
    }

    DevBatch *desc = s->slot.h_desc;
    desc->q_packed = (const uint32_t *)(d + L.q_packed);
    desc->t_packed = (const uint32_t *)(d + L.t_packed);
    desc->q_words = qw;
    desc->t_words = tw;
    desc->q_off = (const int64_t *)(d + L.q_off);
    desc->t_off = (const int64_t *)(d + L.t_off);
    desc->q_len = (const int32_t *)(d + L.q_len);
    desc->t_len = (const int32_t *)(d + L.t_len);
    desc->out = (agatha_result *)(d + L.out);
    desc->n_pairs = n;
    fill_desc(&s->slot, desc, p, lp, d + L.order, d + L.wide, d + L.ovf);

    cudaError_t e = cudaMemcpyAsync(d, h, (size_t)L.in_end, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->slot.d_desc, desc, sizeof(DevBatch), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = slot_run(ctx, &s->slot, lp, st, nullptr, nullptr);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(s->h_out.p, d + L.out, (size_t)n * sizeof(agatha_result), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(s->slot.h_counters, s->slot.counters.ptr, CTR_COUNT * sizeof(int32_t),
                            cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaLaunchHostFunc(st, on_slot_done, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        cudaStreamSynchronize(st);      // nothing of this batch may still run
        cudaGetLastError();
    }
    return e;
}

// Pick the next merged batch from the queue head.  Called with S->mu held.
// Returns false when nothing can start now; *wake is set when a lingering
// head should be reconsidered at a given time.
bool pick_batch(ServeState *S, ServeSlot *s, DevParams *p, int32_t *max_w, Clock::time_point *wake) {
    if (S->queue.empty()) return false;
    const ReqPtr head = S->queue.front();
    const int64_t cap_pairs = S->cfg.max_batch_pairs;
    std::vector<size_t> pick;
    int64_t n = 0, qw = 0, tw = 0;
    for (size_t i = 0; i < S->queue.size(); ++i) {
        const ReqPtr &r = S->queue[i];
        if (!same_params(r->p, head->p)) continue;
        if (!pick.empty() && n + r->n > cap_pairs) break;
        pick.push_back(i);
        n += r->n;
        qw += (int64_t)r->q_words.size();
        tw += (int64_t)r->t_words.size();
        if (n >= cap_pairs) break;
    }
    // linger for more requests while the batch is short and the head is young
    if (!S->stop_requested && S->cfg.linger_us > 0 && n < cap_pairs) {
        const auto until = head->t_submit + std::chrono::microseconds(S->cfg.linger_us);
        if (Clock::now() < until) {
            *wake = until;
            return false;
        }
    }
    // admission: shrink the batch until its block fits the arena's free space
    while (true) {
        const Layout L = make_layout(n, qw, tw);
        const int64_t off = S->arena.alloc(L.total);
        if (off >= 0) {
            s->L = L;
            s->block_off = off;
            s->block_bytes = L.total;
            break;
        }
        if (pick.size() == 1) return false;      // wait for a running launch to finish
        const ReqPtr &last = S->queue[pick.back()];
        n -= last->n;
        qw -= (int64_t)last->q_words.size();
        tw -= (int64_t)last->t_words.size();
        pick.pop_back();
    }
    *p = head->p;
    *max_w = 0;
    s->reqs.clear();
    for (size_t k = pick.size(); k-- > 0;) {
        const ReqPtr r = S->queue[pick[k]];
        *max_w = std::max(*max_w, r->max_w);
        s->reqs.push_back(r);
        S->queue.erase(S->queue.begin() + (std::ptrdiff_t)pick[k]);
    }
    std::reverse(s->reqs.begin(), s->reqs.end());
    s->n = n;
    return true;
}

void scheduler(ServeState *S) {
    cudaSetDevice(S->ctx->device);
    std::unique_lock<std::mutex> lk(S->mu);
    while (true) {
        for (auto &sp : S->slots)
            if (sp->busy && sp->done) reap(S, sp.get());
        if (S->stop_requested && !S->drain) {
            for (const ReqPtr &r : S->queue) r->status = AGATHA_ECANCELED;
            S->queue.clear();
            S->done_cv.notify_all();
        }
        bool idle = true;
        for (auto &sp : S->slots) idle &= !sp->busy;
        if (S->stop_requested && S->queue.empty() && idle) break;

        Clock::time_point wake = Clock::now() + std::chrono::milliseconds(100);
        bool launched = false;
        for (auto &sp : S->slots) {
            ServeSlot *s = sp.get();
            if (s->busy) continue;
            DevParams p;
            int32_t max_w = 0;
            Clock::time_point linger_wake = wake;
            if (!pick_batch(S, s, &p, &max_w, &linger_wake)) {
                wake = std::min(wake, linger_wake);
                break;
            }
            s->busy = true;
            s->done = false;
            s->failed = false;
            s->t_launch = Clock::now();
            if (S->n_busy++ == 0) S->busy_since = s->t_launch;
            S->max_busy = std::max(S->max_busy, S->n_busy);
            S->launches += 1;
            S->peak_bytes = std::max(S->peak_bytes, S->arena.used());
            lk.unlock();
            const cudaError_t e = launch_slot(S, s, p, max_w);
            lk.lock();
            if (e != cudaSuccess) {
                set_error(S->ctx, AGATHA_ECUDA, "serving launch: %s", cudaGetErrorString(e));
                s->failed = true;
                s->done = true;
            }
            launched = true;
        }
        if (launched) continue;
        S->cv.wait_until(lk, wake);
    }
    S->running = false;
}

void release_resources(ServeState *S) {
    for (auto &sp : S->slots) {
        if (sp->stream) cudaStreamSynchronize(sp->stream);
        slot_release(S->ledger, &sp->slot);
        sp->h_in.release();
        sp->h_out.release();
        if (sp->stream) cudaStreamDestroy(sp->stream);
        sp->stream = nullptr;
    }
    if (S->arena_base) cudaFree(S->arena_base);
    S->arena_base = nullptr;
}

}  // namespace

namespace agatha {

void serve_free(agatha_ctx *ctx) {
    if (!ctx || !ctx->serve) return;
    agatha_serve_stop(ctx, 0);
    delete ctx->serve;
    ctx->serve = nullptr;
}

}  // namespace agatha

extern "C" int agatha_serve_start(agatha_ctx *ctx, const agatha_serve_config *cfg) {
    if (!ctx) return AGATHA_EINVAL;
    agatha_serve_config c{};
    if (cfg) c = *cfg;
    const uint32_t plan_bits = AGATHA_WARPS2 | AGATHA_WARPS4 | AGATHA_REGS_HIGH;
    if (c.mem_budget_bytes < 0 || c.max_inflight < 0 || c.max_inflight > kMaxInflight ||
        c.max_batch_pairs < 0 || c.linger_us < 0 || (c.launch_flags & ~plan_bits) ||
        ((c.launch_flags & AGATHA_WARPS2) && (c.launch_flags & AGATHA_WARPS4)))
        return set_error(ctx, AGATHA_EINVAL, "bad serving config");
    if (c.mem_budget_bytes == 0) c.mem_budget_bytes = kDefaultBudget;
    if (c.max_inflight == 0) c.max_inflight = kDefaultInflight;
    if (c.max_batch_pairs == 0) c.max_batch_pairs = kDefaultBatchPairs;
    if (ctx->serve) {
        if (ctx->serve->running) return set_error(ctx, AGATHA_EAGAIN, "already serving");
        delete ctx->serve;
        ctx->serve = nullptr;
    }
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
    auto *S = new (std::nothrow) ServeState();
    if (!S) return AGATHA_ENOMEM;
    S->ctx = ctx;
    S->cfg = c;
    if ((e = cudaMalloc(&S->arena_base, (size_t)c.mem_budget_bytes)) != cudaSuccess) {
        cudaGetLastError();
        S->arena_base = nullptr;
        delete S;
        return set_error(ctx, AGATHA_ENOMEM, "serving arena of %lld bytes: %s", (long long)c.mem_budget_bytes,
                         cudaGetErrorString(e));
    }
    S->arena.reset(c.mem_budget_bytes);
    for (int i = 0; i < c.max_inflight; ++i) {
        auto sp = std::make_unique<ServeSlot>();
        sp->owner = S;
        int rc = slot_init(ctx, S->ledger, &sp->slot);
        if (rc == AGATHA_OK && cudaStreamCreateWithFlags(&sp->stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            rc = AGATHA_ECUDA;
        }
        sp->slot.last_stream = sp->stream;
        S->slots.push_back(std::move(sp));
        if (rc != AGATHA_OK) {
            release_resources(S);
            delete S;
            return rc;
        }
    }
    S->running = true;
    ctx->serve = S;
    S->thread = std::thread(scheduler, S);
    return AGATHA_OK;
}

extern "C" int agatha_serve_submit(agatha_ctx *ctx, const agatha_batch *batch, const agatha_params *params,
                                   agatha_result *out, uint64_t *ticket) {
    if (!ctx || !batch || !params || !ticket) return AGATHA_EINVAL;
    ServeState *S = ctx->serve;
    if (!S || !S->running || S->stop_requested) return set_error(ctx, AGATHA_EINVAL, "not serving");
    DevParams p;
    if (normalise_params(params, &p)) return set_error(ctx, AGATHA_EINVAL, "bad scoring parameters");
    if (batch->n_pairs > 0 && !out) return set_error(ctx, AGATHA_EINVAL, "null out");
    BatchShape shape;
    int rc = validate_host_batch(ctx, batch, p, &shape);
    if (rc) return rc;
    if (shape.max_w_all > plain_kernel_max_w())
        return set_error(ctx, AGATHA_ENOTSUP, "band of %d cells is wider than supported", shape.max_w_all);
    auto r = std::make_shared<Request>();
    r->p = p;
    r->n = batch->n_pairs;
    r->max_w = shape.max_w_all;
    r->out = out;
    const int64_t n = batch->n_pairs;
    if (n > 0) {
        gather_stream(batch->q_packed, batch->q_off, batch->q_len, n, r->q_words, r->q_off);
        gather_stream(batch->t_packed, batch->t_off, batch->t_len, n, r->t_words, r->t_off);
        r->q_len.assign(batch->q_len, batch->q_len + n);
        r->t_len.assign(batch->t_len, batch->t_len + n);
    }
    const Layout L = make_layout(n, (int64_t)r->q_words.size(), (int64_t)r->t_words.size());
    if (L.total > S->arena.size())
        return set_error(ctx, AGATHA_ENOMEM, "request needs %lld device bytes, budget is %lld",
                         (long long)L.total, (long long)S->arena.size());
    std::lock_guard<std::mutex> g(S->mu);
    if (!S->running || S->stop_requested) return set_error(ctx, AGATHA_EINVAL, "not serving");
    r->id = S->next_id++;
    r->t_submit = Clock::now();
    if (n == 0) {
        r->status = AGATHA_OK;          // nothing to align
        S->requests_done += 1;
        S->latencies_ms.push_back(0.0);
    } else {
        S->queue.push_back(r);
        S->cv.notify_all();
    }
    S->tickets.emplace(r->id, r);
    *ticket = r->id;
    return AGATHA_OK;
}

extern "C" int agatha_serve_poll(agatha_ctx *ctx, uint64_t ticket) {
    if (!ctx || !ctx->serve) return AGATHA_EINVAL;
    ServeState *S = ctx->serve;
    std::lock_guard<std::mutex> g(S->mu);
    auto it = S->tickets.find(ticket);
    if (it == S->tickets.end()) return AGATHA_EINVAL;
    return it->second->status;
}

extern "C" int agatha_serve_wait(agatha_ctx *ctx, uint64_t ticket, int32_t timeout_ms) {
    if (!ctx || !ctx->serve) return AGATHA_EINVAL;
    ServeState *S = ctx->serve;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->tickets.find(ticket);
    if (it == S->tickets.end()) return AGATHA_EINVAL;
    ReqPtr r = it->second;
    auto ready = [&] { return r->status != AGATHA_EAGAIN; };
    if (timeout_ms < 0) S->done_cv.wait(lk, ready);
    else if (!S->done_cv.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready)) return AGATHA_ETIMEDOUT;
    S->tickets.erase(ticket);
    return r->status;
}

extern "C" int agatha_serve_stats_get(agatha_ctx *ctx, agatha_serve_stats *st) {
    if (!ctx || !st || !ctx->serve) return AGATHA_EINVAL;
    ServeState *S = ctx->serve;
    std::lock_guard<std::mutex> g(S->mu);
    std::memset(st, 0, sizeof(*st));
    st->requests_done = S->requests_done;
    st->pairs_done = S->pairs_done;
    st->cells_done = S->cells_done;
    st->launches = S->launches;
    st->bytes_in_flight = S->arena.used();
    st->peak_bytes_in_flight = S->peak_bytes;
    st->busy_seconds = S->busy_seconds;
    if (S->n_busy > 0) st->busy_seconds += std::chrono::duration<double>(Clock::now() - S->busy_since).count();
    if (!S->latencies_ms.empty()) {
        std::vector<double> v = S->latencies_ms;
        auto pct = [&](double f) {
            const size_t k = std::min(v.size() - 1, (size_t)(f * (double)(v.size() - 1) + 0.5));
            std::nth_element(v.begin(), v.begin() + (std::ptrdiff_t)k, v.end());
            return v[k];
        };
        st->p50_latency_ms = pct(0.50);
        st->p99_latency_ms = pct(0.99);
    }
    st->max_launches_in_flight = S->max_busy;
    // sweep over the launches' device spans: how many cover each instant
    std::vector<std::pair<uint64_t, int>> ev;
    ev.reserve(2 * S->dev_spans.size());
    for (const auto &sp : S->dev_spans) {
        ev.emplace_back(sp.first, +1);
        ev.emplace_back(sp.second, -1);
    }
    std::sort(ev.begin(), ev.end());          // at equal times an end sorts before a start
    int64_t cover = 0, most = 0;
    uint64_t overlap_ns = 0, prev = 0;
    for (const auto &x : ev) {
        if (cover >= 2) overlap_ns += x.first - prev;
        cover += x.second;
        most = std::max(most, cover);
        prev = x.first;
    }
    st->max_device_concurrency = most;
    st->overlap_seconds = (double)overlap_ns * 1e-9;
    return AGATHA_OK;
}

extern "C" int agatha_serve_stop(agatha_ctx *ctx, int32_t drain) {
    if (!ctx) return AGATHA_EINVAL;
    ServeState *S = ctx->serve;
    if (!S) return AGATHA_OK;
    {
        std::lock_guard<std::mutex> g(S->mu);
        if (!S->thread.joinable()) return AGATHA_OK;
        S->stop_requested = true;
        S->drain = drain != 0;
        S->cv.notify_all();
    }
    S->thread.join();
    release_resources(S);
    std::lock_guard<std::mutex> g(S->mu);
    S->done_cv.notify_all();
    return AGATHA_OK;
}
