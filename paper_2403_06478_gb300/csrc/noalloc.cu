// Allocation-free variant of the batched alignment path.
//
// The batched path needs scratch memory besides its inputs and outputs: the
// batch descriptor the kernels read, the work-queue counters, the bucket
// histogram of the ordering and the two pair lists.  The regular entry point
// keeps them in buffers its context allocates.  Some callers cannot let a
// library call cudaMalloc or cudaFree at all (cudaFree synchronises the whole
// device, and some hosts reserve every byte of device memory up front and hand
// out only pointers into it).  For them this file keeps that scratch in one
// fixed device array and never allocates.
//
// The array lives in device memory of every GPU that loads the library until
// the process exits.  Host code may not use its name as a device address: the
// first call on a device looks the address up with cudaGetSymbolAddress while
// that device is current and remembers it for the device.
#include <mutex>

#include "agatha_dev.cuh"
#include "runtime.h"

namespace {

constexpr size_t kMaxPairs = (size_t)AGATHA_NOALLOC_MAX_PAIRS;
constexpr size_t kOffDesc = 0;
constexpr size_t kOffCounters = 256;
constexpr size_t kOffHist = 512;
constexpr size_t kOffOrder = kOffHist + 256 * sizeof(int64_t);
constexpr size_t kOffWide = kOffOrder + kMaxPairs * sizeof(int32_t);
constexpr size_t kScratchBytes = kOffWide + kMaxPairs * sizeof(int32_t);
static_assert(sizeof(agatha::DevBatch) <= kOffCounters, "descriptor slot too small");
static_assert(agatha::CTR_COUNT * sizeof(int32_t) <= kOffHist - kOffCounters, "counter slot too small");

constexpr int kMaxDevices = 64;

struct DeviceSetup {
    bool ready = false;
    unsigned char *scratch = nullptr;   // device address of the array on this device
    int n_sm = 0;
};

DeviceSetup g_setup[kMaxDevices];
std::mutex g_setup_mu;

}  // namespace

// The scratch array (about 0.5 MiB).  Shared by every call on a device.
static __device__ __align__(256) unsigned char g_agatha_noalloc_scratch[kScratchBytes];

namespace {

int setup_current_device(DeviceSetup **out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return AGATHA_ECUDA;
    }
    std::lock_guard<std::mutex> g(g_setup_mu);
    DeviceSetup &s = g_setup[dev];
    if (!s.ready) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_agatha_noalloc_scratch);
        if (e != cudaSuccess || ptr == nullptr) {
            cudaGetLastError();
            return AGATHA_ECUDA;
        }
        int n_sm = 0;
        if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            agatha::plain_kernel_prepare() != cudaSuccess) {
            cudaGetLastError();
            return AGATHA_ECUDA;
        }
        s.scratch = (unsigned char *)ptr;
        s.n_sm = n_sm;
        s.ready = true;
    }
    *out = &s;
    return AGATHA_OK;
}

cudaError_t launch_warp_any(int C, const agatha::DevBatch *d, int blocks, cudaStream_t s) {
    switch (C) {
        case 4: return agatha::launch_warp_c<4>(d, blocks, s, 1);
        case 8: return agatha::launch_warp_c<8>(d, blocks, s, 1);
        case 16: return agatha::launch_warp_c<16>(d, blocks, s, 1);
        case 24: return agatha::launch_warp_c<24>(d, blocks, s, 1);
        default: return agatha::launch_warp_c<32>(d, blocks, s, 1);
    }
}

}  // namespace

extern "C" int agatha_align_batch_noalloc(const agatha_batch *batch, const agatha_params *params,
                                         agatha_result *out, void *stream) {
    using namespace agatha;
    if (!batch || !params) return AGATHA_EINVAL;
    if (batch->n_pairs < 0 || (size_t)batch->n_pairs > kMaxPairs) return AGATHA_EINVAL;
    if (batch->q_words < 0 || batch->t_words < 0) return AGATHA_EINVAL;
    DevParams p;
    if (normalise_params(params, &p) != AGATHA_OK) return AGATHA_EINVAL;
    if (batch->n_pairs == 0) return AGATHA_OK;
    if (!out || !batch->q_len || !batch->t_len || !batch->q_off || !batch->t_off) return AGATHA_EINVAL;
    // a stream the pairs may read must exist (an empty stream may be null)
    if ((batch->q_words > 0 && !batch->q_packed) || (batch->t_words > 0 && !batch->t_packed))
        return AGATHA_EINVAL;

    DeviceSetup *ds = nullptr;
    int rc = setup_current_device(&ds);
    if (rc != AGATHA_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;

    // kernel plan from the parameters alone (the lengths are on the device)
    const int32_t w_plan = p.w >= 0 ? p.w : 32 * 32 - 1;
    const int C = pick_slots_per_lane(w_plan);
    const int32_t warp_w_max = 32 * C - 1;
    int32_t wide_w = 0;
    if (p.w < 0 || p.w > warp_w_max) {
        wide_w = p.w < 0 ? plain_kernel_max_w() : p.w;
        if (wide_w > plain_kernel_max_w()) return AGATHA_ENOTSUP;
    }
    const int blocks = ds->n_sm * warp_occupancy(C);

    DevBatch desc;
    desc.q_packed = batch->q_packed;
    desc.t_packed = batch->t_packed;
    desc.q_words = batch->q_words;
    desc.t_words = batch->t_words;
    desc.q_off = batch->q_off;
    desc.t_off = batch->t_off;
    desc.q_len = batch->q_len;
    desc.t_len = batch->t_len;
    desc.out = out;
    desc.n_pairs = batch->n_pairs;
    desc.order = (int32_t *)(ds->scratch + kOffOrder);
    desc.counters = (int32_t *)(ds->scratch + kOffCounters);
    desc.wide_order = (int32_t *)(ds->scratch + kOffWide);
    desc.bucket_hist = (int64_t *)(ds->scratch + kOffHist);
    desc.ovf_list = nullptr;          // the 32-bit kernel never hands pairs back
    desc.h0 = nullptr;
    desc.params = p;
    desc.warp_w_max = warp_w_max;
    desc.narrow_w_max = 0;
    const DevBatch *d_desc = (const DevBatch *)(ds->scratch + kOffDesc);

    // the array keeps the previous call's contents: reset what must start at zero
    cudaError_t e = cudaMemcpyAsync((void *)d_desc, &desc, sizeof(desc), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(desc.counters, 0, CTR_COUNT * sizeof(int32_t), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(desc.bucket_hist, 0, 256 * sizeof(int64_t), s);
    if (e == cudaSuccess) e = launch_prep(d_desc, batch->n_pairs, 1, s, ds->n_sm);
    if (e == cudaSuccess) e = launch_warp_any(C, d_desc, blocks, s);
    if (e == cudaSuccess && wide_w > 0) e = launch_plain_kernel(d_desc, (int64_t)ds->n_sm * 2, wide_w, 1, s);
    int32_t ctr[CTR_COUNT] = {0};
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ctr, desc.counters, sizeof(ctr), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return AGATHA_ECUDA;
    }
    return ctr[CTR_ERR] == DEV_ERR_NONE ? AGATHA_OK : AGATHA_EINVAL;
}
