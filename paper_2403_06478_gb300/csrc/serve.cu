// Serving loop (continuous batching).  Filled in by the serving milestone.
#include "runtime.h"

extern "C" int agatha_serve_start(agatha_ctx *ctx, const agatha_serve_config *cfg) {
    (void)ctx; (void)cfg;
    return AGATHA_ENOTSUP;
}
extern "C" int agatha_serve_submit(agatha_ctx *ctx, const agatha_batch *batch, const agatha_params *params,
                                   agatha_result *out, uint64_t *ticket) {
    (void)ctx; (void)batch; (void)params; (void)out; (void)ticket;
    return AGATHA_ENOTSUP;
}
extern "C" int agatha_serve_poll(agatha_ctx *ctx, uint64_t ticket) { (void)ctx; (void)ticket; return AGATHA_ENOTSUP; }
extern "C" int agatha_serve_wait(agatha_ctx *ctx, uint64_t ticket, int32_t timeout_ms) {
    (void)ctx; (void)ticket; (void)timeout_ms;
    return AGATHA_ENOTSUP;
}
extern "C" int agatha_serve_stats_get(agatha_ctx *ctx, agatha_serve_stats *st) { (void)ctx; (void)st; return AGATHA_ENOTSUP; }
extern "C" int agatha_serve_stop(agatha_ctx *ctx, int32_t drain) { (void)ctx; (void)drain; return AGATHA_OK; }
