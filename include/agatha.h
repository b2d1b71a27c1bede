/*
 * agatha.h - C ABI of a GB300 (sm_103a) library for guided extension
 * alignment: banded, two-piece affine, score-only dynamic programming with the
 * exact Z-drop termination rule, batched over many read/reference pairs.
 *
 * The operation (AGAThA, PPoPP'24, arxiv 2403.06478):
 *   - Section 2.1, Eq. 1-3: for a reference (target) T and a query Q the score
 *     table H(t,q) = max(H(t-1,q-1) + S(T[t],Q[q]), E(t,q), F(t,q)) with affine
 *     gap states E (steps in t) and F (steps in q).  Here the gaps are
 *     two-piece affine: a gap of length l costs min(q + l*e, q2 + l*e2), so two
 *     more states E2, F2 run with (q2, e2).  Match scores +a, mismatch -b.
 *   - Section 2.1 "Guiding Strategy": only cells with |t - q| <= w are computed.
 *   - Section 2.1, Eq. 4-7: anti-diagonals r = t + q are visited in order; the
 *     maximum of each (lowest t on ties) either becomes the new global maximum
 *     (strictly greater) or, if it lies at t >= max_t and q >= max_q, ends the
 *     extension when max - H > zdrop + e2 * |(t - max_t) - (q - max_q)|.
 *   - An anti-diagonal with no band cell (|tlen - qlen| > w) also ends the
 *     extension with zdropped = 1.
 *   - Virtual row/column: H(-1,-1) = 0, H(-1,q) = -gap(q+1), H(t,-1) =
 *     -gap(t+1); they are not band-restricted.  Only real cells are banded.
 *
 * Conventions used by every entry point:
 *   - Return value: AGATHA_OK (0) or a negative AGATHA_E* code.  No C++
 *     exception crosses this boundary.  agatha_strerror() names a code and
 *     agatha_last_error() gives the context's last detailed message.
 *   - Ownership: the caller owns every buffer it passes.  The library never
 *     keeps a pointer to caller memory after a call returns (after the stream
 *     work completes, with AGATHA_ASYNC).
 *   - Sequences: 2-bit codes A=0, C=1, G=2, T=3, 16 bases per uint32 word;
 *     base k of a packed stream sits at bits 2*(k%16)..2*(k%16)+1 of word k/16.
 *     N is not representable: agatha_pack_ascii rejects it with AGATHA_EINVAL.
 *   - NEG_INF (-2^30) in a result means "not reached".
 */
#ifndef AGATHA_H
#define AGATHA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define AGATHA_NEG_INF (-0x40000000)

/* Error codes. */
#define AGATHA_OK          0
#define AGATHA_EINVAL     -1   /* bad parameter, offset or length            */
#define AGATHA_ENOMEM     -2   /* device or host allocation failed / budget   */
#define AGATHA_ECUDA      -3   /* a CUDA runtime call failed                  */
#define AGATHA_ETIMEDOUT  -4   /* serve wait ran out of time                  */
#define AGATHA_EAGAIN     -5   /* serve ticket still pending                  */
#define AGATHA_ECANCELED  -6   /* request cancelled by agatha_serve_stop      */
#define AGATHA_EDEVICE    -7   /* the device reported an error status         */
#define AGATHA_ENOTSUP    -8   /* configuration not supported                 */
#define AGATHA_ERANGE     -9   /* caller's output buffer too small            */

/* Flags for agatha_align_batch. */
#define AGATHA_HOST_PTRS   0x00u  /* batch arrays and `out` are host memory  */
#define AGATHA_DEVICE_PTRS 0x01u  /* batch arrays and `out` are device memory*/
#define AGATHA_PLAIN       0x02u  /* plain kernel: one pair per block, input
                                     order, one launch (the comparison path) */
#define AGATHA_ASYNC       0x04u  /* DEVICE_PTRS only: return once enqueued   */
#define AGATHA_NO_SORT     0x08u  /* batched kernel in input order (no LPT)   */
#define AGATHA_FORCE32     0x10u  /* never use 16-bit packed lanes            */
#define AGATHA_NO_GRAPH    0x20u  /* launch directly, no CUDA graph replay    */
#define AGATHA_EDGE_PATH_ONLY 0x40u /* batched kernel: run every anti-diagonal
                                     through the masked edge path (testing)  */
#define AGATHA_REGS_HIGH   0x80u  /* 16-bit kernel at its larger register
                                     budget (one resident block per SM less)  */
#define AGATHA_NO_TUNE     0x100u /* ignore the autotuner for this call       */
#define AGATHA_TB_TWO_PASS 0x200u /* agatha_align_cigar: score path, then a
                                     separate traceback pass (not fused)    */
#define AGATHA_WARPS2      0x400u /* 16-bit kernel with 2 warps sharing each
                                     pair's band (bands of 256..767 slots)   */
#define AGATHA_WARPS4      0x800u /* the same with 4 warps per pair           */
#define AGATHA_HALF_WARP   0x1000u /* 16-bit kernel with two pairs per warp,
                                      16 lanes of 8 slots each (bands up to
                                      127; AGATHA_ENOTSUP for wider ones,
                                      AGATHA_EINVAL with WARPS2/WARPS4)     */
#define AGATHA_ONE_FRAME   0x2000u /* every pair on the batch's slot frame:
                                      without it, on a 24-slot batch, pairs
                                      whose own band fits 640 slots take a
                                      20-slot kernel after the main launch  */

/* Flags for agatha_config.flags. */
#define AGATHA_CFG_TIMING  0x1    /* record CUDA events around the main kernel
                                     of every batch (agatha_last_kernel_ms)   */
#define AGATHA_CFG_AUTOTUNE 0x2   /* pick the kernel variant per length class
                                     by measurement (see agatha_tune_variants) */

typedef struct agatha_ctx agatha_ctx;

/* Scoring and guiding parameters (minimap2 naming).
 *   a >= 0 match score, b >= 0 mismatch penalty, q/e gap open/extend (piece 1),
 *   q2/e2 (piece 2); all penalties >= 0.  If q2 <= q or e2 >= e the model is
 *   single-piece (q2 = q, e2 = e), as the second piece can then never be the
 *   cheaper one for long gaps.  w != 0 is the band half-width (w < 0: no band);
 *   zdrop < 0 disables Z-drop; end_bonus only affects reach_end. */
typedef struct {
    int32_t a, b, q, e, q2, e2, w, zdrop, end_bonus;
} agatha_params;

/* A batch of pairs.  Pair i is Q = q_packed bases [q_off[i], q_off[i]+q_len[i])
 * and T = t_packed bases [t_off[i], t_off[i]+t_len[i]).  q_words/t_words give
 * the size of each packed stream in uint32 words; every sequence must lie
 * inside its stream (EINVAL otherwise).  Lengths >= 0 and < 2^24. */
typedef struct {
    int64_t n_pairs;
    const uint32_t *q_packed;
    const uint32_t *t_packed;
    int64_t q_words;
    int64_t t_words;
    const int64_t *q_off;
    const int64_t *t_off;
    const int32_t *q_len;
    const int32_t *t_len;
} agatha_batch;

/* Per-pair result (48 bytes).
 *   max, te, qe   : global maximum and its cell (target end, query end);
 *                   max = 0, te = qe = -1 when nothing beats the origin.
 *   gscore        : H(tlen-1, qlen-1) if the last anti-diagonal was reached
 *                   and that cell is in band, else NEG_INF.
 *   mqe, mqe_t    : best H on the last query column (q = qlen-1), its t.
 *   mte, mte_q    : best H on the last target row (t = tlen-1), its q.
 *   cells         : band cells of all anti-diagonals processed, up to and
 *                   including the one where the extension stopped.
 *   zdropped      : 1 if Z-drop (or the band leaving the table) stopped it.
 *   reach_end     : !zdropped && mqe + end_bonus > max.
 *   lane16        : 1 if the pair ran on 16-bit packed lanes. */
typedef struct {
    int32_t max, qe, te, gscore, mqe, mqe_t, mte, mte_q;
    int64_t cells;
    uint8_t zdropped, reach_end, lane16, pad[5];
} agatha_result;

/* Context configuration.  device: CUDA ordinal.  mem_budget_bytes: device
 * memory the context may hold for batch buffers (0: no limit).  max_pairs:
 * hint for the first allocation (0: grow on demand).  tune_cache_path: file
 * where the autotuner keeps its choices (NULL: in memory only). */
typedef struct {
    int32_t device;
    int32_t flags;
    int64_t mem_budget_bytes;
    int64_t max_pairs;
    const char *tune_cache_path;
} agatha_config;

/* Create a context on cfg->device (cfg may be NULL: device 0, defaults).
 * Allocates the context's stream and small control buffers.  Errors:
 * EINVAL (ctx NULL, bad device), ECUDA, ENOMEM. */
int agatha_init(agatha_ctx **ctx, const agatha_config *cfg);

/* Release every resource of the context (stops serving first).  NULL is a
 * no-op. */
void agatha_destroy(agatha_ctx *ctx);

/* Align every pair of `batch` with `params` and write out[0..n_pairs).
 *   flags: AGATHA_HOST_PTRS (default) - batch arrays and out in host memory;
 *          the library copies them to the device on `stream` and copies the
 *          results back before returning.
 *          AGATHA_DEVICE_PTRS - all arrays are device pointers on ctx's device;
 *          with AGATHA_ASYNC the call returns after enqueueing on `stream`.
 *          AGATHA_PLAIN selects the plain one-pair-per-block kernel;
 *          otherwise the batched persistent kernel runs (work queue ordered by
 *          predicted band cells, longest first, CUDA graph replay).
 *   stream: cudaStream_t to run on (NULL: the context's own stream).
 * Errors: EINVAL (bad params: w == 0, a negative score or penalty, lengths or
 * offsets outside the streams; checked before any kernel runs for host
 * batches, and by a device check before the alignment for device batches),
 * ENOMEM, ECUDA, EDEVICE. */
int agatha_align_batch(agatha_ctx *ctx, const agatha_batch *batch,
                       const agatha_params *params, agatha_result *out,
                       uint32_t flags, void *stream);

/* The BWA-MEM variant of the extension (paper Section 5.9 applies the method
 * to BWA-MEM's guided alignment; the rules are this library's reading of
 * BWA-MEM's published seed extension and clipping):
 *   - each pair continues an alignment whose score so far is h0[i] (1 ..
 *     2^24): the origin (-1,-1) holds h0, the virtual row and column
 *     h0 - gap(l);
 *   - a path is kept only while its score stays positive after every move;
 *     cells no such path reaches are empty (score 0) and a diagonal step out
 *     of an empty cell stays empty;
 *   - the termination test runs one query position (row q) at a time: the
 *     row's best cell (lowest t on ties) becomes the best so far (max, te,
 *     qe) when strictly higher; otherwise the extension stops when
 *     max - row_best > zdrop + |(q - qe) - (t_row - te)| * e2 (zdrop < 0:
 *     off); a row with no positive cell, or no band cell, ends it too
 *     (zdropped = 1 for either);
 *   - mqe/mqe_t: the best cell of the last query row; mte/mte_q: the best
 *     positive cell of the last target base; gscore: cell (tlen-1, qlen-1)
 *     (each from the rows processed, else AGATHA_NEG_INF / -1);
 *     reach_end = !zdropped && mqe + end_bonus > max (BWA-MEM's clipping
 *     rule: the end-to-end alignment is kept unless the local one beats it by
 *     more than the end bonus); cells: band cells of the rows processed; an
 *     extension nothing improves returns max = h0, qe = te = -1.
 * Same batch layout, ownership and flags as agatha_align_batch (h0 follows
 * AGATHA_DEVICE_PTRS like the other arrays), one warp per pair on int32
 * lanes, pairs ordered longest first (AGATHA_NO_SORT: input order).  The band
 * is required: 1 <= w <= 511.
 * Errors: EINVAL (as agatha_align_batch, and h0 outside [1, 2^24]; for
 * device batches found by the device check), ENOTSUP (w < 0 or w > 511,
 * AGATHA_PLAIN), ENOMEM, ECUDA. */
int agatha_align_batch_local(agatha_ctx *ctx, const agatha_batch *batch,
                             const agatha_params *params, const int32_t *h0,
                             agatha_result *out, uint32_t flags, void *stream);

/* Duration in milliseconds of the main alignment kernel of the last batch
 * run on ctx (the warp kernel of the batched path, the block kernel of the
 * plain path), from CUDA events recorded around its launch on its stream.
 * Waits for the end event.  ENOTSUP unless the context was created with
 * AGATHA_CFG_TIMING; EAGAIN before the first batch. */
int agatha_last_kernel_ms(agatha_ctx *ctx, float *ms);

/* Check parameters on the host without touching the GPU: AGATHA_OK or
 * AGATHA_EINVAL.  `normalised` (may be NULL) receives the parameters the
 * kernels use (two-piece collapsed when the second piece never helps). */
int agatha_check_params(const agatha_params *params, agatha_params *normalised);

/* Pack n bases given as codes 0..3 into 16-base words.  out must hold
 * (n + 15) / 16 words; unused high bits of the last word are zero.
 * EINVAL if a code is > 3 or n < 0. */
int agatha_pack_codes(const uint8_t *codes, int64_t n, uint32_t *out);

/* Same from ASCII A/C/G/T (either case).  EINVAL on any other byte (N too). */
int agatha_pack_ascii(const char *ascii, int64_t n, uint32_t *out);

/* Band cells of the whole table of a tlen x qlen pair with half-width w
 * (w < 0: unbanded): the work estimate used for scheduling. */
int64_t agatha_band_cells(int32_t tlen, int32_t qlen, int32_t w);

/* Autotuner.  With AGATHA_CFG_AUTOTUNE the first host batch for a scoring
 * and band class is used to choose the kernel plan by measurement.  Each of
 * four length classes by predicted band cells (the Section 4.5 model:
 * >= 2^25, >= 2^23, >= 2^21, smaller; up to 4096 pairs each) is timed with
 * each variant (0: 16-bit lanes, 1: 16-bit lanes at the larger register
 * budget, 2: int32 lanes).  The batch (up to 131072 of its pairs) is then
 * timed as one launch of each 16-bit variant (and of int32 lanes if a class
 * preferred them) and, if the classes disagree, with one launch per class.  The fastest plan
 * is kept (anything but one launch of variant 0 must win by 2% on a class's
 * sample and by 1% on the batch), per context
 * and in tune_cache_path (one line per key, read at agatha_init).  Every
 * variant gives bit-identical results.  agatha_tune_variants writes what was
 * tuned for `params` (band half-width w_max: the widest effective band of
 * the batches) into variants[0..4]: the four class variants (all equal when
 * one launch is used), then 1 if one launch per class is used.  AGATHA_OK,
 * AGATHA_EAGAIN if not tuned yet, AGATHA_ENOTSUP if 16-bit lanes do not apply
 * to these parameters (nothing to choose). */
int agatha_tune_variants(agatha_ctx *ctx, const agatha_params *params, int32_t w_max,
                         int32_t *variants);

/* ---------------------------------------------------------------------- */
/* Traceback: the CIGAR of each extension.  The paper reports scores only;  */
/* the traceback is the step a mapper runs next on the same banded table    */
/* (Section 2.1, Eq. 1-3 with the two-piece gap states).                    */
/*                                                                          */
/* For every pair the path runs from the origin to the extension's end      */
/* cell: (mqe_t, qlen-1) when reach_end, else (te, qe), the cell of the     */
/* maximum; its score is mqe or max respectively.  Where several paths      */
/* score the same, the one taken is fixed by this rule: walking back from   */
/* the end, H(t,q) came from the first of diagonal, E, F, E2, F2 that       */
/* equals it, and a gap state extended its predecessor's state only when    */
/* that was strictly better than opening from the predecessor's H.  The     */
/* virtual row/column are leading gaps (reaching (-1,q): q+1 insertions;    */
/* (t,-1): t+1 deletions).                                                  */
/*                                                                          */
/* Runs are uint32 values (length << 4) | op, op AGATHA_CIGAR_M (diagonal:  */
/* match or mismatch, one base of each), AGATHA_CIGAR_I (one query base,    */
/* F states) or AGATHA_CIGAR_D (one target base, E states), from the start  */
/* of the extension, adjacent runs of one op merged.                        */

#define AGATHA_CIGAR_M 0u
#define AGATHA_CIGAR_I 1u
#define AGATHA_CIGAR_D 2u

/* Align a host batch (as agatha_align_batch with AGATHA_HOST_PTRS: same
 * results in `out`, same flags except DEVICE_PTRS/ASYNC, which give ENOTSUP)
 * and trace every extension back.
 *   cigar_off: host array of n_pairs + 1; pair i's runs are
 *              cigar[cigar_off[i] .. cigar_off[i+1]).  Written on success and
 *              on ERANGE.  A pair with an empty sequence or whose maximum is
 *              the origin has no runs.
 *   cigar:     host array of cigar_cap runs.  The runs of pair i number at
 *              most t_len[i] + q_len[i]; on ERANGE (cigar_off[n] > cap)
 *              nothing is written to it.
 * Kernels: when the scoring allows 16-bit packed lanes (as for the score
 * path), one fused kernel aligns each pair and records one direction byte
 * per band slot of every anti-diagonal it computes, then traces the path
 * back.  With AGATHA_TB_TWO_PASS (or AGATHA_PLAIN) the score path runs
 * first and a traceback kernel then recomputes each band up to its end
 * cell.  AGATHA_FORCE32, a scoring beyond the 16-bit lanes, or a pair whose
 * scores leave their range use int32 lanes (two passes).  Every form gives
 * the same results and CIGARs.
 * Device memory: besides the score path's buffers, a direction table of 32*C
 * bytes per anti-diagonal (C the kernel's slots per lane for the batch's
 * widest band: 4, 8, 16 or 24 on 16-bit lanes, up to 32 on int32 lanes),
 * for every anti-diagonal of a pair in the fused form, up to the end cell in
 * the two-pass form, plus about 8 bytes per base of the pair for the runs.
 * Pairs run in waves whose tables fit in the context's budget (else in the
 * device's free memory less min(1/16 of it, 4 GiB)); the context keeps the
 * largest table made until agatha_destroy.
 * Errors: EINVAL (bad batch or parameters), ENOTSUP (a band wider than 1023
 * cells, or device pointers), ENOMEM (one pair's table does not fit), ERANGE,
 * ECUDA. */
int agatha_align_cigar(agatha_ctx *ctx, const agatha_batch *batch,
                       const agatha_params *params, agatha_result *out,
                       int64_t *cigar_off, uint32_t *cigar, int64_t cigar_cap,
                       uint32_t flags, void *stream);

/* Duration in milliseconds of the traceback kernels (all waves, between CUDA
 * events on the call's stream) of the last agatha_align_cigar call on ctx;
 * agatha_last_kernel_ms gives its score kernels.  ENOTSUP without
 * AGATHA_CFG_TIMING, EAGAIN before the first traceback. */
int agatha_last_traceback_ms(agatha_ctx *ctx, float *ms);

/* What the last agatha_align_cigar call on ctx ran: pairs given to a 16-bit
 * traceback kernel, pairs the int32 kernel traced (including those a 16-bit
 * kernel handed back), kernel launches (waves), and how many of the 16-bit
 * pairs went through the fused kernel (score path and traceback in one
 * pass over the band). */
typedef struct {
    int64_t pairs16, pairs32, waves, fused;
} agatha_tb_info;
int agatha_last_traceback_info(agatha_ctx *ctx, agatha_tb_info *info);

/* ---------------------------------------------------------------------- */
/* Serving: continuous batching of alignment requests on one device.       */
/* Not an operation of the paper, which aligns one prepared batch; it feeds */
/* the batched kernels (Section 4) from a stream of small requests.         */
/*                                                                          */
/* A scheduler thread merges queued requests that share their (normalised)  */
/* scoring into one batch of at most max_batch_pairs pairs whenever one of  */
/* max_inflight launch slots is free, and runs it like agatha_align_batch.  */
/* Every launch holds one block of a device arena of mem_budget_bytes made  */
/* at start; a request too large for the whole arena is refused, a batch   */
/* that does not fit now waits, so requests never hold more device memory   */
/* than the budget (plus about 4 KiB of fixed scratch per slot).  Results   */
/* are those agatha_align_batch gives each request on its own.              */

typedef struct {
    int64_t mem_budget_bytes;   /* arena for admitted requests; 0: 1 GiB   */
    int32_t max_inflight;       /* launch slots on the device; 0: 2, <= 16 */
    int32_t max_batch_pairs;    /* pairs merged into one launch; 0: 8192   */
    int32_t linger_us;          /* hold a short head batch this long for   */
                                /* more requests; 0: launch at once        */
    uint32_t launch_flags;      /* plan of every launch: 0 = the context's */
                                /* autotuned plan; AGATHA_WARPS2 or        */
                                /* AGATHA_WARPS4 = 2 or 4 warps per pair   */
                                /* (shorter latency for long pairs; a     */
                                /* launch whose band has no such kernel    */
                                /* runs one warp per pair), with or       */
                                /* without AGATHA_REGS_HIGH; any other bit */
                                /* is EINVAL                               */
} agatha_serve_config;

typedef struct {
    int64_t requests_done, pairs_done, cells_done;
    int64_t launches;
    int64_t bytes_in_flight, peak_bytes_in_flight;
    double busy_seconds;        /* wall time with work on the device        */
    double p50_latency_ms, p99_latency_ms;
    /* Overlap of launches.  max_launches_in_flight: the most launches that
     * were enqueued and not yet retired at one time (host view).  From the
     * device's global timer, per finished launch, the span from the first
     * block of its first kernel to the last warp of its alignment kernels:
     * max_device_concurrency is the most spans covering one instant and
     * overlap_seconds the device time covered by two or more spans. */
    int64_t max_launches_in_flight, max_device_concurrency;
    double overlap_seconds;
} agatha_serve_stats;

/* Start the scheduler thread of ctx (one server per context).  EINVAL on a
 * bad config, EAGAIN if already serving, ENOMEM if the arena cannot be
 * allocated.  Independent of agatha_align_batch on the same context. */
int agatha_serve_start(agatha_ctx *ctx, const agatha_serve_config *cfg);

/* Submit a request (host pointers; copied before return).  `out` (host,
 * n_pairs results) must stay valid until the ticket completes.  ENOMEM if the
 * request alone exceeds the memory budget; EINVAL on a bad batch or when the
 * server is not running; ENOTSUP for a band wider than supported. */
int agatha_serve_submit(agatha_ctx *ctx, const agatha_batch *batch,
                        const agatha_params *params, agatha_result *out,
                        uint64_t *ticket);

/* AGATHA_OK if the ticket is complete (results written), AGATHA_EAGAIN if
 * pending, AGATHA_ECANCELED if cancelled, EINVAL for an unknown ticket. */
int agatha_serve_poll(agatha_ctx *ctx, uint64_t ticket);

/* Wait up to timeout_ms (< 0: forever).  Returns the ticket's final status
 * (OK, ECANCELED, EDEVICE, ECUDA), ETIMEDOUT, or EINVAL for an unknown
 * ticket.  A ticket is forgotten once a wait returned its final status. */
int agatha_serve_wait(agatha_ctx *ctx, uint64_t ticket, int32_t timeout_ms);

/* Snapshot of the server's counters. */
int agatha_serve_stats_get(agatha_ctx *ctx, agatha_serve_stats *stats);

/* Stop the scheduler.  drain != 0: finish every admitted and queued request;
 * drain == 0: finish requests already on the device, cancel queued ones.
 * Returns after the device work ended and the arena was freed; tickets stay
 * readable until agatha_destroy or the next agatha_serve_start. */
int agatha_serve_stop(agatha_ctx *ctx, int32_t drain);

/* ---------------------------------------------------------------------- */
/* Allocation-free alignment.  The paper has no counterpart: this entry point
 * exists for callers that cannot let a library call cudaMalloc or cudaFree -
 * for example a host application that reserves all device memory up front and
 * only hands out pointers into it, or one that must not pay the device-wide
 * synchronisation cudaFree implies in the middle of its work.
 *
 * It runs the same batched path as agatha_align_batch (validation, ordering,
 * warp kernel) on the current device and allocates nothing.  The scratch
 * memory the path needs (descriptor, queue counters, ordering lists) sits in a
 * fixed device array of the library, about 0.5 MiB, sized for at most
 * AGATHA_NOALLOC_MAX_PAIRS pairs; every GPU that loads the library keeps that
 * array until the process exits.
 *   batch: every array is device memory of the current device.
 *   out:   device memory for batch->n_pairs results.
 *   stream: cudaStream_t (NULL: the legacy default stream).  The call waits
 *          for its work on that stream before returning.
 * The first call on a device looks up the array's device address and
 * prepares the kernels; make that first call before any stream capture.
 * Every call copies its batch descriptor from host memory into the array and
 * then waits for the stream, so it returns only after the results are written.
 * All calls share the one array and it keeps the last call's contents (the
 * call clears what must start at zero): calls whose work overlaps on the GPU
 * (other streams or host threads) race, so the caller must serialise them.
 * Errors: EINVAL (n_pairs > AGATHA_NOALLOC_MAX_PAIRS, bad parameters, a null
 * array the pairs need - q_packed with q_words > 0, t_packed with t_words > 0,
 * lengths, offsets or out -, a pair outside its stream: that pair's record is
 * written empty and the others are aligned), ENOTSUP (band wider than
 * supported), ECUDA. */
#define AGATHA_NOALLOC_MAX_PAIRS 65536
int agatha_align_batch_noalloc(const agatha_batch *batch, const agatha_params *params,
                               agatha_result *out, void *stream);

/* ---------------------------------------------------------------------- */

const char *agatha_strerror(int code);
const char *agatha_last_error(agatha_ctx *ctx);
/* Library version (major*10000 + minor*100 + patch). */
int32_t agatha_version(void);

#ifdef __cplusplus
}
#endif
#endif /* AGATHA_H */
