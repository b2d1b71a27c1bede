/*
 * CPU oracle for guided (banded, Z-drop) extension alignment.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark load this file.  It shares no code, header or
 * constant with the CUDA library: it is a plain, slow restatement of what the
 * method computes, written so a reader can check it against the paper by eye.
 *
 * What is computed (paper Section 2.1):
 *   - Eq. 1-3: affine-gap dynamic programming over the score table of a
 *     reference (target) T and a query Q, H(i,j) = max(E, F, H(i-1,j-1)+S).
 *     Extended to two-piece affine gaps: a gap of length l costs
 *     min(q + l*e, q2 + l*e2), so two extra gap states E2/F2 run with (q2, e2).
 *     The paper's alpha/beta (open/extend) map to q+e and e.
 *   - "Guiding strategy": only the band |t - q| <= w is computed (k-banding).
 *   - Eq. 4-7: exact termination (Z-drop).  For every anti-diagonal c in
 *     order, take its maximum H (lowest t on ties).  If it beats the global
 *     maximum the global maximum moves there; otherwise, if it lies below and
 *     to the right of the global maximum and the drop exceeds
 *     Z + e2*|(i-i')-(j-j')|, the extension stops.
 *   - After the score path, the traceback (CIGAR) of one extension: the
 *     edit operations of a best path to its end cell, under a stated tie
 *     rule (orc_traceback_pair, at the end of this file).
 *   - The BWA-MEM variant of the extension (Section 5.9): local extension
 *     from an initial score with BWA-MEM's row-by-row termination
 *     (orc_align_pair_local).
 * Readings where the paper is silent (boundary, tie-breaks, outputs) follow the
 * minimap2 extension convention and are listed in the design notes.
 *
 * Arithmetic is int64 with a sentinel far below any reachable score, so no
 * wrap-around can occur; only the outputs use -2^30 as "not reached".
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

#define ORC_OUT_NEG_INF (-0x40000000)
#define ORC_MINUS_INF (INT64_MIN / 4)

typedef struct {
    int32_t a, b, q, e, q2, e2, w, zdrop, end_bonus;
} orc_params;

typedef struct {
    int32_t max, qe, te, gscore, mqe, mqe_t, mte, mte_q;
    int64_t cells;
    uint8_t zdropped, reach_end, pad[6];
} orc_result;

static int64_t imax64(int64_t x, int64_t y) { return x > y ? x : y; }
static int64_t imin64(int64_t x, int64_t y) { return x < y ? x : y; }

/* Cost of one gap of length l >= 1 under the two-piece model. */
static int64_t gap_cost(const orc_params *p, int64_t l)
{
    return imin64((int64_t)p->q + l * p->e, (int64_t)p->q2 + l * p->e2);
}

/* A real cell (t, q) of the table that lies inside the band. */
static int in_band(int64_t t, int64_t q, int64_t tlen, int64_t qlen, int64_t w)
{
    if (t < 0 || q < 0 || t >= tlen || q >= qlen) return 0;
    int64_t k = t - q;
    return k <= w && -k <= w;
}

/* One cell's state: H and the four gap states ending at that cell. */
typedef struct { int64_t H, E, F, E2, F2; } cell_state;

/*
 * Align one pair.  T (length tlen) is the reference, Q (length qlen) the
 * query, both as codes 0..3.  Parameters must already be normalised
 * (see orc_normalise).
 */
void orc_align_pair(const uint8_t *T, int32_t tlen, const uint8_t *Q, int32_t qlen,
                    const orc_params *p_in, orc_result *out)
{
    orc_params p = *p_in;
    memset(out, 0, sizeof(*out));
    out->max = 0; out->qe = -1; out->te = -1;
    out->gscore = ORC_OUT_NEG_INF; out->mqe = ORC_OUT_NEG_INF; out->mte = ORC_OUT_NEG_INF;
    out->mqe_t = -1; out->mte_q = -1;
    if (tlen <= 0 || qlen <= 0) return;

    int64_t w = p.w;
    if (w < 0 || w > (int64_t)(tlen > qlen ? tlen : qlen)) w = tlen > qlen ? tlen : qlen;

    /* prev1[t]: cells of anti-diagonal r-1, prev2[t]: r-2, cur[t]: r.  Index t. */
    cell_state *prev2 = (cell_state *)malloc(sizeof(cell_state) * (size_t)tlen);
    cell_state *prev1 = (cell_state *)malloc(sizeof(cell_state) * (size_t)tlen);
    cell_state *cur = (cell_state *)malloc(sizeof(cell_state) * (size_t)tlen);
    if (!prev2 || !prev1 || !cur) { free(prev2); free(prev1); free(cur); out->zdropped = 255; return; }

    int64_t gmax = 0, gmax_t = -1, gmax_q = -1;   /* the origin (-1,-1), score 0 */
    int64_t mqe = ORC_MINUS_INF, mqe_t = -1, mte = ORC_MINUS_INF, mte_q = -1;
    int64_t gscore = ORC_MINUS_INF;
    int64_t cells = 0;
    int zdropped = 0;
    const int64_t last_r = (int64_t)tlen + qlen - 2;

    for (int64_t r = 0; r <= last_r; ++r) {
        /* band cells of anti-diagonal r: t in [st, en] */
        int64_t st = 0, en = tlen - 1;
        if (r - qlen + 1 > st) st = r - qlen + 1;
        int64_t lo = r - w;                              /* t >= ceil((r-w)/2) */
        int64_t lo2 = lo >= 0 ? (lo + 1) / 2 : -((-lo) / 2);
        if (lo2 > st) st = lo2;
        if (r < en) en = r;
        int64_t hi = r + w;                              /* t <= floor((r+w)/2) */
        int64_t hi2 = hi >= 0 ? hi / 2 : -((-hi + 1) / 2);
        if (hi2 < en) en = hi2;
        if (st > en) { zdropped = 1; break; }           /* the band left the table */

        int64_t m = ORC_MINUS_INF, m_t = -1;
        for (int64_t t = st; t <= en; ++t) {
            int64_t q = r - t;
            /* diagonal predecessor H(t-1, q-1) */
            int64_t Hdiag;
            if (t == 0 && q == 0) Hdiag = 0;
            else if (t == 0) Hdiag = -gap_cost(&p, q);          /* H(-1, q-1) */
            else if (q == 0) Hdiag = -gap_cost(&p, t);          /* H(t-1, -1) */
            else Hdiag = prev2[t - 1].H;                        /* same diagonal: in band */
            /* upper predecessor (t-1, q): opens/extends E and E2 */
            int64_t Hup, Eup, E2up;
            if (t == 0) { Hup = -gap_cost(&p, q + 1); Eup = ORC_MINUS_INF; E2up = ORC_MINUS_INF; }
            else if (in_band(t - 1, q, tlen, qlen, w)) { Hup = prev1[t - 1].H; Eup = prev1[t - 1].E; E2up = prev1[t - 1].E2; }
            else { Hup = ORC_MINUS_INF; Eup = ORC_MINUS_INF; E2up = ORC_MINUS_INF; }
            /* left predecessor (t, q-1): opens/extends F and F2 */
            int64_t Hleft, Fleft, F2left;
            if (q == 0) { Hleft = -gap_cost(&p, t + 1); Fleft = ORC_MINUS_INF; F2left = ORC_MINUS_INF; }
            else if (in_band(t, q - 1, tlen, qlen, w)) { Hleft = prev1[t].H; Fleft = prev1[t].F; F2left = prev1[t].F2; }
            else { Hleft = ORC_MINUS_INF; Fleft = ORC_MINUS_INF; F2left = ORC_MINUS_INF; }

            int64_t E = imax64(Hup - p.q - p.e, Eup - p.e);
            int64_t E2 = imax64(Hup - p.q2 - p.e2, E2up - p.e2);
            int64_t F = imax64(Hleft - p.q - p.e, Fleft - p.e);
            int64_t F2 = imax64(Hleft - p.q2 - p.e2, F2left - p.e2);
            int64_t s = (T[t] == Q[q]) ? p.a : -(int64_t)p.b;
            int64_t H = Hdiag + s;
            H = imax64(H, E); H = imax64(H, F); H = imax64(H, E2); H = imax64(H, F2);
            cur[t].H = H; cur[t].E = E; cur[t].F = F; cur[t].E2 = E2; cur[t].F2 = F2;
            if (H > m) { m = H; m_t = t; }                  /* lowest t on ties */
        }
        cells += en - st + 1;

        /* best score reaching the last target base / the last query base */
        if (en == tlen - 1 && r - (tlen - 1) >= 0 && r - (tlen - 1) < qlen) {
            int64_t H = cur[tlen - 1].H;
            if (H > mte) { mte = H; mte_q = r - (tlen - 1); }
        }
        {
            int64_t tq = r - (qlen - 1);
            if (tq >= st && tq <= en) {
                int64_t H = cur[tq].H;
                if (H > mqe) { mqe = H; mqe_t = tq; }
            }
        }
        /* Eq. 4-7: global max update, else the Z-drop test */
        int64_t m_q = r - m_t;
        if (m > gmax) {
            gmax = m; gmax_t = m_t; gmax_q = m_q;
        } else if (m_t >= gmax_t && m_q >= gmax_q && p.zdrop >= 0) {
            int64_t dt = m_t - gmax_t, dq = m_q - gmax_q;
            int64_t l = dt > dq ? dt - dq : dq - dt;
            if (gmax - m > (int64_t)p.zdrop + l * p.e2) { zdropped = 1; break; }
        }
        if (r == last_r && en == tlen - 1) gscore = cur[tlen - 1].H;

        cell_state *tmp = prev2; prev2 = prev1; prev1 = cur; cur = tmp;
    }

    out->max = (int32_t)gmax; out->te = (int32_t)gmax_t; out->qe = (int32_t)gmax_q;
    out->gscore = gscore == ORC_MINUS_INF ? ORC_OUT_NEG_INF : (int32_t)gscore;
    out->mqe = mqe == ORC_MINUS_INF ? ORC_OUT_NEG_INF : (int32_t)mqe;
    out->mte = mte == ORC_MINUS_INF ? ORC_OUT_NEG_INF : (int32_t)mte;
    out->mqe_t = (int32_t)mqe_t; out->mte_q = (int32_t)mte_q;
    out->cells = cells;
    out->zdropped = (uint8_t)zdropped;
    out->reach_end = (uint8_t)(!zdropped && mqe != ORC_MINUS_INF &&
                               mqe + p.end_bonus > gmax);
    free(prev2); free(prev1); free(cur);
}

/*
 * Two-piece parameters that cannot help collapse to one piece: with
 * q2 <= q or e2 >= e the second piece is never the cheaper one for long gaps
 * and the model is the single-piece one, (q2, e2) = (q, e).
 */
void orc_normalise(orc_params *p)
{
    if (p->q2 <= p->q || p->e2 >= p->e) { p->q2 = p->q; p->e2 = p->e; }
}

/* ----------------------------------------------------------------------- */
/*
 * Local extension from an initial score: the BWA-MEM variant of the
 * extension (the paper applies its kernel to BWA-MEM's guided alignment,
 * Section 5.9).  This implementation's reading of BWA-MEM's published
 * extension rules (the BWA-MEM paper, seed extension and clipping), also
 * listed in the design notes:
 *   - the extension continues an alignment whose score so far is h0 > 0: the
 *     origin (-1,-1) holds h0, the virtual row and column h0 - gap(l);
 *   - a path is kept only while its score stays positive: every cell state
 *     (H, E, F, E2, F2) holds the best score of a path ending there whose
 *     score was positive after every step, and 0 when there is none; a
 *     diagonal step out of an empty cell (H = 0) stays empty;
 *   - the table is processed one query position (row q) at a time; the best
 *     cell of a row (lowest t on ties) becomes the best so far when strictly
 *     higher, otherwise the Z-drop test stops the extension when
 *     best - row_best > zdrop + |(q - qe) - (t_row - te)| e2 (always tested,
 *     zdrop < 0: off); a row with no positive cell ends the extension;
 *   - mqe/mqe_t: the best cell of the last query row, mte/mte_q the best
 *     positive cell of the last target base, gscore the cell (tlen-1,
 *     qlen-1), each only from the rows processed; reach_end (the end-to-end
 *     choice of BWA-MEM's clipping rule): no early stop and mqe + end_bonus
 *     beats the best local score;
 *   - zdropped is set by either kind of early stop; cells counts the band
 *     cells of the rows processed, the stopping one included.
 * Nothing beats h0: max = h0, qe = te = -1.
 */
static int64_t pos64(int64_t x) { return x > 0 ? x : 0; }

void orc_align_pair_local(const uint8_t *T, int32_t tlen, const uint8_t *Q, int32_t qlen,
                          const orc_params *p_in, int32_t h0, orc_result *out)
{
    orc_params p = *p_in;
    memset(out, 0, sizeof(*out));
    out->max = h0; out->qe = -1; out->te = -1;
    out->gscore = ORC_OUT_NEG_INF; out->mqe = ORC_OUT_NEG_INF; out->mte = ORC_OUT_NEG_INF;
    out->mqe_t = -1; out->mte_q = -1;
    if (tlen <= 0 || qlen <= 0) return;

    int64_t w = p.w;
    if (w < 0 || w > (int64_t)(tlen > qlen ? tlen : qlen)) w = tlen > qlen ? tlen : qlen;

    /* prev[t]: row q-1, cur[t]: row q */
    cell_state *prev = (cell_state *)malloc(sizeof(cell_state) * (size_t)tlen);
    cell_state *cur = (cell_state *)malloc(sizeof(cell_state) * (size_t)tlen);
    if (!prev || !cur) { free(prev); free(cur); out->zdropped = 255; return; }

    int64_t gmax = h0, gmax_t = -1, gmax_q = -1;
    int64_t mqe = ORC_MINUS_INF, mqe_t = -1, mte = ORC_MINUS_INF, mte_q = -1;
    int64_t gscore = ORC_MINUS_INF;
    int64_t cells = 0;
    int zdropped = 0;

    for (int64_t q = 0; q < qlen; ++q) {
        int64_t lo = q - w > 0 ? q - w : 0;
        int64_t hi = q + w < tlen - 1 ? q + w : tlen - 1;
        if (lo > hi) { zdropped = 1; break; }           /* the band left the table */
        int64_t row_best = 0, row_t = -1;
        for (int64_t t = lo; t <= hi; ++t) {
            /* diagonal predecessor H(t-1, q-1) */
            int64_t Hdiag;
            if (t == 0 && q == 0) Hdiag = h0;
            else if (t == 0) Hdiag = pos64(h0 - gap_cost(&p, q));        /* H(-1, q-1) */
            else if (q == 0) Hdiag = pos64(h0 - gap_cost(&p, t));        /* H(t-1, -1) */
            else Hdiag = in_band(t - 1, q - 1, tlen, qlen, w) ? prev[t - 1].H : 0;
            /* (t-1, q), the previous cell of this row: E and E2 */
            int64_t Hup, Eup, E2up;
            if (t == 0) { Hup = pos64(h0 - gap_cost(&p, q + 1)); Eup = 0; E2up = 0; }
            else if (t - 1 >= lo) { Hup = cur[t - 1].H; Eup = cur[t - 1].E; E2up = cur[t - 1].E2; }
            else { Hup = 0; Eup = 0; E2up = 0; }
            /* (t, q-1), the previous row: F and F2 */
            int64_t Hleft, Fleft, F2left;
            if (q == 0) { Hleft = pos64(h0 - gap_cost(&p, t + 1)); Fleft = 0; F2left = 0; }
            else if (in_band(t, q - 1, tlen, qlen, w)) { Hleft = prev[t].H; Fleft = prev[t].F; F2left = prev[t].F2; }
            else { Hleft = 0; Fleft = 0; F2left = 0; }

            int64_t E = pos64(imax64(Hup - p.q - p.e, Eup - p.e));
            int64_t E2 = pos64(imax64(Hup - p.q2 - p.e2, E2up - p.e2));
            int64_t F = pos64(imax64(Hleft - p.q - p.e, Fleft - p.e));
            int64_t F2 = pos64(imax64(Hleft - p.q2 - p.e2, F2left - p.e2));
            int64_t s = (T[t] == Q[q]) ? p.a : -(int64_t)p.b;
            int64_t H = Hdiag > 0 ? pos64(Hdiag + s) : 0;
            H = imax64(H, E); H = imax64(H, F); H = imax64(H, E2); H = imax64(H, F2);
            cur[t].H = H; cur[t].E = E; cur[t].F = F; cur[t].E2 = E2; cur[t].F2 = F2;
            if (H > row_best) { row_best = H; row_t = t; }  /* positive only, lowest t */
        }
        cells += hi - lo + 1;

        /* the last target base and the last query row */
        if (hi == tlen - 1 && cur[tlen - 1].H > 0 && cur[tlen - 1].H > mte) {
            mte = cur[tlen - 1].H; mte_q = q;
        }
        if (q == qlen - 1 && row_best > 0) { mqe = row_best; mqe_t = row_t; }
        if (row_best == 0) { zdropped = 1; break; }      /* no live cell left */
        if (row_best > gmax) {
            gmax = row_best; gmax_t = row_t; gmax_q = q;
        } else if (p.zdrop >= 0) {
            int64_t dq = q - gmax_q, dt = row_t - gmax_t;
            int64_t l = dq > dt ? dq - dt : dt - dq;
            if (gmax - row_best > (int64_t)p.zdrop + l * p.e2) { zdropped = 1; break; }
        }
        if (q == qlen - 1 && hi == tlen - 1 && cur[tlen - 1].H > 0) gscore = cur[tlen - 1].H;

        cell_state *tmp = prev; prev = cur; cur = tmp;
    }

    out->max = (int32_t)gmax; out->te = (int32_t)gmax_t; out->qe = (int32_t)gmax_q;
    out->gscore = gscore == ORC_MINUS_INF ? ORC_OUT_NEG_INF : (int32_t)gscore;
    out->mqe = mqe == ORC_MINUS_INF ? ORC_OUT_NEG_INF : (int32_t)mqe;
    out->mte = mte == ORC_MINUS_INF ? ORC_OUT_NEG_INF : (int32_t)mte;
    out->mqe_t = (int32_t)mqe_t; out->mte_q = (int32_t)mte_q;
    out->cells = cells;
    out->zdropped = (uint8_t)zdropped;
    out->reach_end = (uint8_t)(!zdropped && mqe != ORC_MINUS_INF && mqe + p.end_bonus > gmax);
    free(prev); free(cur);
}

/* ----------------------------------------------------------------------- */
/* Batch driver: pairs spread over threads, longest first, for timing only. */

typedef struct {
    const uint8_t *q_codes, *t_codes;
    const int64_t *q_off, *t_off;
    const int32_t *q_len, *t_len;
    const int64_t *order;
    int64_t n;
    orc_params p;
    const int32_t *h0;        /* non-null: the local extension with these initial scores */
    orc_result *out;
    int64_t next;
    pthread_mutex_t lock;
} orc_job;

static void *orc_worker(void *arg)
{
    orc_job *job = (orc_job *)arg;
    for (;;) {
        pthread_mutex_lock(&job->lock);
        int64_t k = job->next;
        job->next += 1;
        pthread_mutex_unlock(&job->lock);
        if (k >= job->n) break;
        int64_t i = job->order ? job->order[k] : k;
        if (job->h0)
            orc_align_pair_local(job->t_codes + job->t_off[i], job->t_len[i],
                                 job->q_codes + job->q_off[i], job->q_len[i], &job->p, job->h0[i],
                                 &job->out[i]);
        else
            orc_align_pair(job->t_codes + job->t_off[i], job->t_len[i],
                           job->q_codes + job->q_off[i], job->q_len[i], &job->p, &job->out[i]);
    }
    return NULL;
}

static int orc_run_batch(const uint8_t *q_codes, const uint8_t *t_codes,
                         const int64_t *q_off, const int64_t *t_off,
                         const int32_t *q_len, const int32_t *t_len,
                         const int64_t *order, int64_t n, const orc_params *p,
                         const int32_t *h0, orc_result *out, int n_threads)
{
    orc_job job;
    job.q_codes = q_codes; job.t_codes = t_codes; job.q_off = q_off; job.t_off = t_off;
    job.q_len = q_len; job.t_len = t_len; job.order = order; job.n = n;
    job.p = *p; orc_normalise(&job.p);
    job.h0 = h0;
    job.out = out; job.next = 0;
    pthread_mutex_init(&job.lock, NULL);
    if (n_threads < 1) n_threads = 1;
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)n_threads);
    if (!th) return -1;
    int started = 0;
    for (int i = 0; i < n_threads; ++i)
        if (pthread_create(&th[i], NULL, orc_worker, &job) == 0) ++started;
    if (started == 0) orc_worker(&job);
    for (int i = 0; i < started; ++i) pthread_join(th[i], NULL);
    free(th);
    pthread_mutex_destroy(&job.lock);
    return 0;
}

/* Align n pairs with n_threads threads; order (may be NULL) is the schedule. */
int orc_align_batch(const uint8_t *q_codes, const uint8_t *t_codes,
                    const int64_t *q_off, const int64_t *t_off,
                    const int32_t *q_len, const int32_t *t_len,
                    const int64_t *order, int64_t n, const orc_params *p,
                    orc_result *out, int n_threads)
{
    return orc_run_batch(q_codes, t_codes, q_off, t_off, q_len, t_len, order, n, p, NULL, out,
                         n_threads);
}

/* The same for the local extension, h0[i] the initial score of pair i. */
int orc_align_batch_local(const uint8_t *q_codes, const uint8_t *t_codes,
                          const int64_t *q_off, const int64_t *t_off,
                          const int32_t *q_len, const int32_t *t_len,
                          const int64_t *order, int64_t n, const orc_params *p,
                          const int32_t *h0, orc_result *out, int n_threads)
{
    return orc_run_batch(q_codes, t_codes, q_off, t_off, q_len, t_len, order, n, p, h0, out,
                         n_threads);
}

int orc_result_size(void) { return (int)sizeof(orc_result); }

/* ----------------------------------------------------------------------- */
/*
 * Traceback of one extension: the edit operations of a best-scoring path from
 * the origin (-1,-1) to a chosen end cell (end_t, end_q).  The paper reports
 * scores only; the traceback is the step a mapper runs next on the same table.
 * The rule (this implementation's reading, stated once here and in the
 * design notes):
 *   - H(t,q) was reached from the first of, in this order, the diagonal
 *     H(t-1,q-1)+S, E, F, E2, F2 whose value equals H(t,q) (Eq. 1);
 *   - a gap state E(t,q) (likewise F, E2, F2; Eq. 2-3 and the second piece)
 *     extended the same state of its predecessor only when that was strictly
 *     better than opening from the predecessor's H; on a tie it opened.
 *   - The virtual first row and column are leading gaps: reaching (-1, q)
 *     adds q+1 insertions, reaching (t, -1) adds t+1 deletions.
 * Operations: M (diagonal, match or mismatch) consumes one base of each
 * sequence, I (F states) one query base, D (E states) one target base.  They
 * are returned run-length encoded from the start of the extension, as
 * (length << 4) | op with op M=0, I=1, D=2.
 *
 * The table is filled row by row (t outer, q inner) over t <= end_t,
 * q <= end_q inside the band, from the same recurrences as orc_align_pair;
 * cells beyond the end cell cannot lie on a path to it.
 *
 * Returns the number of runs, or -1 (end cell outside the table or band,
 * allocation failure, or more than `cap` runs).  *score_out receives
 * H(end_t, end_q) (0 for an empty path: end_t < 0 or end_q < 0).
 */
#define ORC_OP_M 0u
#define ORC_OP_I 1u
#define ORC_OP_D 2u

typedef struct { uint32_t *ops; int64_t n, cap; uint32_t op, len; } orc_runs;

/* Prepend (the walk goes backwards) `len` operations `op`. */
static void orc_push(orc_runs *r, uint32_t op, uint32_t len)
{
    if (len == 0) return;
    if (r->len > 0 && r->op == op) { r->len += len; return; }
    if (r->len > 0) {
        if (r->n < r->cap) r->ops[r->n] = (r->len << 4) | r->op;
        r->n++;
    }
    r->op = op; r->len = len;
}

int64_t orc_traceback_pair(const uint8_t *T, int32_t tlen, const uint8_t *Q, int32_t qlen,
                           const orc_params *p_in, int32_t end_t, int32_t end_q,
                           uint32_t *ops, int64_t cap, int64_t *score_out)
{
    orc_params p = *p_in;
    *score_out = 0;
    if (end_t < 0 || end_q < 0) return 0;
    if (end_t >= tlen || end_q >= qlen) return -1;
    int64_t w = p.w;
    if (w < 0 || w > (int64_t)(tlen > qlen ? tlen : qlen)) w = tlen > qlen ? tlen : qlen;
    if (!in_band(end_t, end_q, tlen, qlen, w)) return -1;

    const int64_t nt = (int64_t)end_t + 1, nq = (int64_t)end_q + 1, bw = 2 * w + 1;
    /* per band cell: bits 0-2 the source of H (0 diagonal, 1 E, 2 F, 3 E2,
       4 F2); bits 3-6 whether E, F, E2, F2 of this cell extended */
    uint8_t *dir = (uint8_t *)calloc((size_t)(nt * bw), 1);
    cell_state *row_prev = (cell_state *)malloc(sizeof(cell_state) * (size_t)nq);
    cell_state *row_cur = (cell_state *)malloc(sizeof(cell_state) * (size_t)nq);
    if (!dir || !row_prev || !row_cur) { free(dir); free(row_prev); free(row_cur); return -1; }
    const cell_state outside = {ORC_MINUS_INF, ORC_MINUS_INF, ORC_MINUS_INF, ORC_MINUS_INF, ORC_MINUS_INF};
    for (int64_t q = 0; q < nq; ++q) row_prev[q] = row_cur[q] = outside;

    for (int64_t t = 0; t < nt; ++t) {
        /* row t's band cells are q in [lo, hi].  Entries of the row arrays
           outside the previous row's band hold minus infinity: index hi of
           row_prev was never written (earlier bands end further left) and
           index lo-1 of row_cur, left over from row t-2, is reset here. */
        const int64_t lo = t - w > 0 ? t - w : 0;
        const int64_t hi = t + w < nq - 1 ? t + w : nq - 1;
        if (lo > 0) row_cur[lo - 1] = outside;
        for (int64_t q = lo; q <= hi; ++q) {
            cell_state *c = &row_cur[q];
            /* predecessors, with the virtual row/column of Section 2.1's
               extension boundary and minus infinity outside the band */
            int64_t Hdiag;
            if (t == 0 && q == 0) Hdiag = 0;
            else if (t == 0) Hdiag = -gap_cost(&p, q);
            else if (q == 0) Hdiag = -gap_cost(&p, t);
            else Hdiag = row_prev[q - 1].H;
            int64_t Hup, Eup, E2up, Hleft, Fleft, F2left;
            if (t == 0) { Hup = -gap_cost(&p, q + 1); Eup = E2up = ORC_MINUS_INF; }
            else { Hup = row_prev[q].H; Eup = row_prev[q].E; E2up = row_prev[q].E2; }
            if (q == 0) { Hleft = -gap_cost(&p, t + 1); Fleft = F2left = ORC_MINUS_INF; }
            else { Hleft = row_cur[q - 1].H; Fleft = row_cur[q - 1].F; F2left = row_cur[q - 1].F2; }

            uint8_t d = 0;
            int64_t open = Hup - p.q - p.e, ext = Eup - p.e;
            c->E = ext > open ? ext : open;     if (ext > open) d |= 8;
            open = Hleft - p.q - p.e; ext = Fleft - p.e;
            c->F = ext > open ? ext : open;     if (ext > open) d |= 16;
            open = Hup - p.q2 - p.e2; ext = E2up - p.e2;
            c->E2 = ext > open ? ext : open;    if (ext > open) d |= 32;
            open = Hleft - p.q2 - p.e2; ext = F2left - p.e2;
            c->F2 = ext > open ? ext : open;    if (ext > open) d |= 64;

            const int64_t s = (T[t] == Q[q]) ? p.a : -(int64_t)p.b;
            const int64_t cand[5] = {Hdiag + s, c->E, c->F, c->E2, c->F2};
            int src = 0;
            for (int k = 1; k < 5; ++k)
                if (cand[k] > cand[src]) src = k;      /* first of the equal ones */
            c->H = cand[src];
            dir[t * bw + (q - t + w)] = (uint8_t)(d | src);
        }
        cell_state *tmp = row_prev; row_prev = row_cur; row_cur = tmp;
    }
    *score_out = row_prev[end_q].H;

    /* walk back from the end cell in state H */
    enum { S_H = 0, S_E = 1, S_F = 2, S_E2 = 3, S_F2 = 4, S_DIAG = 5 };
    orc_runs runs = {ops, 0, cap, 0, 0};
    int64_t t = end_t, q = end_q;
    int st = S_H;
    while (t >= 0 && q >= 0) {
        const uint8_t d = dir[t * bw + (q - t + w)];
        if (st == S_H) st = (d & 7) ? (d & 7) : S_DIAG;
        if (st == S_DIAG) {
            orc_push(&runs, ORC_OP_M, 1); --t; --q; st = S_H;
        } else if (st == S_E || st == S_E2) {
            orc_push(&runs, ORC_OP_D, 1);
            const int extended = (st == S_E) ? (d & 8) : (d & 32);
            --t;
            if (!extended) st = S_H;
        } else {
            orc_push(&runs, ORC_OP_I, 1);
            const int extended = (st == S_F) ? (d & 16) : (d & 64);
            --q;
            if (!extended) st = S_H;
        }
    }
    /* leading gap along the virtual row or column */
    if (t < 0 && q >= 0) orc_push(&runs, ORC_OP_I, (uint32_t)(q + 1));
    if (q < 0 && t >= 0) orc_push(&runs, ORC_OP_D, (uint32_t)(t + 1));
    orc_push(&runs, 0xfu, 1);                   /* flush the last run */
    free(dir); free(row_prev); free(row_cur);
    if (runs.n > cap) return -1;
    /* the runs were collected end first: reverse them */
    const int64_t n = runs.n;
    for (int64_t i = 0; i < n / 2; ++i) {
        uint32_t x = ops[i]; ops[i] = ops[n - 1 - i]; ops[n - 1 - i] = x;
    }
    return n;
}
