/*
 * Drives the CPU oracle under the compiler's sanitizers (address and
 * undefined behaviour, or thread): random and edge-case pairs through
 * orc_align_pair, orc_traceback_pair (at the extension's end cell and at
 * random band cells) and the threaded batch driver.  Exits 0 when every call
 * returned what the C interface promises; a sanitizer report aborts it.
 * Test infrastructure only (tests/test_oracle_sanitizers.py builds and runs it).
 */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

typedef struct { int32_t a, b, q, e, q2, e2, w, zdrop, end_bonus; } orc_params;
typedef struct {
    int32_t max, qe, te, gscore, mqe, mqe_t, mte, mte_q;
    int64_t cells;
    uint8_t zdropped, reach_end, pad[6];
} orc_result;

void orc_align_pair(const uint8_t *T, int32_t tlen, const uint8_t *Q, int32_t qlen,
                    const orc_params *p, orc_result *out);
void orc_normalise(orc_params *p);
int orc_align_batch(const uint8_t *q_codes, const uint8_t *t_codes, const int64_t *q_off,
                    const int64_t *t_off, const int32_t *q_len, const int32_t *t_len,
                    const int64_t *order, int64_t n, const orc_params *p, orc_result *out,
                    int n_threads);
int64_t orc_traceback_pair(const uint8_t *T, int32_t tlen, const uint8_t *Q, int32_t qlen,
                           const orc_params *p, int32_t end_t, int32_t end_q, uint32_t *ops,
                           int64_t cap, int64_t *score_out);

static uint64_t rng = 0x2403064780ull;
static uint32_t next_u32(void)
{
    rng = rng * 6364136223846793005ull + 1442695040888963407ull;
    return (uint32_t)(rng >> 33);
}

/* a query and a mutated copy as the target */
static int32_t make_pair(uint8_t *T, uint8_t *Q, int32_t max_len, int32_t *qlen)
{
    const int32_t n = (int32_t)(next_u32() % (uint32_t)(max_len + 1));
    int32_t t = 0;
    for (int32_t i = 0; i < n; ++i) Q[i] = (uint8_t)(next_u32() & 3);
    for (int32_t i = 0; i < n && t < 2 * max_len; ++i) {
        const uint32_t u = next_u32() % 100;
        if (u < 5) T[t++] = (uint8_t)((Q[i] + 1) & 3);
        else if (u < 8) continue;
        else if (u < 11) { T[t++] = Q[i]; T[t++] = (uint8_t)(next_u32() & 3); }
        else T[t++] = Q[i];
    }
    *qlen = n;
    return t;
}

static int check_runs(const uint32_t *ops, int64_t n, int32_t et, int32_t eq)
{
    int64_t dt = 0, dq = 0;
    for (int64_t i = 0; i < n; ++i) {
        const uint32_t len = ops[i] >> 4, op = ops[i] & 15;
        if (len == 0 || op > 2) return 0;
        if (op != 1) dt += len;
        if (op != 2) dq += len;
    }
    return dt == (int64_t)et + 1 && dq == (int64_t)eq + 1;
}

int main(void)
{
    const orc_params sets[] = {
        {2, 4, 4, 2, 24, 1, 100, 400, 0}, {1, 4, 6, 2, 26, 1, 20, 200, 5}, {2, 4, 4, 2, 24, 1, 1, 0, 0},
        {2, 4, 4, 2, 24, 1, -1, -1, 0},   {3, 2, 0, 1, 2, 0, 7, 10, 3},    {10, 90, 100, 50, 200, 20, 30, 5000, 0},
    };
    enum { MAXL = 300 };
    uint8_t *T = malloc(2 * MAXL + 2), *Q = malloc(MAXL + 1);
    uint32_t *ops = malloc(sizeof(uint32_t) * (3 * MAXL + 4));
    int bad = 0, calls = 0;
    for (size_t s = 0; s < sizeof(sets) / sizeof(sets[0]); ++s) {
        orc_params p = sets[s];
        orc_normalise(&p);
        for (int k = 0; k < 40; ++k) {
            int32_t qlen;
            const int32_t tlen = make_pair(T, Q, k < 3 ? k : MAXL, &qlen);
            orc_result r;
            orc_align_pair(T, tlen, Q, qlen, &p, &r);
            ++calls;
            int32_t et = r.reach_end ? r.mqe_t : r.te, eq = r.reach_end ? qlen - 1 : r.qe;
            if (tlen == 0 || qlen == 0) et = eq = -1;
            int64_t score = 0;
            const int64_t n = orc_traceback_pair(T, tlen, Q, qlen, &p, et, eq, ops, 3 * MAXL + 4, &score);
            if (n < 0 || (et >= 0 && !check_runs(ops, n, et, eq))) { ++bad; fprintf(stderr, "set %zu pair %d\n", s, k); }
            /* random cells, in band or not: the call must not overrun */
            for (int j = 0; j < 4 && tlen > 0 && qlen > 0; ++j) {
                const int32_t ct = (int32_t)(next_u32() % (uint32_t)tlen), cq = (int32_t)(next_u32() % (uint32_t)qlen);
                const int64_t m = orc_traceback_pair(T, tlen, Q, qlen, &p, ct, cq, ops, 3 * MAXL + 4, &score);
                if (m >= 0 && !check_runs(ops, m, ct, cq)) { ++bad; fprintf(stderr, "cell (%d,%d)\n", ct, cq); }
            }
        }
    }
    /* the threaded batch driver */
    enum { NB = 64 };
    uint8_t *qc = malloc(NB * MAXL + 1), *tc = malloc(NB * 2 * MAXL + 1);
    int64_t q_off[NB], t_off[NB], order[NB];
    int32_t q_len[NB], t_len[NB];
    int64_t qo = 0, to = 0;
    for (int i = 0; i < NB; ++i) {
        int32_t ql;
        const int32_t tl = make_pair(tc + to, qc + qo, MAXL, &ql);
        q_off[i] = qo; t_off[i] = to; q_len[i] = ql; t_len[i] = tl;
        qo += ql; to += tl;
        order[i] = NB - 1 - i;
    }
    orc_result *out = malloc(sizeof(orc_result) * NB);
    if (orc_align_batch(qc, tc, q_off, t_off, q_len, t_len, order, NB, &sets[0], out, 4) != 0) ++bad;
    for (int i = 0; i < NB; ++i) {
        orc_result one;
        orc_params p0 = sets[0];
        orc_normalise(&p0);
        orc_align_pair(tc + t_off[i], t_len[i], qc + q_off[i], q_len[i], &p0, &one);
        if (memcmp(&one, &out[i], sizeof(one)) != 0) { ++bad; fprintf(stderr, "batch pair %d\n", i); }
    }
    free(out); free(qc); free(tc); free(T); free(Q); free(ops);
    printf("%d calls, %d bad\n", calls, bad);
    return bad ? 1 : 0;
}
