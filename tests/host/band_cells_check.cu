// Host-side check of band_cells_through (agatha_dev.cuh), the closed form
// of the band cells the 16-bit kernel reports: every prefix 0..R of every
// table up to 40 x 40 at every band half-width, plus a few long tables,
// against the sum of en(r) - st(r) + 1 taken anti-diagonal by anti-diagonal
// (stopping where the band leaves the table).  Runs on the CPU only.
#include <cstdio>

#include "agatha_dev.cuh"

using agatha::band_cells_through;
using agatha::ceil_div2;
using agatha::effective_w;
using agatha::floor_div2;

static long check(int tl, int ql, int w0, long *n) {
    const int w = effective_w(w0, tl, ql);
    long bad = 0;
    long long acc = 0;
    for (int r = 0; r <= tl + ql - 2; ++r) {
        int st = r - ql + 1 > 0 ? r - ql + 1 : 0;
        if (ceil_div2(r - w) > st) st = ceil_div2(r - w);
        int en = tl - 1 < r ? tl - 1 : r;
        if (floor_div2(r + w) < en) en = floor_div2(r + w);
        if (st > en) break;
        acc += en - st + 1;
        ++*n;
        const long long got = band_cells_through(tl, ql, w, r);
        if (got != acc) {
            if (bad < 5) std::printf("tlen %d qlen %d w %d r %d: %lld, want %lld\n", tl, ql, w, r, got, acc);
            ++bad;
        }
    }
    return bad;
}

int main() {
    long bad = 0, n = 0;
    for (int tl = 1; tl <= 40; ++tl)
        for (int ql = 1; ql <= 40; ++ql)
            for (int w = 1; w <= 45; ++w) bad += check(tl, ql, w, &n);
    const int big[][3] = {{100000, 99000, 750}, {5000, 20000, 500}, {20000, 5000, 500},
                          {1000, 1000, 750}, {600, 620, 750}, {150, 152, 100}, {30000, 30000, -1}};
    for (const auto &c : big) bad += check(c[0], c[1], c[2], &n);
    std::printf("%ld prefixes, %ld wrong\n", n, bad);
    return bad != 0;
}
