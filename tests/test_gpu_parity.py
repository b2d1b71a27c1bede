"""GPU parity: every kernel path must reproduce the CPU oracle bit for bit.

Integer outputs (scores, coordinates, cell counts, flags) are compared for
exact equality: the method computes exact integers, so the tolerance is 0.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2403_06478_gb300 import agatha as A
from paper_2403_06478_gb300 import build as B
from paper_2403_06478_gb300 import workload as W

pytestmark = pytest.mark.gpu

FIELDS = O.COMPARE_FIELDS

PATHS = {
    "batched": 0,
    "plain": A.AGATHA_PLAIN,
    "edge_only": A.AGATHA_EDGE_PATH_ONLY,
    "no_sort": A.AGATHA_NO_SORT,
    "no_graph": A.AGATHA_NO_GRAPH,
    "force32": A.AGATHA_FORCE32,
    "force32_edge": A.AGATHA_FORCE32 | A.AGATHA_EDGE_PATH_ONLY,
    "regs_high": A.AGATHA_REGS_HIGH,
    "regs_high_edge": A.AGATHA_REGS_HIGH | A.AGATHA_EDGE_PATH_ONLY,
    "half_warp": A.AGATHA_HALF_WARP,            # two pairs per warp (bands up to 127)
    "one_frame": A.AGATHA_ONE_FRAME,            # no narrower frame for short pairs
}


@pytest.fixture(scope="module")
def ctx():
    B.build()
    c = A.Context(0)
    yield c
    c.close()


def _assert_same(got, ref, batch, label):
    bad = A.results_equal(got, ref, FIELDS)
    if bad.size:
        i = int(bad[0])
        diff = {f: (int(got[i][f]), int(ref[i][f])) for f in FIELDS if got[i][f] != ref[i][f]}
        raise AssertionError(f"{label}: {bad.size} of {got.shape[0]} pairs differ; first pair {i} "
                             f"(tlen={int(batch.t_len[i])}, qlen={int(batch.q_len[i])}) "
                             f"got/expected: {diff}")


@pytest.mark.parametrize("path", sorted(PATHS))
def test_small_config_all_paths(ctx, path):
    batch = W.make_config("small")
    ref = O.align_batch(batch)
    got = A.agatha_align_batch(ctx, batch, flags=PATHS[path])
    _assert_same(got, ref, batch, f"small/{path}")
    assert int(ref["cells"].sum()) > 0


ADVERSARIAL_SCORINGS = [
    W.Scoring(2, 4, 4, 2, 24, 1, 100, 400, 0),
    W.Scoring(2, 4, 4, 2, 24, 1, 7, 30, 0),        # narrow band, frequent Z-drop
    W.Scoring(1, 4, 6, 2, 26, 1, 33, 20, 5),       # HiFi scoring, end bonus
    W.Scoring(2, 4, 4, 2, 24, 1, -1, -1, 0),       # unbanded, no Z-drop
    W.Scoring(2, 3, 2, 3, 5, 1, 16, 0, 0),         # zdrop 0: stops at the first drop
    W.Scoring(3, 2, 0, 1, 2, 0, 31, 10, 0),        # free gap extension on piece 2
    W.Scoring(2, 4, 4, 2, 4, 2, 127, 200, 0),      # single piece, w = 32*4-1
    W.Scoring(2, 4, 4, 2, 24, 1, 128, 200, 0),     # w = 32*4: next slot class
    W.Scoring(2, 4, 4, 2, 24, 1, 511, 400, 0),     # C = 16 exactly full
    W.Scoring(2, 4, 4, 2, 24, 1, 750, 400, 0),     # C = 24
    W.Scoring(2, 4, 4, 2, 24, 1, 1000, 400, 0),    # C = 32
]


def _adversarial_batch(rng, scoring):
    qs, ts = [], []
    w = scoring.w if scoring.w > 0 else 64
    lens = [0, 1, 2, 3, 5, 16, 17, 31, 32, 33, 63, 64, 65, 100, 200, 333, 600, 1200]
    for L in lens:
        q = rng.integers(0, 4, L).astype(np.uint8)
        qs.append(q); ts.append(q.copy())                                   # identical
        qs.append(q); ts.append(((q + 1) % 4).astype(np.uint8))             # all mismatch
        qs.append(np.zeros(L, np.uint8)); ts.append(np.zeros(L + 3, np.uint8))   # homopolymer
        t = rng.integers(0, 4, max(0, L + int(rng.integers(-w - 2, w + 3)))).astype(np.uint8)
        qs.append(q); ts.append(t)                                          # length gap near w
        mq = q.copy()
        if L:
            mq[rng.integers(0, L, max(1, L // 20))] = rng.integers(0, 4, max(1, L // 20))
        qs.append(mq); ts.append(np.concatenate([q[: L // 2], rng.integers(0, 4, L - L // 2)]).astype(np.uint8))
    b2 = W.random_pairs(rng, 60, 400, scoring, min_len=0, related=0.7)
    for i in range(b2.n_pairs):
        qs.append(b2.query(i)); ts.append(b2.target(i))
    return W.from_pairs(qs, ts, scoring, name="adversarial")


@pytest.mark.parametrize("si", range(len(ADVERSARIAL_SCORINGS)))
def test_adversarial_pairs(ctx, si):
    scoring = ADVERSARIAL_SCORINGS[si]
    batch = _adversarial_batch(np.random.default_rng(100 + si), scoring)
    ref = O.align_batch(batch)
    paths = ["batched", "plain", "edge_only", "force32", "regs_high", "one_frame"]
    if 0 < scoring.w <= 127:                    # the band two pairs per warp take
        paths.append("half_warp")
    for path in paths:
        got = A.agatha_align_batch(ctx, batch, flags=PATHS[path])
        _assert_same(got, ref, batch, f"adversarial[{si}]/{path}")


@pytest.mark.parametrize("name", ["small", "ont", "hifi", "skewed"])   # 8, 16, 16, 24 slots per lane
def test_16bit_lanes_used_and_exact(ctx, name):
    batch = W.make_config(name, n_pairs=300)
    got = A.agatha_align_batch(ctx, batch)
    assert got["lane16"].mean() > 0.99          # these bands and scorings fit 16-bit lanes
    ref = A.agatha_align_batch(ctx, batch, flags=A.AGATHA_FORCE32)
    assert (ref["lane16"] == 0).all()
    assert A.results_equal(got, ref).size == 0


@pytest.mark.parametrize("scoring", [
    W.Scoring(1, 20, 4, 30, 4, 30, 511, -1, 0),     # steep single-piece gaps, no Z-drop
    W.Scoring(2, 30, 33, 31, 33, 31, 767, -1, 0),   # the largest step the 16-bit lanes take
    W.Scoring(1, 9, 16, 3, 41, 1, 300, -1, 0),      # assembly-like two-piece
    W.Scoring(1, 19, 39, 3, 81, 1, 200, -1, 0),     # step bound 82 (> 64)
    W.Scoring(10, 90, 100, 50, 200, 20, 127, 5000, 0),   # step bound 220, 4 slots per lane
])
def test_16bit_lanes_with_steep_penalties(ctx, scoring):
    # far past the table's end (the band's last w anti-diagonals) and before
    # its start, cells off the table fall by the full gap cost per base; they
    # must stay clear of the cells of the table sharing their registers
    rng = np.random.default_rng(23)
    qs, ts = [], []
    for L in (300, 700, 1200, 2500):
        for k in range(6):
            x = rng.integers(0, 4, L).astype(np.uint8)
            y = x.copy()
            y[rng.integers(0, L, L // 30)] = rng.integers(0, 4, L // 30)
            cut = int(rng.integers(0, min(scoring.w, L // 2)))
            qs.append(x)
            ts.append(y[: L - cut] if k % 2 else np.concatenate([y, rng.integers(0, 4, cut)]).astype(np.uint8))
    batch = W.from_pairs(qs, ts, scoring)
    ref = O.align_batch(batch)
    for path in ("batched", "edge_only", "regs_high"):
        got = A.agatha_align_batch(ctx, batch, flags=PATHS[path])
        _assert_same(got, ref, batch, f"steep/{path}")
    got = A.agatha_align_batch(ctx, batch)
    assert got["lane16"].mean() > 0.5


def test_16bit_overflow_hands_pairs_to_int32(ctx):
    # identical sequences with a = b = 64 and a 1 + 63 l gap cost: on every
    # anti-diagonal the band edge sits about 32*511 + gap(511) = 48.5k below the
    # maximum, more spread than the 16-bit lanes keep at this step size (~44.7k),
    # so these pairs must come back exact from the int32 recomputation
    rng = np.random.default_rng(17)
    scoring = W.Scoring(64, 64, 1, 63, 1, 63, 511, -1, 0)
    qs, ts = [], []
    for k in range(6):
        x = rng.integers(0, 4, 2500 + 100 * k).astype(np.uint8)
        qs.append(x)
        ts.append(x.copy())
    for k in range(6):                           # short pairs stay within 16 bits
        x = rng.integers(0, 4, 250).astype(np.uint8)
        qs.append(x)
        ts.append(x.copy())
    batch = W.from_pairs(qs, ts, scoring)
    got = A.agatha_align_batch(ctx, batch)
    _assert_same(got, O.align_batch(batch), batch, "overflow")
    assert (got["lane16"][:6] == 0).all()         # recomputed on int32 lanes
    assert (got["lane16"][6:] == 1).all()


def test_empty_batch_and_empty_pairs(ctx):
    b = W.from_pairs([], [], W.SMALL_SCORING)
    assert A.agatha_align_batch(ctx, b).shape[0] == 0
    b = W.from_pairs(["", "A", ""], ["", "", "ACGT"], W.SMALL_SCORING)
    got = A.agatha_align_batch(ctx, b)
    for r in got:
        assert (r["max"], r["qe"], r["te"], r["gscore"], r["cells"], r["zdropped"]) == (
            0, -1, -1, A.NEG_INF, 0, 0)


def test_results_independent_of_batch_composition(ctx):
    full = W.make_config("ont", n_pairs=400)
    ref = A.agatha_align_batch(ctx, full)
    idx = np.random.default_rng(5).permutation(400)[:150]
    sub = A.agatha_align_batch(ctx, full.subset(idx))
    bad = A.results_equal(sub, ref[idx])
    assert bad.size == 0


def _sampled_parity(ctx, name, n_sample, seed):
    batch = W.make_config(name)                    # full size, bench launch configuration
    got = A.agatha_align_batch(ctx, batch)
    rng = np.random.default_rng(seed)
    # the longest pairs and a uniform sample: the oracle computes them one by one
    longest = np.argsort(-(batch.q_len.astype(np.int64) + batch.t_len))[:8]
    idx = np.unique(np.concatenate([longest, rng.choice(batch.n_pairs, n_sample, replace=False)]))
    ref = O.align_batch(batch, idx=idx)
    _assert_same(got[idx], ref, batch.subset(idx), f"{name}/sampled")
    # properties that hold for every pair
    assert (got["cells"] > 0).all() == (batch.q_len > 0).all()
    assert set(np.unique(got["zdropped"])) <= {0, 1}
    assert (got["max"] >= 0).all()
    return batch, got


def test_ont_full_size_sampled(ctx):
    batch, got = _sampled_parity(ctx, "ont", 250, 1)
    # the plain kernel agrees with the batched one on every pair
    plain = A.agatha_align_batch(ctx, batch, flags=A.AGATHA_PLAIN)
    assert A.results_equal(plain, got).size == 0


def test_short_reads_with_bwa_parameters(ctx):
    # 150 bp extensions with BWA-MEM's default scoring (w=100, Z-drop 100,
    # end bonus 5): every pair of a 3,000-pair slice, batched and plain
    batch = W.make_config("short", n_pairs=3000)
    ref = O.align_batch(batch)
    for path in ("batched", "plain", "force32", "half_warp"):
        _assert_same(A.agatha_align_batch(ctx, batch, flags=PATHS[path]), ref, batch, f"short/{path}")
    assert ref["reach_end"].sum() > 0          # the end bonus takes effect


def test_hifi_full_size_sampled(ctx):
    _sampled_parity(ctx, "hifi", 120, 2)


def test_skewed_full_size_sampled(ctx):
    _sampled_parity(ctx, "skewed", 400, 3)


def test_host_batch_errors_before_launch(ctx):
    batch = W.make_config("small", n_pairs=4)
    pb = A.pack_batch(batch)
    pb.q_off = pb.q_off.copy()
    pb.q_off[2] = int(pb.q_packed.shape[0]) * 16      # outside the stream
    with pytest.raises(A.AgathaError) as e:
        ctx.align_host(pb, batch.scoring)
    assert e.value.code == A.AGATHA_EINVAL
    with pytest.raises(A.AgathaError) as e:
        ctx.align_host(A.pack_batch(batch), W.Scoring(w=0))
    assert e.value.code == A.AGATHA_EINVAL


def test_device_pointers_and_device_side_check(ctx):
    torch = pytest.importorskip("torch")
    batch = W.make_config("small", n_pairs=64)
    pb = A.pack_batch(batch)
    dev = {k: torch.from_numpy(getattr(pb, k)).cuda() for k in
           ("q_packed", "t_packed", "q_off", "t_off", "q_len", "t_len")}
    out = torch.zeros(pb.n_pairs * 48, dtype=torch.uint8, device="cuda")
    for flags in (0, A.AGATHA_PLAIN):
        ctx.align_device(dev["q_packed"], dev["t_packed"], dev["q_off"], dev["t_off"], dev["q_len"],
                         dev["t_len"], out, batch.scoring, flags=flags)
        got = out.cpu().numpy().view(A.RESULT_DTYPE)
        _assert_same(got, O.align_batch(batch), batch, f"device/{flags}")
    bad_off = dev["t_off"].clone()
    bad_off[5] = int(pb.t_packed.shape[0]) * 16 + 100
    with pytest.raises(A.AgathaError) as e:
        ctx.align_device(dev["q_packed"], dev["t_packed"], dev["q_off"], bad_off, dev["q_len"],
                         dev["t_len"], out, batch.scoring)
    assert e.value.code == A.AGATHA_EINVAL


@pytest.mark.parametrize("f", [0.01, 0.1, 0.5])
def test_long_ratio_mix_matches_oracle(ctx, f):
    # the paper's load-balancing mix (Section 5.6): a fraction f of 4096 bp
    # pairs among 128 bp ones; every pair against the oracle on the
    # longest-first queue, the same queue in input order and the plain kernel
    batch = W.make_long_ratio(f, n_pairs=2000)
    assert int((batch.q_len == 4096).sum()) == round(f * 2000)
    ref = O.align_batch(batch)
    for path in ("batched", "no_sort", "plain"):
        got = A.agatha_align_batch(ctx, batch, flags=PATHS[path])
        _assert_same(got, ref, batch, f"long_ratio {f}/{path}")


# 2 and 4 warps sharing each pair's band (bands of 256..767 slots)
WARPS_SCORINGS = [
    W.Scoring(2, 4, 4, 2, 24, 1, 300, 400, 0),
    W.Scoring(2, 4, 4, 2, 24, 1, 511, 400, 0),      # 16-slot frame exactly full
    W.Scoring(1, 4, 6, 2, 26, 1, 600, 200, 5),      # HiFi scoring, end bonus, 24-slot frame
    W.Scoring(2, 4, 4, 2, 24, 1, 767, 30, 0),       # 24-slot frame full, frequent Z-drop
    W.Scoring(2, 3, 2, 3, 5, 1, 256, 0, 0),         # zdrop 0
    W.Scoring(1, 20, 4, 30, 4, 30, 400, -1, 0),     # steep single-piece gaps, no Z-drop
]


@pytest.mark.parametrize("si", range(len(WARPS_SCORINGS)))
@pytest.mark.parametrize("warps", ["warps2", "warps4"])
def test_warps_per_pair_match_oracle(ctx, si, warps):
    scoring = WARPS_SCORINGS[si]
    flags = A.AGATHA_WARPS2 if warps == "warps2" else A.AGATHA_WARPS4
    batch = _adversarial_batch(np.random.default_rng(300 + si), scoring)
    ref = O.align_batch(batch)
    _assert_same(A.agatha_align_batch(ctx, batch, flags=flags), ref, batch, f"{warps}[{si}]")
    _assert_same(A.agatha_align_batch(ctx, batch, flags=flags | A.AGATHA_EDGE_PATH_ONLY), ref, batch,
                 f"{warps}[{si}]/edge")


@pytest.mark.parametrize("name", ["ont", "skewed"])
@pytest.mark.parametrize("warps", ["warps2", "warps4"])
def test_warps_per_pair_on_workloads(ctx, name, warps):
    # the longest pairs of the workload (the ones this variant is for) and a
    # sample of the rest, against the oracle
    flags = A.AGATHA_WARPS2 if warps == "warps2" else A.AGATHA_WARPS4
    batch = W.make_config(name, n_pairs=4000)
    L = np.maximum(batch.q_len, batch.t_len).astype(np.int64)
    idx = np.unique(np.concatenate([np.argsort(-L)[:24],
                                    np.random.default_rng(41).choice(batch.n_pairs, 200, replace=False)]))
    sub = batch.subset(idx)
    got = A.agatha_align_batch(ctx, sub, flags=flags)
    assert got["lane16"].mean() > 0.99
    _assert_same(got, O.align_batch(sub), sub, f"{name}/{warps}")
    # and the whole 4,000 pairs equal the one-warp kernel's results
    assert A.results_equal(A.agatha_align_batch(ctx, batch, flags=flags),
                           A.agatha_align_batch(ctx, batch)).size == 0


def test_warps_per_pair_hand_back_overflow(ctx):
    # the 16-bit overflow case with 2 and 4 warps: every warp of the group
    # must agree to hand the pair to the int32 kernel
    rng = np.random.default_rng(17)
    scoring = W.Scoring(64, 64, 1, 63, 1, 63, 511, -1, 0)
    xs = [rng.integers(0, 4, 2500 + 100 * k).astype(np.uint8) for k in range(4)]
    ys = [rng.integers(0, 4, 250).astype(np.uint8) for _ in range(4)]
    batch = W.from_pairs(xs + ys, [x.copy() for x in xs + ys], scoring)
    ref = O.align_batch(batch)
    for flags in (A.AGATHA_WARPS2, A.AGATHA_WARPS4):
        got = A.agatha_align_batch(ctx, batch, flags=flags)
        _assert_same(got, ref, batch, f"overflow/{flags}")
        assert (got["lane16"][:4] == 0).all() and (got["lane16"][4:] == 1).all()


def test_warps_per_pair_rejects_other_bands(ctx):
    batch = W.make_config("small", n_pairs=8)          # w = 100: 4-slot frame
    with pytest.raises(A.AgathaError) as e:
        A.agatha_align_batch(ctx, batch, flags=A.AGATHA_WARPS2)
    assert e.value.code == A.AGATHA_ENOTSUP


def test_half_warp_rejects_wider_bands(ctx):
    batch = W.make_config("ont", n_pairs=8)            # w = 500: 16-slot frame
    with pytest.raises(A.AgathaError) as e:
        A.agatha_align_batch(ctx, batch, flags=A.AGATHA_HALF_WARP)
    assert e.value.code == A.AGATHA_ENOTSUP
    with pytest.raises(A.AgathaError) as e:
        A.agatha_align_batch(ctx, W.make_config("small", n_pairs=8),
                             flags=A.AGATHA_HALF_WARP | A.AGATHA_WARPS2)
    assert e.value.code == A.AGATHA_EINVAL


def test_half_warp_pairs_of_uneven_lengths(ctx):
    # two pairs per warp whose lengths, stops and overflows differ: each half
    # warp takes its own pairs and goes its own way through the steps
    rng = np.random.default_rng(23)
    scoring = W.Scoring(2, 4, 4, 2, 24, 1, 60, 40, 3)
    qs, ts = [], []
    for k in range(600):
        L = int(rng.integers(0, 400))
        q = rng.integers(0, 4, L).astype(np.uint8)
        if k % 3 == 0:
            t = q.copy()
        elif k % 3 == 1:
            t = rng.integers(0, 4, max(0, L + int(rng.integers(-70, 70)))).astype(np.uint8)
        else:
            t = np.concatenate([q[: L // 3], rng.integers(0, 4, L - L // 3)]).astype(np.uint8)
        qs.append(q); ts.append(t)
    batch = W.from_pairs(qs, ts, scoring, name="uneven")
    ref = O.align_batch(batch)
    for flags in (A.AGATHA_HALF_WARP, A.AGATHA_HALF_WARP | A.AGATHA_NO_SORT):
        _assert_same(A.agatha_align_batch(ctx, batch, flags=flags), ref, batch, f"uneven/{flags}")


def test_short_pairs_of_a_wide_band_on_the_narrower_frame(ctx):
    # a 24-slot batch (w = 750): pairs whose own band fits 640 slots run on
    # the 20-slot kernel after the main launch; with AGATHA_ONE_FRAME all run
    # on the 24-slot one.  Both against the oracle on every pair, with lengths
    # on both sides of the 638 boundary.
    rng = np.random.default_rng(31)
    sk = W.make_config("skewed", n_pairs=2500)
    qs = [sk.query(i) for i in range(sk.n_pairs)]
    ts = [sk.target(i) for i in range(sk.n_pairs)]
    for L in (1, 60, 400, 636, 637, 638, 639, 640, 700):
        q = rng.integers(0, 4, L).astype(np.uint8)
        qs += [q, q]
        ts += [q.copy(), rng.integers(0, 4, max(1, L + int(rng.integers(-3, 4)))).astype(np.uint8)]
    batch = W.from_pairs(qs, ts, sk.scoring, name="narrow")
    weff = np.minimum(np.maximum(batch.t_len, batch.q_len), sk.scoring.w)
    assert (weff <= 638).sum() > 100 and (weff > 638).sum() > 100
    ref = O.align_batch(batch)
    for flags in (0, A.AGATHA_ONE_FRAME, A.AGATHA_REGS_HIGH):
        _assert_same(A.agatha_align_batch(ctx, batch, flags=flags), ref, batch, f"narrow/{flags}")
