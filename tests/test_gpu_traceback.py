"""GPU parity of the traceback path (agatha_align_cigar).

Every pair's CIGAR runs must equal the oracle's traceback bit for bit (the
same tie rule on the same integer table), and the results must equal those
of the score path alone.  At full size the oracle traces the longest pairs
and a uniform sample; every pair is checked for the lengths its runs consume.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2403_06478_gb300 import agatha as A
from paper_2403_06478_gb300 import build as B
from paper_2403_06478_gb300 import workload as W
from test_gpu_parity import ADVERSARIAL_SCORINGS, _adversarial_batch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    B.build()
    c = A.Context(0, timing=True)
    yield c
    c.close()


def _runs(off, cig, i):
    return cig[off[i]:off[i + 1]]


def _consumed(off, cig, n):
    """Target and query bases each pair's runs consume (vectorised)."""
    lens = (cig >> 4).astype(np.int64)
    op = cig & 15
    pair = np.repeat(np.arange(n), np.diff(off))
    t = np.bincount(pair, weights=lens * (op != A.AGATHA_CIGAR_I), minlength=n).astype(np.int64)
    q = np.bincount(pair, weights=lens * (op != A.AGATHA_CIGAR_D), minlength=n).astype(np.int64)
    return t, q


def _end_cells(res, batch):
    et = np.where(res["reach_end"] == 1, res["mqe_t"], res["te"]).astype(np.int64)
    eq = np.where(res["reach_end"] == 1, batch.q_len.astype(np.int64) - 1, res["qe"]).astype(np.int64)
    empty = (batch.t_len <= 0) | (batch.q_len <= 0) | (et < 0) | (eq < 0)
    et[empty] = -1
    eq[empty] = -1
    return et, eq


def _check(ctx, batch, label, idx=None, flags=0):
    pb = A.pack_batch(batch)
    res, off, cig = ctx.align_cigar(pb, batch.scoring, flags=flags)
    alone = A.agatha_align_batch(ctx, batch, flags=flags)
    assert A.results_equal(res, alone).size == 0, f"{label}: results differ from the score path"
    n = batch.n_pairs
    assert off.shape == (n + 1,) and off[0] == 0 and (np.diff(off) >= 0).all()
    # every pair: the runs reach exactly the end cell
    et, eq = _end_cells(res, batch)
    t, q = _consumed(off, cig, n)
    assert (t == et + 1).all() and (q == eq + 1).all(), f"{label}: a path misses its end cell"
    assert ((cig >> 4) > 0).all() and ((cig & 15) <= 2).all()
    # the oracle, pair by pair
    idx = np.arange(n) if idx is None else np.asarray(idx)
    ref = O.align_batch(batch, idx=idx)
    bad = A.results_equal(res[idx], ref, O.COMPARE_FIELDS)
    assert bad.size == 0, f"{label}: results differ from the oracle at {idx[bad[:5]]}"
    cigs, scores = O.traceback_batch(batch, {int(i): ref[k] for k, i in enumerate(idx)}, idx)
    for k, i in enumerate(idx):
        got = _runs(off, cig, int(i))
        if not np.array_equal(got, cigs[k]):
            raise AssertionError(f"{label}: pair {int(i)} (tlen={int(batch.t_len[i])}, "
                                 f"qlen={int(batch.q_len[i])}) CIGAR {A.cigar_string(got)[:200]} "
                                 f"!= oracle {O.cigar_string(cigs[k])[:200]}")
        want = int(ref[k]["mqe"]) if ref[k]["reach_end"] else int(ref[k]["max"])
        if et[i] >= 0:
            assert scores[k] == want
    return res, off, cig


# the three traceback forms: fused (default), two-pass on 16-bit lanes, int32
TB_FLAGS = [0, A.AGATHA_TB_TWO_PASS, A.AGATHA_FORCE32]


def _kernels(ctx, res, batch, flags):
    """The traceback kernel that ran, and that no pair was handed back: the
    fused kernel takes every non-empty pair, the two-pass kernels every pair
    with a path (16-bit lanes unless FORCE32)."""
    info = ctx.last_traceback_info()
    et, _ = _end_cells(res, batch)
    traced = int((et >= 0).sum())
    nonempty = int(((batch.t_len > 0) & (batch.q_len > 0)).sum())
    if flags & A.AGATHA_FORCE32:
        assert info["pairs16"] == 0 and info["pairs32"] == traced and info["fused"] == 0, info
    elif flags & (A.AGATHA_TB_TWO_PASS | A.AGATHA_PLAIN):
        assert info["pairs16"] == traced and info["pairs32"] == 0 and info["fused"] == 0, info
    else:
        assert info["pairs16"] == nonempty == info["fused"] and info["pairs32"] == 0, info
    assert info["waves"] >= (1 if traced else 0)


@pytest.mark.parametrize("flags", TB_FLAGS + [A.AGATHA_PLAIN])
def test_small_config_every_pair(ctx, flags):
    batch = W.make_config("small")
    res, _, _ = _check(ctx, batch, f"small/{flags}", flags=flags)
    _kernels(ctx, res, batch, flags)
    assert ctx.last_traceback_ms() > 0


@pytest.mark.parametrize("si", [i for i, s in enumerate(ADVERSARIAL_SCORINGS) if s.w >= 0])
def test_adversarial_pairs(ctx, si):
    scoring = ADVERSARIAL_SCORINGS[si]
    batch = _adversarial_batch(np.random.default_rng(100 + si), scoring)
    for flags in TB_FLAGS:
        _check(ctx, batch, f"adversarial[{si}]/{flags}", flags=flags)


@pytest.mark.parametrize("name,n", [("ont", 120), ("hifi", 120), ("skewed", 600), ("short", 2000)])
@pytest.mark.parametrize("flags", TB_FLAGS)
def test_workload_mixes_every_pair(ctx, name, n, flags):
    batch = W.make_config(name, n_pairs=n)
    res, _, _ = _check(ctx, batch, f"{name}/{flags}", flags=flags)
    _kernels(ctx, res, batch, flags)


def test_16bit_overflow_hands_pairs_to_int32(ctx):
    # pairs whose band spreads scores beyond what 16-bit lanes keep (as in the
    # score path's overflow test): the 16-bit traceback kernel hands them back
    # and the int32 kernel traces them; the short ones stay on 16-bit lanes
    rng = np.random.default_rng(17)
    scoring = W.Scoring(64, 64, 1, 63, 1, 63, 511, -1, 0)
    qs, ts = [], []
    for k in range(4):
        x = rng.integers(0, 4, 2500 + 100 * k).astype(np.uint8)
        y = x.copy()
        y[rng.integers(0, x.size, 20)] = rng.integers(0, 4, 20)
        qs.append(x)
        ts.append(y)
    for k in range(5):
        x = rng.integers(0, 4, 250).astype(np.uint8)
        qs.append(x)
        ts.append(x.copy())
    batch = W.from_pairs(qs, ts, scoring)
    for flags in (0, A.AGATHA_TB_TWO_PASS):
        res, _, _ = _check(ctx, batch, f"overflow/{flags}", flags=flags)
        assert (res["lane16"][:4] == 0).all()       # recomputed on int32 lanes
        assert (res["lane16"][4:] == 1).all()
        info = ctx.last_traceback_info()
        assert info["pairs16"] == 9 and 1 <= info["pairs32"] <= 4, info


@pytest.mark.parametrize("scoring", [
    W.Scoring(1, 20, 4, 30, 4, 30, 511, -1, 0),     # steep single-piece gaps, no Z-drop
    W.Scoring(1, 9, 16, 3, 41, 1, 300, -1, 0),      # assembly-like two-piece
    W.Scoring(10, 90, 100, 50, 200, 20, 127, 5000, 0),
    W.Scoring(2, 1, 0, 1, 3, 0, 64, 40, 4),         # free gap opening: many ties
])
def test_steep_and_tied_scorings(ctx, scoring):
    rng = np.random.default_rng(29)
    qs, ts = [], []
    for L in (50, 300, 900, 2000):
        for k in range(5):
            x = rng.integers(0, 2 + 2 * (k % 2), L).astype(np.uint8)
            y = x.copy()
            y[rng.integers(0, L, L // 25)] = rng.integers(0, 4, L // 25)
            cut = int(rng.integers(0, min(scoring.w, L // 2)))
            qs.append(x)
            ts.append(y[: L - cut] if k % 2 else np.concatenate([y, rng.integers(0, 4, cut)]).astype(np.uint8))
    batch = W.from_pairs(qs, ts, scoring)
    for flags in TB_FLAGS:
        _check(ctx, batch, f"steep/{scoring}/{flags}", flags=flags)


def test_empty_and_degenerate_pairs(ctx):
    sc = W.Scoring(2, 4, 4, 2, 24, 1, 20, 40, 0)
    qs = ["", "A", "", "ACGT", "AAAA", "ACGTACGT", "C"]
    ts = ["", "", "ACGT", "ACGT", "CCCC", "ACGTACGT", "C"]
    batch = W.from_pairs(qs, ts, sc)
    res, off, cig = _check(ctx, batch, "degenerate")
    assert list(np.diff(off)) == [0, 0, 0, 1, 0, 1, 1]      # AAAA/CCCC: maximum at the origin
    assert A.cigar_string(_runs(off, cig, 3)) == "4M"
    assert A.cigar_string(_runs(off, cig, 5)) == "8M"
    empty = W.from_pairs([], [], sc)
    res, off, cig = ctx.align_cigar(A.pack_batch(empty), sc)
    assert res.shape == (0,) and list(off) == [0] and cig.size == 0


def test_errors(ctx):
    batch = W.make_config("small", n_pairs=16)
    pb = A.pack_batch(batch)
    with pytest.raises(A.AgathaError) as e:
        ctx.align_cigar(pb, batch.scoring, cigar_cap=3)
    assert e.value.code == A.AGATHA_ERANGE
    with pytest.raises(A.AgathaError) as e:
        ctx.align_cigar(pb, batch.scoring, flags=A.AGATHA_DEVICE_PTRS)
    assert e.value.code == A.AGATHA_ENOTSUP
    wide = W.from_pairs([np.zeros(1500, np.uint8)], [np.zeros(1500, np.uint8)], W.Scoring(w=-1))
    with pytest.raises(A.AgathaError) as e:
        ctx.align_cigar(A.pack_batch(wide), wide.scoring)
    assert e.value.code == A.AGATHA_ENOTSUP
    # the context still works after the errors
    _check(ctx, W.make_config("small", n_pairs=32), "after errors")


@pytest.mark.parametrize("flags", [0, A.AGATHA_TB_TWO_PASS])
def test_waves_under_a_small_budget(flags):
    # a budget that holds the tables of only a few pairs at a time: many
    # waves, same CIGARs as one wave
    batch = W.make_config("ont", n_pairs=60)
    with A.Context(0) as big:
        r1, o1, c1 = big.align_cigar(A.pack_batch(batch), batch.scoring, flags=flags)
        assert big.last_traceback_info()["waves"] == 1
    with A.Context(0, mem_budget_bytes=120 << 20) as small:
        r2, o2, c2 = small.align_cigar(A.pack_batch(batch), batch.scoring, flags=flags)
        assert small.last_traceback_info()["waves"] > 1
    assert A.results_equal(r1, r2).size == 0
    assert np.array_equal(o1, o2) and np.array_equal(c1, c2)


def test_ont_full_size_sampled(ctx):
    # the bench's traceback workload: 20,000 ONT-like pairs, one call
    batch = W.make_config("ont")
    rng = np.random.default_rng(11)
    longest = np.argsort(-(batch.q_len.astype(np.int64) + batch.t_len))[:6]
    idx = np.unique(np.concatenate([longest, rng.choice(batch.n_pairs, 40, replace=False)]))
    res, _, _ = _check(ctx, batch, "ont/full", idx=idx)
    _kernels(ctx, res, batch, 0)
