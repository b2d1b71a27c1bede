"""The local extension from an initial score (the BWA-MEM variant) on the
GPU, through agatha_align_batch_local, against the CPU oracle: every pair,
every output field, exact (integer outputs, tolerance 0)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2403_06478_gb300 import agatha as A
from paper_2403_06478_gb300 import build as B
from paper_2403_06478_gb300 import workload as W

pytestmark = pytest.mark.gpu

FIELDS = O.COMPARE_FIELDS


@pytest.fixture(scope="module")
def ctx():
    B.build()
    c = A.Context(0)
    yield c
    c.close()


def _same(got, ref, batch, h0, label):
    bad = A.results_equal(got, ref, FIELDS)
    if bad.size:
        i = int(bad[0])
        diff = {f: (int(got[i][f]), int(ref[i][f])) for f in FIELDS if got[i][f] != ref[i][f]}
        raise AssertionError(f"{label}: {bad.size} of {got.shape[0]} pairs differ; first pair {i} "
                             f"(tlen={int(batch.t_len[i])}, qlen={int(batch.q_len[i])}, h0={int(h0[i])}) "
                             f"got/expected: {diff}")


def _run(ctx, batch, h0, flags=0):
    return ctx.align_local(A.pack_batch(batch), batch.scoring, h0, flags=flags)


SCORINGS = [
    W.BWA_SCORING,                                   # a=1 b=4 q=6 e=1, w=100, zdrop 100, end bonus 5
    W.Scoring(1, 4, 6, 1, 6, 1, 7, 20, 5),           # narrow band, frequent Z-drop
    W.Scoring(2, 4, 4, 2, 24, 1, 50, 60, 0),         # two-piece
    W.Scoring(3, 2, 1, 1, 3, 0, 31, 0, 2),           # zdrop 0, free second piece
    W.Scoring(1, 4, 6, 1, 6, 1, 127, -1, 5),         # no Z-drop, 4-slot frame full
    W.Scoring(2, 4, 4, 2, 24, 1, 300, 100, 0),       # 16 slots per lane
]


def _adversarial(rng, scoring):
    qs, ts = [], []
    w = scoring.w
    for L in (0, 1, 2, 3, 5, 16, 31, 32, 33, 64, 100, 150, 250, 400):
        q = rng.integers(0, 4, L).astype(np.uint8)
        qs.append(q); ts.append(q.copy())                                  # identical
        qs.append(q); ts.append(((q + 1) % 4).astype(np.uint8))            # all mismatch: dies at once
        t = rng.integers(0, 4, max(0, L + int(rng.integers(-w - 2, w + 3)))).astype(np.uint8)
        qs.append(q); ts.append(t)                                         # unrelated, length gap near w
        mq = q.copy()
        if L:
            mq[rng.integers(0, L, max(1, L // 20))] = rng.integers(0, 4, max(1, L // 20))
        qs.append(mq); ts.append(np.concatenate([q[: L // 2], rng.integers(0, 4, L - L // 2)]).astype(np.uint8))
    b2 = W.random_pairs(rng, 80, 300, scoring, min_len=0, related=0.7)
    for i in range(b2.n_pairs):
        qs.append(b2.query(i)); ts.append(b2.target(i))
    return W.from_pairs(qs, ts, scoring, name="adversarial")


@pytest.mark.parametrize("si", range(len(SCORINGS)))
def test_adversarial_pairs_match_oracle(ctx, si):
    scoring = SCORINGS[si]
    rng = np.random.default_rng(700 + si)
    batch = _adversarial(rng, scoring)
    h0 = rng.choice([1, 3, 8, 20, 45, 200], batch.n_pairs).astype(np.int32)
    ref = O.align_batch(batch, h0=h0)
    _same(_run(ctx, batch, h0), ref, batch, h0, f"local[{si}]")
    _same(_run(ctx, batch, h0, A.AGATHA_NO_SORT), ref, batch, h0, f"local[{si}]/no_sort")


def test_short_reads_with_bwa_parameters(ctx):
    # 150 bp extensions with BWA-MEM's default scoring from seed scores of 19-60
    batch = W.make_config("short", n_pairs=20000)
    h0 = W.seed_scores(batch.n_pairs)
    ref = O.align_batch(batch, h0=h0)
    got = _run(ctx, batch, h0)
    _same(got, ref, batch, h0, "short/local")
    assert ref["reach_end"].sum() > 0 and ref["zdropped"].sum() > 0


def test_ont_pairs_with_a_band_of_100(ctx):
    batch = W.make_config("ont", n_pairs=300).with_scoring(w=100, zdrop=100)
    h0 = W.seed_scores(batch.n_pairs, seed=3)
    ref = O.align_batch(batch, h0=h0)
    _same(_run(ctx, batch, h0), ref, batch, h0, "ont/local")


def test_device_pointers(ctx):
    torch = pytest.importorskip("torch")
    import ctypes
    batch = W.make_config("short", n_pairs=500)
    h0 = W.seed_scores(batch.n_pairs, seed=5)
    pb = A.pack_batch(batch)
    dev = {k: torch.from_numpy(getattr(pb, k)).cuda() for k in
           ("q_packed", "t_packed", "q_off", "t_off", "q_len", "t_len")}
    dh0 = torch.from_numpy(h0).cuda()
    out = torch.zeros(pb.n_pairs * 48, dtype=torch.uint8, device="cuda")
    b = A.agatha_batch(pb.n_pairs, dev["q_packed"].data_ptr(), dev["t_packed"].data_ptr(),
                       pb.q_packed.shape[0], pb.t_packed.shape[0], dev["q_off"].data_ptr(),
                       dev["t_off"].data_ptr(), dev["q_len"].data_ptr(), dev["t_len"].data_ptr())
    p = A.make_params(batch.scoring)
    rc = A.lib().agatha_align_batch_local(ctx.handle, ctypes.byref(b), ctypes.byref(p), dh0.data_ptr(),
                                          out.data_ptr(), A.AGATHA_DEVICE_PTRS, None)
    assert rc == A.AGATHA_OK
    got = out.cpu().numpy().view(A.RESULT_DTYPE)
    _same(got, O.align_batch(batch, h0=h0), batch, h0, "device")
    # an initial score outside [1, 2^24] found by the device check
    bad = dh0.clone()
    bad[7] = 0
    rc = A.lib().agatha_align_batch_local(ctx.handle, ctypes.byref(b), ctypes.byref(p), bad.data_ptr(),
                                          out.data_ptr(), A.AGATHA_DEVICE_PTRS, None)
    assert rc == A.AGATHA_EINVAL
    r = out.cpu().numpy().view(A.RESULT_DTYPE)[7]
    assert (r["max"], r["qe"], r["te"], r["cells"]) == (0, -1, -1, 0)


def test_host_errors(ctx):
    batch = W.make_config("short", n_pairs=10)
    h0 = W.seed_scores(batch.n_pairs)
    h0[3] = -1
    with pytest.raises(A.AgathaError) as e:
        _run(ctx, batch, h0)
    assert e.value.code == A.AGATHA_EINVAL
    with pytest.raises(A.AgathaError) as e:
        ctx.align_local(A.pack_batch(batch), W.Scoring(1, 4, 6, 1, 6, 1, -1, 100, 5), W.seed_scores(batch.n_pairs))
    assert e.value.code == A.AGATHA_ENOTSUP
    empty = W.from_pairs(["", "ACGT", ""], ["", "", "AC"], W.BWA_SCORING)
    got = _run(ctx, empty, np.array([5, 6, 7], np.int32))
    assert list(got["max"]) == [5, 6, 7] and (got["qe"] == -1).all() and (got["cells"] == 0).all()
