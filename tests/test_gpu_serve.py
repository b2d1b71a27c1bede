"""Serving loop on the GPU: merged launches give every request exactly the
results it gets alone (and the oracle's), the memory budget is never
exceeded, and the ticket states (timeout, cancel, drain) behave as declared."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2403_06478_gb300 import agatha as A
from paper_2403_06478_gb300 import build as B
from paper_2403_06478_gb300 import workload as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    B.build()
    c = A.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def pools():
    return {
        "ont": W.make_config("ont", n_pairs=600),
        "hifi": W.make_config("hifi", n_pairs=120),
        "small": W.make_config("small"),
    }


def _requests(pools, n_req, seed, max_pairs=48):
    rng = np.random.default_rng(seed)
    names = sorted(pools)
    reqs = []
    for _ in range(n_req):
        pool = pools[names[int(rng.integers(0, len(names)))]]
        k = int(rng.integers(1, max_pairs + 1))
        reqs.append(pool.subset(rng.choice(pool.n_pairs, k, replace=False)))
    return reqs


def _device_bytes(b):
    """Upper bound of one request's device block: the words its pairs touch,
    offsets, lengths, results and three index lists, each rounded to 256 B."""
    words = int(((b.q_len.astype(np.int64) + 31) // 16).sum() + ((b.t_len.astype(np.int64) + 31) // 16).sum())
    return 4 * words + b.n_pairs * (8 + 8 + 4 + 4 + 48 + 12) + 10 * 256


def _serve_all(ctx, reqs, **cfg):
    srv = A.Server(ctx, **cfg)
    try:
        tickets = [srv.submit(A.pack_batch(b), b.scoring) for b in reqs]
        got = [srv.wait(t, 120_000) for t in tickets]
        return got, srv.stats()
    finally:
        srv.stop(drain=True)


def test_mixed_requests_match_alone_and_oracle(ctx, pools):
    reqs = _requests(pools, 60, 11)
    # linger so that requests with the same scoring are merged into launches
    got, st = _serve_all(ctx, reqs, max_inflight=2, max_batch_pairs=400, linger_us=3000)
    assert st["requests_done"] == len(reqs)
    assert st["pairs_done"] == sum(b.n_pairs for b in reqs)
    assert st["launches"] < len(reqs)                  # merging happened
    assert 0 < st["p50_latency_ms"] <= st["p99_latency_ms"]
    cells = 0
    for i, (b, g) in enumerate(zip(reqs, got)):
        alone = A.agatha_align_batch(ctx, b)
        assert A.results_equal(g, alone).size == 0, f"request {i} differs from its own batch"
        cells += int(g["cells"].sum())
    assert st["cells_done"] == cells
    for i in (0, 7, 23):                                # whole requests against the oracle
        ref = O.align_batch(reqs[i])
        assert A.results_equal(got[i], ref, O.COMPARE_FIELDS).size == 0


def test_budget_is_never_exceeded(ctx, pools):
    reqs = _requests(pools, 40, 12, max_pairs=64)
    # room for about two of the largest requests at once
    budget = 2 * max(_device_bytes(b) for b in reqs)
    got, st = _serve_all(ctx, reqs, mem_budget_bytes=budget, max_inflight=4, max_batch_pairs=4096)
    assert st["requests_done"] == len(reqs)
    assert 0 < st["peak_bytes_in_flight"] <= budget
    assert st["bytes_in_flight"] == 0
    for b, g in zip(reqs, got):
        assert A.results_equal(g, A.agatha_align_batch(ctx, b)).size == 0


def test_request_larger_than_budget_is_refused(ctx, pools):
    srv = A.Server(ctx, mem_budget_bytes=1 << 16)
    try:
        big = pools["ont"].subset(np.arange(200))
        with pytest.raises(A.AgathaError) as e:
            srv.submit(A.pack_batch(big), big.scoring)
        assert e.value.code == A.AGATHA_ENOMEM
        small = pools["small"].subset(np.arange(2))
        t = srv.submit(A.pack_batch(small), small.scoring)
        assert A.results_equal(srv.wait(t, 60_000), A.agatha_align_batch(ctx, small)).size == 0
    finally:
        srv.stop()


def test_timeout_cancel_and_drain(ctx, pools):
    b = pools["small"].subset(np.arange(8))
    # a long linger keeps a lone short request queued
    srv = A.Server(ctx, linger_us=20_000_000, max_batch_pairs=100_000)
    t1 = srv.submit(A.pack_batch(b), b.scoring)
    assert srv.wait_code(t1, 20) == A.AGATHA_ETIMEDOUT
    assert srv.poll(t1) == A.AGATHA_EAGAIN
    srv.stop(drain=False)
    assert srv.poll(t1) == A.AGATHA_ECANCELED
    assert srv.wait_code(t1, 0) == A.AGATHA_ECANCELED
    assert srv.poll(t1) == A.AGATHA_EINVAL             # forgotten after the final status
    with pytest.raises(A.AgathaError) as e:
        srv.submit(A.pack_batch(b), b.scoring)
    assert e.value.code == A.AGATHA_EINVAL

    srv = A.Server(ctx, linger_us=20_000_000, max_batch_pairs=100_000)
    t2 = srv.submit(A.pack_batch(b), b.scoring)
    srv.stop(drain=True)                               # drain launches the lingering batch
    assert srv.poll(t2) == A.AGATHA_OK
    assert A.results_equal(srv.wait(t2, 0), A.agatha_align_batch(ctx, b)).size == 0


def test_empty_request_and_bad_input(ctx, pools):
    srv = A.Server(ctx)
    try:
        e0 = W.from_pairs([], [], W.SMALL_SCORING)
        t = srv.submit(A.pack_batch(e0), e0.scoring)
        assert srv.wait(t, 1000).shape[0] == 0
        b = pools["small"].subset(np.arange(4))
        with pytest.raises(A.AgathaError) as e:
            srv.submit(A.pack_batch(b), W.Scoring(w=0))
        assert e.value.code == A.AGATHA_EINVAL
        pb = A.pack_batch(b)
        pb.q_off = pb.q_off.copy()
        pb.q_off[1] = int(pb.q_packed.shape[0]) * 16
        with pytest.raises(A.AgathaError) as e:
            srv.submit(pb, b.scoring)
        assert e.value.code == A.AGATHA_EINVAL
        assert srv.poll(987654321) == A.AGATHA_EINVAL
    finally:
        srv.stop()


def test_serving_uses_the_tuned_plan(tmp_path, ctx, pools):
    import torch
    prop = torch.cuda.get_device_properties(0)
    s = pools["ont"].scoring
    key = (f"sm{prop.multi_processor_count}_cc{prop.major}{prop.minor}_a{s.a}_b{s.b}_q{s.q}_e{s.e}"
           f"_q2{s.q2}_e2{s.e2}_w{s.w}_z{s.zdrop}_c16")
    path = tmp_path / "tune.txt"
    path.write_text(key + " 2 1 0 1 1\n")           # one launch per class, mixed variants
    reqs = [r for r in _requests(pools, 30, 13) if r.scoring == s]
    with A.Context(0, autotune=True, tune_cache_path=str(path)) as tuned:
        got, st = _serve_all(tuned, reqs, max_inflight=2, max_batch_pairs=400, linger_us=2000)
    assert st["requests_done"] == len(reqs)
    for b, g in zip(reqs, got):
        assert A.results_equal(g, A.agatha_align_batch(ctx, b)).size == 0


def test_burst_runs_launches_concurrently_on_the_device(ctx, pools):
    # a burst of ONT-like requests, one request per launch: the next launch's
    # kernels start while the previous one's longest pairs still run, which
    # the device's global timer shows (first block of a launch's first kernel
    # before the last warp of the running launch finished)
    rng = np.random.default_rng(31)
    pool = pools["ont"]
    reqs = [pool.subset(rng.choice(pool.n_pairs, 64, replace=False)) for _ in range(24)]
    got, st = _serve_all(ctx, reqs, max_inflight=3, max_batch_pairs=64)
    assert st["requests_done"] == len(reqs)
    assert st["launches"] == len(reqs)
    assert st["max_launches_in_flight"] >= 2
    assert st["max_device_concurrency"] >= 2
    assert st["overlap_seconds"] > 0
    for i, (b, g) in enumerate(zip(reqs, got)):
        assert A.results_equal(g, A.agatha_align_batch(ctx, b)).size == 0, f"request {i}"
    for i in (0, 11):
        assert A.results_equal(got[i], O.align_batch(reqs[i]), O.COMPARE_FIELDS).size == 0


@pytest.mark.parametrize("flags", [A.AGATHA_WARPS2 | A.AGATHA_REGS_HIGH, A.AGATHA_WARPS4])
def test_serving_with_several_warps_per_pair(ctx, pools, flags):
    # the server's own plan: 2 or 4 warps per pair where the band has those
    # kernels (ONT, HiFi: w = 500), one warp per pair elsewhere (small: w = 100)
    reqs = _requests(pools, 40, 17)
    got, st = _serve_all(ctx, reqs, max_inflight=2, max_batch_pairs=400, linger_us=2000,
                         launch_flags=flags)
    assert st["requests_done"] == len(reqs)
    for i, (b, g) in enumerate(zip(reqs, got)):
        assert A.results_equal(g, A.agatha_align_batch(ctx, b)).size == 0, f"request {i}"
    ref = O.align_batch(reqs[3])
    assert A.results_equal(got[3], ref, O.COMPARE_FIELDS).size == 0


def test_serving_rejects_other_launch_flags(ctx):
    for bad in (A.AGATHA_PLAIN, A.AGATHA_WARPS2 | A.AGATHA_WARPS4, A.AGATHA_HALF_WARP):
        with pytest.raises(A.AgathaError) as e:
            A.Server(ctx, launch_flags=bad)
        assert e.value.code == A.AGATHA_EINVAL
