"""The seeded input generators: shapes, determinism and the error profile they
claim (they feed both the GPU path and the oracle, so they are checked here
on their own)."""
import numpy as np
import pytest

from paper_2403_06478_gb300 import workload as W


def test_configs_are_deterministic_and_shaped():
    a = W.make_config("small")
    b = W.make_config("small")
    assert a.n_pairs == 256 and (a.q_len == 1000).all()
    assert np.array_equal(a.q_codes, b.q_codes) and np.array_equal(a.t_codes, b.t_codes)
    assert a.q_codes.max() <= 3 and a.t_codes.max() <= 3
    assert (a.q_off[1:] == np.cumsum(a.q_len)[:-1]).all()
    ont = W.make_config("ont", n_pairs=3000)
    assert ont.q_len.min() >= 500 and ont.q_len.max() <= 50_000
    assert 3500 < np.median(ont.q_len) < 6500          # log-normal, median 5 kbp


def test_error_rates_are_near_the_stated_ones():
    b = W.make_config("small")
    # lengths move by insertions minus deletions: 2.5% each, so about zero on average
    assert abs(float(np.mean(b.t_len.astype(np.int64) - b.q_len))) < 5
    # identity of the aligned prefix before the first indel is about 95%
    same = [np.mean(b.query(i)[:20] == b.target(i)[:20]) for i in range(b.n_pairs)]
    assert 0.7 < float(np.mean(same)) <= 1.0


@pytest.mark.parametrize("f", [0.0, 0.1, 0.5])
def test_long_ratio_mix(f):
    b = W.make_long_ratio(f, n_pairs=400)
    n_long = int((b.q_len == 4096).sum())
    assert n_long == int(round(f * 400))
    assert set(np.unique(b.q_len)) <= {128, 4096}
    again = W.make_long_ratio(f, n_pairs=400)
    assert np.array_equal(b.q_len, again.q_len) and np.array_equal(b.t_codes, again.t_codes)


def test_poisson_requests():
    rng = np.random.default_rng(1)
    reqs = W.poisson_requests(rng, 100.0, 2000, 500, 512)
    t = np.array([r.arrival_s for r in reqs])
    assert (np.diff(t) >= 0).all()
    assert 15 < t[-1] < 25                              # 2000 arrivals at 100/s
    sizes = np.array([len(r.pair_idx) for r in reqs])
    assert sizes.min() >= 1 and sizes.max() <= 512
    assert all((r.pair_idx >= 0).all() and (r.pair_idx < 500).all() for r in reqs)


def test_short_read_workload():
    b = W.make_config("short", n_pairs=2000)
    assert b.n_pairs == 2000 and (b.q_len == 150).all()
    assert b.scoring == W.BWA_SCORING and b.scoring.end_bonus == 5
    assert abs(float(np.mean(b.t_len.astype(np.int64) - b.q_len))) < 1
    again = W.make_config("short", n_pairs=2000)
    assert np.array_equal(b.t_codes, again.t_codes)


def test_full_batch_oracle_digests_match_the_generator():
    # the stored oracle digests of the full-size workloads (written by
    # tests/golden/full_batch_digests.py from the oracle alone) were taken on
    # exactly the inputs this generator draws; the GPU test of every pair
    # relies on that, and falls back to a live oracle run where it fails
    from golden import full_batch_digests as G
    recs = G.read_golden()
    assert sorted(recs) == sorted(G.CONFIGS)
    for name, rec in recs.items():
        batch = W.make_config(name)
        assert rec["n_pairs"] == batch.n_pairs
        assert len(rec["chunks"]) == -(-batch.n_pairs // rec["chunk"])
        assert G.input_digest(batch) == rec["input"], name
        assert 0 < rec["zdropped"] < batch.n_pairs
