"""Autotuner on the GPU: the per-length-class launches give the same results
whatever variant each class runs, tuning fills the cache file, and a new
context reads it back."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2403_06478_gb300 import agatha as A
from paper_2403_06478_gb300 import build as B
from paper_2403_06478_gb300 import workload as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def batch():
    B.build()
    # ONT-like lengths fill three of the four length classes
    return W.make_config("ont", n_pairs=3000)


@pytest.fixture(scope="module")
def reference(batch):
    with A.Context(0) as ctx:
        return A.agatha_align_batch(ctx, batch)


def _key(scoring, c16):
    import torch
    prop = torch.cuda.get_device_properties(0)
    s = scoring
    return (f"sm{prop.multi_processor_count}_cc{prop.major}{prop.minor}_a{s.a}_b{s.b}_q{s.q}_e{s.e}"
            f"_q2{s.q2}_e2{s.e2}_w{s.w}_z{s.zdrop}_c{c16}")


def test_tuning_fills_cache_and_keeps_results(tmp_path, batch, reference):
    path = str(tmp_path / "tune.txt")
    with A.Context(0, autotune=True, tune_cache_path=path) as ctx:
        assert ctx.tune_variants(batch.scoring) is None
        got = A.agatha_align_batch(ctx, batch)
        v = ctx.tune_variants(batch.scoring)
        assert v is not None and len(v) == 5
        assert all(0 <= x < len(A.VARIANT_NAMES) for x in v[:4]) and v[4] in (0, 1)
        assert A.results_equal(got, reference).size == 0
        again = A.agatha_align_batch(ctx, batch)             # the tuned plan
        assert A.results_equal(again, reference).size == 0
    lines = open(path).read().split("\n")
    assert lines[0].split()[0] == _key(batch.scoring, 16)
    assert [int(x) for x in lines[0].split()[1:]] == v
    with A.Context(0, autotune=True, tune_cache_path=path) as ctx2:
        assert ctx2.tune_variants(batch.scoring) == v     # read back, nothing measured
        assert A.results_equal(A.agatha_align_batch(ctx2, batch), reference).size == 0


@pytest.mark.parametrize("variants", [(2, 1, 0, 2), (1, 2, 1, 0), (0, 0, 2, 1), (2, 2, 2, 2),
                                      (0, 0, 0, 0), (3, 3, 1, 1), (4, 3, 0, 1), (4, 4, 4, 4),
                                      (3, 1, 2, 3)])
def test_every_class_variant_is_exact(tmp_path, batch, reference, variants):
    path = tmp_path / "tune.txt"
    path.write_text(_key(batch.scoring, 16) + " " + " ".join(map(str, variants)) + " 1\n")
    with A.Context(0, autotune=True, tune_cache_path=str(path)) as ctx:
        assert ctx.tune_variants(batch.scoring) == list(variants) + [1]
        got = A.agatha_align_batch(ctx, batch)
        assert A.results_equal(got, reference).size == 0
        # device-resident batches take the tuned split as well
        torch = pytest.importorskip("torch")
        pb = A.pack_batch(batch)
        dev = {k: torch.from_numpy(getattr(pb, k)).cuda() for k in
               ("q_packed", "t_packed", "q_off", "t_off", "q_len", "t_len")}
        out = torch.zeros(pb.n_pairs * 48, dtype=torch.uint8, device="cuda")
        ctx.align_device(dev["q_packed"], dev["t_packed"], dev["q_off"], dev["t_off"], dev["q_len"],
                         dev["t_len"], out, batch.scoring)
        assert A.results_equal(out.cpu().numpy().view(A.RESULT_DTYPE), reference).size == 0


@pytest.mark.parametrize("variant", [1, 2, 3, 4])
def test_single_launch_of_another_variant_is_exact(tmp_path, batch, reference, variant):
    path = tmp_path / "tune.txt"
    path.write_text(_key(batch.scoring, 16) + f" {variant} {variant} {variant} {variant} 0\n")
    with A.Context(0, autotune=True, tune_cache_path=str(path)) as ctx:
        assert ctx.tune_variants(batch.scoring) == [variant] * 4 + [0]
        assert A.results_equal(A.agatha_align_batch(ctx, batch), reference).size == 0


def test_split_launches_match_oracle_on_a_sample(tmp_path, batch, reference):
    path = tmp_path / "tune.txt"
    path.write_text(_key(batch.scoring, 16) + " 2 1 0 1 1\n")
    with A.Context(0, autotune=True, tune_cache_path=str(path)) as ctx:
        got = A.agatha_align_batch(ctx, batch)
    idx = np.unique(np.concatenate([np.argsort(-(batch.q_len.astype(np.int64) + batch.t_len))[:4],
                                    np.random.default_rng(9).choice(batch.n_pairs, 60, replace=False)]))
    ref = O.align_batch(batch, idx=idx)
    assert A.results_equal(got[idx], ref, O.COMPARE_FIELDS).size == 0


def test_malformed_cache_lines_are_ignored(tmp_path, batch):
    path = tmp_path / "tune.txt"
    path.write_text("garbage\n" + _key(batch.scoring, 16) + " 0 1 9 0 1\n"
                    + _key(batch.scoring, 16) + " 0 1 2 0 7\n")
    with A.Context(0, autotune=True, tune_cache_path=str(path)) as ctx:
        assert ctx.tune_variants(batch.scoring) is None


@pytest.fixture(scope="module")
def short_batch():
    B.build()
    return W.make_config("short", n_pairs=4000)


@pytest.mark.parametrize("variants,split", [((5, 5, 5, 5), 0), ((5, 1, 0, 5), 1), ((1, 5, 2, 5), 1)])
def test_half_warp_variant_is_exact(tmp_path, short_batch, variants, split):
    """Two pairs per warp (variant 5, the 4-slot band only), alone and beside
    other variants per length class, against the oracle on every pair."""
    path = tmp_path / "tune.txt"
    path.write_text(_key(short_batch.scoring, 4) + " " + " ".join(map(str, variants)) + f" {split}\n")
    ref = O.align_batch(short_batch)
    with A.Context(0, autotune=True, tune_cache_path=str(path)) as ctx:
        assert ctx.tune_variants(short_batch.scoring) == list(variants) + [split]
        got = A.agatha_align_batch(ctx, short_batch)
    assert A.results_equal(got, ref, O.COMPARE_FIELDS).size == 0


def test_half_warp_variant_not_taken_for_wider_bands(tmp_path, batch, reference):
    # a cache entry naming it for a 16-slot band falls back to the default plan
    path = tmp_path / "tune.txt"
    path.write_text(_key(batch.scoring, 16) + " 5 5 5 5 0\n")
    with A.Context(0, autotune=True, tune_cache_path=str(path)) as ctx:
        assert A.results_equal(A.agatha_align_batch(ctx, batch), reference).size == 0
