"""The allocation-free entry point against the regular one, through the C ABI.

agatha_align_batch_noalloc serves callers that cannot let the library call
cudaMalloc/cudaFree (hosts that reserve all device memory up front, or that
cannot afford the device-wide synchronisation of cudaFree).  It keeps its
scratch in a fixed device array shared by every call, so two calls in a row
on different batches must each reproduce the regular entry point exactly:
the second call must not see anything the first one left in the array.
This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_2403_06478_gb300 import agatha as A
from paper_2403_06478_gb300 import build as B
from paper_2403_06478_gb300 import workload as W

pytestmark = pytest.mark.gpu


def _device_batch(torch, batch):
    pb = A.pack_batch(batch)
    dev = {k: torch.from_numpy(getattr(pb, k)).cuda() for k in
           ("q_packed", "t_packed", "q_off", "t_off", "q_len", "t_len")}
    return pb, dev


def _regular(ctx, dev, scoring, n, torch):
    out = torch.zeros(n * 48, dtype=torch.uint8, device="cuda")
    ctx.align_device(dev["q_packed"], dev["t_packed"], dev["q_off"], dev["t_off"], dev["q_len"],
                     dev["t_len"], out, scoring)
    return out.cpu().numpy().view(A.RESULT_DTYPE).copy()


def _noalloc(dev, scoring, n, torch):
    out = torch.full((n * 48,), 0xAB, dtype=torch.uint8, device="cuda")
    A.agatha_align_batch_noalloc(dev["q_packed"], dev["t_packed"], dev["q_off"], dev["t_off"],
                                 dev["q_len"], dev["t_len"], out, scoring)
    torch.cuda.synchronize()
    return out.cpu().numpy().view(A.RESULT_DTYPE).copy()


def test_noalloc_matches_regular_entry_point_on_two_calls_in_a_row():
    torch = pytest.importorskip("torch")
    B.build()
    first = W.make_config("ont", n_pairs=600)
    second = W.make_config("small", n_pairs=200)
    with A.Context(0) as ctx:
        expected = []
        for batch in (first, second):
            pb, dev = _device_batch(torch, batch)
            expected.append((batch, dev, _regular(ctx, dev, batch.scoring, pb.n_pairs, torch)))
    for batch, dev, ref in expected:
        got = _noalloc(dev, batch.scoring, batch.n_pairs, torch)
        # integer results: the tolerance is exact equality, as in every parity test
        bad = A.results_equal(got, ref)
        assert bad.size == 0, (batch.name, bad[:10])
        assert int(got["cells"].sum()) == int(ref["cells"].sum()) > 0


@pytest.mark.parametrize("w", [750, 1000, -1, 1500])
def test_noalloc_wide_bands_match_regular_entry_point(w):
    # w = 750 and 1000 run the 24- and 32-slot warp kernels; w = -1 (unbanded)
    # and w = 1500 send every pair through the plain block kernel's list in the
    # scratch array, whose counter must restart at zero on every call
    torch = pytest.importorskip("torch")
    B.build()
    batch = W.make_config("ont", n_pairs=600).with_scoring(w=w)
    # unbanded and w = 1500 pairs go to the plain kernel, whose band (shared
    # memory) holds about 4,600 slots: keep the tables below that
    lens = np.maximum(batch.q_len, batch.t_len)
    batch = batch.subset(np.flatnonzero(lens <= 3000)[:200])
    pb, dev = _device_batch(torch, batch)
    with A.Context(0) as ctx:
        ref = _regular(ctx, dev, batch.scoring, pb.n_pairs, torch)
    for _ in range(2):
        got = _noalloc(dev, batch.scoring, batch.n_pairs, torch)
        bad = A.results_equal(got, ref)
        assert bad.size == 0, (w, bad[:10])


def test_noalloc_reports_a_pair_outside_its_stream():
    torch = pytest.importorskip("torch")
    B.build()
    batch = W.make_config("small", n_pairs=64)
    pb, dev = _device_batch(torch, batch)
    with A.Context(0) as ctx:
        ref = _regular(ctx, dev, batch.scoring, pb.n_pairs, torch)
    bad_off = dev["t_off"].clone()
    bad_off[5] = int(pb.t_packed.shape[0]) * 16 + 100      # past the end of the target stream
    out = torch.full((pb.n_pairs * 48,), 0xAB, dtype=torch.uint8, device="cuda")
    with pytest.raises(A.AgathaError) as e:
        A.agatha_align_batch_noalloc(dev["q_packed"], dev["t_packed"], dev["q_off"], bad_off,
                                     dev["q_len"], dev["t_len"], out, batch.scoring)
    assert e.value.code == A.AGATHA_EINVAL
    got = out.cpu().numpy().view(A.RESULT_DTYPE).copy()
    r = got[5]
    assert (r["max"], r["qe"], r["te"], r["gscore"], r["cells"], r["zdropped"]) == (
        0, -1, -1, A.NEG_INF, 0, 0)
    keep = np.arange(pb.n_pairs) != 5
    assert A.results_equal(got[keep], ref[keep]).size == 0
    # the next call on good input is unaffected by the error the last one left
    got = _noalloc(dev, batch.scoring, batch.n_pairs, torch)
    assert A.results_equal(got, ref).size == 0


def test_noalloc_rejects_batches_over_its_limit():
    torch = pytest.importorskip("torch")
    B.build()
    with pytest.raises(A.AgathaError) as e:
        A.agatha_align_batch_noalloc(None, None, None, None, None, None, None, W.ONT_SCORING,
                                     n_pairs=A.AGATHA_NOALLOC_MAX_PAIRS + 1)
    assert e.value.code == A.AGATHA_EINVAL
    assert torch.cuda.is_available()
