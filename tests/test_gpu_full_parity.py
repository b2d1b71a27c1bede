"""Every pair of the full-size ONT-like, HiFi-like and skewed batches against
the CPU oracle, in the launch configuration the benchmark times (an
autotuned context, one host batch per call).

The oracle's results on these batches are stored as digests
(``tests/golden/full_batch_oracle.txt``, written by
``tests/golden/full_batch_digests.py``, which calls only the oracle and the
input generator): the library's results must give the same digest for every
chunk of 1,000 pairs.  A chunk that differs is recomputed by the oracle here
to name its pairs.  If the seeded inputs on this machine differ from those the
digests were written for (the input digest tells), the oracle aligns the whole
batch here, on all host cores, and every pair is compared directly.

Tolerance 0: every output is an integer.
"""
import numpy as np
import pytest

from golden import full_batch_digests as G
from oracle import oracle as O
from paper_2403_06478_gb300 import agatha as A
from paper_2403_06478_gb300 import build as B
from paper_2403_06478_gb300 import workload as W

pytestmark = pytest.mark.gpu

FIELDS = O.COMPARE_FIELDS
GOLDEN = G.read_golden()


@pytest.fixture(scope="module")
def tuned_ctx():
    B.build()
    c = A.Context(0, autotune=True)
    yield c
    c.close()


def _first_difference(got, ref, batch, idx, label):
    bad = A.results_equal(got, ref, FIELDS)
    if bad.size == 0:
        return
    i = int(bad[0])
    p = int(idx[i])
    diff = {f: (int(got[i][f]), int(ref[i][f])) for f in FIELDS if got[i][f] != ref[i][f]}
    raise AssertionError(f"{label}: {bad.size} of {got.shape[0]} pairs differ from the oracle; "
                         f"first pair {p} (tlen={int(batch.t_len[p])}, qlen={int(batch.q_len[p])}) "
                         f"got/expected: {diff}")


@pytest.mark.parametrize("name", ["ont", "hifi", "skewed"])
def test_every_pair_matches_the_oracle(tuned_ctx, name):
    batch = W.make_config(name)
    got = A.agatha_align_batch(tuned_ctx, batch)
    rec = GOLDEN.get(name)
    if rec is None or G.input_digest(batch) != rec["input"]:
        # inputs differ from the stored ones: the oracle aligns the whole batch here
        ref = O.align_batch(batch)
        _first_difference(got, ref, batch, np.arange(batch.n_pairs), f"{name}/live oracle")
        return
    assert got.shape[0] == rec["n_pairs"]
    chunks = G.chunk_digests(got, rec["chunk"])
    bad = [k for k, (a, b) in enumerate(zip(chunks, rec["chunks"])) if a != b]
    for k in bad[:3]:
        idx = np.arange(k * rec["chunk"], min((k + 1) * rec["chunk"], batch.n_pairs))
        ref = O.align_batch(batch, idx=idx)
        _first_difference(got[idx], ref, batch, idx, f"{name}/chunk {k}")
    assert not bad, f"{name}: chunks {bad[:10]} differ from the oracle's digests"
    assert G.result_digest(got) == rec["result"]
    assert int(got["cells"].sum()) == rec["cells"]
    assert int(got["zdropped"].sum()) == rec["zdropped"]
