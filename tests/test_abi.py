"""CPU checks of the C ABI: the library loads, exports every declared symbol,
and its host-only entry points (packing, parameter checks) behave."""
import os
import re
import subprocess

import numpy as np
import pytest

from paper_2403_06478_gb300 import agatha as A
from paper_2403_06478_gb300 import build as B
from paper_2403_06478_gb300 import workload as W

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "agatha.h")


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(agatha_\w+)\s*\(", text)))


def test_header_declares_the_abi():
    names = declared_functions()
    for n in ("agatha_init", "agatha_align_batch", "agatha_destroy", "agatha_serve_start",
              "agatha_serve_submit", "agatha_serve_wait", "agatha_serve_stop", "agatha_pack_codes"):
        assert n in names


def test_library_exports_every_declared_symbol():
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT (agatha_\w+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    # the binding wraps exactly the declared functions
    assert sorted(A.declared_symbols()) == declared_functions()


def test_library_loads_and_binds():
    L = A.lib()
    assert L.agatha_version() >= 100
    assert L.agatha_strerror(A.AGATHA_EINVAL) == b"invalid argument"


@pytest.mark.parametrize("n", [0, 1, 15, 16, 17, 1000, 33333])
def test_pack_codes_layout(n):
    rng = np.random.default_rng(n)
    codes = rng.integers(0, 4, n).astype(np.uint8)
    words = A.agatha_pack_codes(codes)
    assert words.shape[0] == max(1, (n + 15) // 16)
    # base k at bits 2*(k%16) of word k/16
    k = np.arange(n)
    unpacked = (words[k // 16] >> (2 * (k % 16)).astype(np.uint32)) & 3
    assert np.array_equal(unpacked.astype(np.uint8), codes)
    if n % 16:
        assert words[-1] >> np.uint32(2 * (n % 16)) == 0


def test_pack_large_uses_threads_and_matches():
    rng = np.random.default_rng(1)
    codes = rng.integers(0, 4, (1 << 20) * 16 + 5).astype(np.uint8)
    words = A.agatha_pack_codes(codes)
    k = np.arange(0, codes.shape[0], 9973)
    assert np.array_equal(((words[k // 16] >> (2 * (k % 16)).astype(np.uint32)) & 3).astype(np.uint8), codes[k])


def test_pack_rejects_bad_codes_and_letters():
    with pytest.raises(A.AgathaError) as e:
        A.agatha_pack_codes(np.array([0, 1, 4], np.uint8))
    assert e.value.code == A.AGATHA_EINVAL
    with pytest.raises(A.AgathaError):
        A.agatha_pack_ascii(b"ACGTN")
    w = A.agatha_pack_ascii(b"ACGTacgt")
    assert w[0] == sum(c << (2 * i) for i, c in enumerate([0, 1, 2, 3, 0, 1, 2, 3]))


def test_check_params_normalises_and_rejects():
    p = A.agatha_check_params(W.Scoring(2, 4, 4, 2, 24, 1, 500, 400, 0))
    assert (p.q2, p.e2) == (24, 1)
    p = A.agatha_check_params(W.Scoring(2, 4, 4, 2, 3, 1, 500, 400, 0))    # q2 <= q
    assert (p.q2, p.e2) == (4, 2)
    p = A.agatha_check_params(W.Scoring(2, 4, 4, 2, 30, 2, 500, 400, 0))   # e2 >= e
    assert (p.q2, p.e2) == (4, 2)
    for bad in (W.Scoring(w=0), W.Scoring(b=-1), W.Scoring(e2=-1), W.Scoring(a=-2)):
        with pytest.raises(A.AgathaError) as e:
            A.agatha_check_params(bad)
        assert e.value.code == A.AGATHA_EINVAL


def _band_cells_ref(tlen, qlen, w):
    if tlen <= 0 or qlen <= 0:
        return 0
    if w < 0 or w > max(tlen, qlen):
        w = max(tlen, qlen)
    return sum(1 for t in range(tlen) for q in range(qlen) if abs(t - q) <= w)


@pytest.mark.parametrize("tl,ql,w", [(0, 5, 3), (5, 5, 1), (7, 30, 4), (30, 7, 4), (50, 50, -1),
                                      (100, 60, 20), (1, 1, 1)])
def test_band_cells(tl, ql, w):
    assert A.agatha_band_cells(tl, ql, w) == _band_cells_ref(tl, ql, w)


def test_noalloc_rejects_null_streams_on_the_host():
    # host-side checks only: these calls return before any CUDA call, so they
    # run without a GPU (the pointer values are never dereferenced)
    for qp, tp in ((None, 16), (16, None)):
        with pytest.raises(A.AgathaError) as e:
            A.agatha_align_batch_noalloc(qp, tp, 8, 8, 8, 8, 8, W.ONT_SCORING, n_pairs=1,
                                         words=(4, 4))
        assert e.value.code == A.AGATHA_EINVAL
    with pytest.raises(A.AgathaError) as e:
        A.agatha_align_batch_noalloc(16, 16, 8, 8, 8, 8, 8, W.ONT_SCORING,
                                     n_pairs=A.AGATHA_NOALLOC_MAX_PAIRS + 1, words=(4, 4))
    assert e.value.code == A.AGATHA_EINVAL
