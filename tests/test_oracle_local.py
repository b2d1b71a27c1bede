"""Pins of the oracle's local extension from an initial score (the BWA-MEM
variant, paper Section 5.9; the rules are this build's reading of BWA-MEM's
published extension: positive-score paths from h0, row-by-row Z-drop, the
end-bonus clipping choice).

- brute force: every path from the origin with score h0 whose score stays
  positive after each move, scored run by run, then the row rules applied
  by independent code (tests/pins.py);
- closed forms (identical sequences, an extension that dies at once);
- with an initial score too large for any path to reach zero and no Z-drop,
  every score is the global method's plus h0;
- planted mistakes in a copy of the oracle, each caught by a pinned case.
"""
import ctypes
import os
import subprocess
import tempfile

import numpy as np
import pytest

import pins
from oracle import oracle as O
from paper_2403_06478_gb300 import workload as W

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "agatha_oracle.c")
FIELDS = O.COMPARE_FIELDS

PSETS = [
    dict(a=1, b=4, q=6, e=1, q2=6, e2=1, w=3, zdrop=5, end_bonus=5),       # BWA-MEM's scoring
    dict(a=2, b=4, q=4, e=2, q2=24, e2=1, w=2, zdrop=4, end_bonus=0),     # two-piece
    dict(a=3, b=2, q=1, e=1, q2=3, e2=0, w=4, zdrop=0, end_bonus=2),      # zdrop 0, free second piece
    dict(a=2, b=5, q=3, e=2, q2=3, e2=2, w=1, zdrop=-1, end_bonus=0),     # narrow band, no Z-drop
    dict(a=1, b=1, q=0, e=1, q2=2, e2=0, w=-1, zdrop=3, end_bonus=1),     # unbanded
]


def _local(T, Q, p, h0):
    sc = W.Scoring(**p)
    r = O.align_pair_local(np.array(T, np.uint8), np.array(Q, np.uint8), sc, h0)
    return {f: int(r[f]) for f in FIELDS}


def _brute(T, Q, p, h0):
    return pins.scan_rows_local(pins.brute_force_H_local(list(T), list(Q), p, h0), len(T), len(Q), p, h0)


def _corpus():
    rng = np.random.default_rng(5959)
    cases = []
    for p in PSETS:
        for k in range(22):
            alphabet = 2 if k % 2 else 4
            T = rng.integers(0, alphabet, int(rng.integers(1, 7))).astype(np.uint8)
            Q = rng.integers(0, alphabet, int(rng.integers(1, 7))).astype(np.uint8)
            h0 = int(rng.choice([1, 2, 4, 7, 12, 30]))
            cases.append((T, Q, p, h0))
    # targeted: an extension that dies on its first row, a dead diagonal next
    # to a live gap, ties along a row, a band that leaves the table
    cases += [
        (np.array([1, 0, 0], np.uint8), np.array([0, 0, 0], np.uint8), PSETS[0], 3),
        (np.array([0, 1, 1, 1], np.uint8), np.array([1, 1, 1], np.uint8), PSETS[0], 8),
        (np.array([0, 0, 0, 0], np.uint8), np.array([0, 0], np.uint8), PSETS[2], 2),
        (np.array([0, 0], np.uint8), np.array([0, 0, 0, 0, 0, 0], np.uint8), PSETS[3], 9),
        (np.array([2, 3, 2, 3, 2], np.uint8), np.array([3, 2, 3], np.uint8), PSETS[1], 5),
    ]
    return [(T, Q, p, h0, _brute(T, Q, p, h0)) for T, Q, p, h0 in cases]


@pytest.fixture(scope="module")
def corpus():
    return _corpus()


def test_local_oracle_matches_brute_force(corpus):
    for T, Q, p, h0, ref in corpus:
        assert _local(T, Q, p, h0) == ref, (list(T), list(Q), p, h0)


def test_corpus_exercises_each_rule(corpus):
    refs = [c[4] for c in corpus]
    assert any(r["zdropped"] and r["qe"] == -1 for r in refs)        # died on the first row
    assert any(r["zdropped"] and r["qe"] >= 0 for r in refs)         # Z-drop or a dead row later
    assert any(r["reach_end"] for r in refs)
    assert any(not r["zdropped"] and not r["reach_end"] for r in refs)


@pytest.mark.parametrize("n", [1, 5, 40])
def test_identical_sequences(n):
    rng = np.random.default_rng(n)
    x = rng.integers(0, 4, n).astype(np.uint8)
    p = dict(PSETS[0], w=10, zdrop=100)
    r = _local(x, x, p, 7)
    assert (r["max"], r["te"], r["qe"], r["gscore"], r["mqe"], r["mqe_t"]) == (
        7 + n, n - 1, n - 1, 7 + n, 7 + n, n - 1)
    assert r["zdropped"] == 0 and r["reach_end"] == 1         # mqe = max, end bonus 5 > 0


def test_extension_that_dies_at_once():
    # first bases differ, h0 below the mismatch penalty and every gap's cost:
    # no live cell on row 0
    p = dict(PSETS[0], w=5, zdrop=100)
    T = np.array([1, 0, 0, 0], np.uint8)
    Q = np.array([0, 0, 0, 0], np.uint8)
    r = _local(T, Q, p, 3)
    assert (r["max"], r["qe"], r["te"], r["zdropped"], r["gscore"], r["mqe"]) == (3, -1, -1, 1, O.OUT_NEG_INF, O.OUT_NEG_INF)
    assert r["cells"] == 4                                      # row 0: t = 0..3


@pytest.mark.parametrize("seed", range(6))
def test_large_h0_reduces_to_the_global_method(seed):
    # no path can reach zero, no Z-drop: every score is h0 more than the
    # global method's, over the same cells (row order and anti-diagonal
    # order then agree on values; their tie-breaks may pick other cells)
    rng = np.random.default_rng(seed)
    sc = W.Scoring(2, 4, 4, 2, 24, 1, int(rng.integers(3, 40)), -1, 0)
    n = int(rng.integers(20, 120))
    Q = rng.integers(0, 4, n).astype(np.uint8)
    T = rng.integers(0, 4, n + int(rng.integers(-2, 3))).astype(np.uint8)
    h0 = 10 ** 6
    a = O.align_pair_local(T, Q, sc, h0)
    g = O.align_pair(T, Q, sc)
    assert int(a["max"]) == h0 + int(g["max"])
    assert int(a["gscore"]) == h0 + int(g["gscore"])
    assert int(a["mqe"]) == h0 + int(g["mqe"]) and int(a["mte"]) == h0 + int(g["mte"])
    assert int(a["cells"]) == int(g["cells"]) and a["zdropped"] == g["zdropped"] == 0


LOCAL_MUTANTS = {
    "zdrop_uses_e": ("(int64_t)p.zdrop + l * p.e2) { zdropped = 1; break; }",
                     "(int64_t)p.zdrop + l * p.e) { zdropped = 1; break; }"),
    "revive_dead_diagonal": ("int64_t H = Hdiag > 0 ? pos64(Hdiag + s) : 0;", "int64_t H = pos64(Hdiag + s);"),
    "row_tie_highest_t": ("if (H > row_best) { row_best = H; row_t = t; }",
                          "if (H >= row_best && H > 0) { row_best = H; row_t = t; }"),
    "no_dead_row_stop": ("if (row_best == 0) { zdropped = 1; break; }", "if (row_best == 0) { break; }"),
    "zdrop_without_l": ("if (gmax - row_best > (int64_t)p.zdrop + l * p.e2)",
                        "if (gmax - row_best > (int64_t)p.zdrop)"),
    "origin_zero": ("if (t == 0 && q == 0) Hdiag = h0;", "if (t == 0 && q == 0) Hdiag = 0;"),
    "gscore_before_last_row": ("if (q == qlen - 1 && hi == tlen - 1 && cur[tlen - 1].H > 0) gscore",
                               "if (hi == tlen - 1 && cur[tlen - 1].H > 0) gscore"),
    "mqe_from_last_column": ("if (q == qlen - 1 && row_best > 0) { mqe = row_best; mqe_t = row_t; }",
                             "if (hi == tlen - 1 && row_best > 0 && row_best > mqe) { mqe = row_best; mqe_t = row_t; }"),
    "max_ge": ("if (row_best > gmax) {", "if (row_best >= gmax) {"),
    "left_from_this_row": ("Hleft = prev[t].H; Fleft = prev[t].F; F2left = prev[t].F2;",
                           "Hleft = cur[t].H; Fleft = prev[t].F; F2left = prev[t].F2;"),
}


def _compile(src, d):
    path = os.path.join(d, "m.c")
    lib = os.path.join(d, "m.so")
    with open(path, "w") as fh:
        fh.write(src)
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-pthread", path, "-o", lib])
    L = ctypes.CDLL(lib)
    L.orc_align_pair_local.restype = None
    L.orc_align_pair_local.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32,
                                       ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p]
    L.orc_normalise.argtypes = [ctypes.c_void_p]
    return L


def _run(L, T, Q, p, h0):
    par = (ctypes.c_int32 * 9)(p["a"], p["b"], p["q"], p["e"], p["q2"], p["e2"], p["w"], p["zdrop"],
                               p["end_bonus"])
    L.orc_normalise(par)
    out = np.zeros(1, dtype=O.RESULT_DTYPE)
    T = np.ascontiguousarray(T, np.uint8)
    Q = np.ascontiguousarray(Q, np.uint8)
    L.orc_align_pair_local(T.ctypes.data, len(T), Q.ctypes.data, len(Q), par, int(h0), out.ctypes.data)
    return {f: int(out[0][f]) for f in FIELDS}


@pytest.mark.parametrize("name", sorted(LOCAL_MUTANTS))
def test_local_mutant_is_caught(name, corpus):
    old, new = LOCAL_MUTANTS[name]
    src = open(SRC).read()
    a = src.index("Local extension from an initial score")
    b = src.index("Batch driver")
    region = src[a:b]
    assert region.count(old) == 1, f"mutation site for {name} not found exactly once"
    with tempfile.TemporaryDirectory() as d:
        L = _compile(src[:a] + region.replace(old, new) + src[b:], d)
        caught = any(_run(L, T, Q, p, h0) != ref for T, Q, p, h0, ref in corpus)
    assert caught, f"planted mistake {name!r} is not caught by any pinned case"
