"""The pins must be strong enough to catch plausible mistakes in the oracle.

Each mutant is a copy of the oracle's C source with one planted mistake (a
dropped term, a wrong comparison, an off-by-one index, a transposed operand),
compiled into a temporary directory.  At least one pinned case must disagree
with it.  The mistakes are planted on the CPU only.
"""
import ctypes
import os
import subprocess
import tempfile

import numpy as np
import pytest

import pins
from oracle import oracle

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "oracle", "agatha_oracle.c")

MUTANTS = {
    "tie_highest_t": ("if (H > m) { m = H; m_t = t; }", "if (H >= m) { m = H; m_t = t; }"),
    "global_max_ge": ("if (m > gmax) {", "if (m >= gmax) {"),
    "zdrop_ge": ("if (gmax - m > (int64_t)p.zdrop + l * p.e2)",
                 "if (gmax - m >= (int64_t)p.zdrop + l * p.e2)"),
    "zdrop_uses_e": ("(int64_t)p.zdrop + l * p.e2", "(int64_t)p.zdrop + l * p.e"),
    "zdrop_no_quadrant": ("} else if (m_t >= gmax_t && m_q >= gmax_q && p.zdrop >= 0) {",
                          "} else if (p.zdrop >= 0) {"),
    "drop_E2": ("H = imax64(H, E2); H = imax64(H, F2);", "H = imax64(H, F2);"),
    "drop_F": ("H = imax64(H, E); H = imax64(H, F);", "H = imax64(H, E);"),
    "open_without_extend": ("int64_t E = imax64(Hup - p.q - p.e, Eup - p.e);",
                            "int64_t E = imax64(Hup - p.q, Eup - p.e);"),
    "edge_off_by_one": ("else if (t == 0) Hdiag = -gap_cost(&p, q);",
                        "else if (t == 0) Hdiag = -gap_cost(&p, q + 1);"),
    "left_edge_off_by_one": ("if (q == 0) { Hleft = -gap_cost(&p, t + 1);",
                             "if (q == 0) { Hleft = -gap_cost(&p, t);"),
    "band_floor": ("int64_t lo2 = lo >= 0 ? (lo + 1) / 2 : -((-lo) / 2);",
                   "int64_t lo2 = lo >= 0 ? lo / 2 : -((-lo + 1) / 2);"),
    "wrong_neighbour": ("Hup = prev1[t - 1].H; Eup = prev1[t - 1].E;",
                        "Hup = prev1[t].H; Eup = prev1[t - 1].E;"),
    "transposed_score": ("int64_t s = (T[t] == Q[q]) ? p.a : -(int64_t)p.b;",
                         "int64_t s = (T[t] == Q[q]) ? p.b : -(int64_t)p.a;"),
    "mte_ge": ("if (H > mte) { mte = H;", "if (H >= mte) { mte = H;"),
    "mqe_wrong_t": ("if (H > mqe) { mqe = H; mqe_t = tq; }", "if (H > mqe) { mqe = H; mqe_t = tq + 1; }"),
    "reach_end_ge": ("mqe + p.end_bonus > gmax", "mqe + p.end_bonus >= gmax"),
    "cells_off_by_one": ("cells += en - st + 1;", "cells += en - st;"),
    "no_band_stop": ("if (st > en) { zdropped = 1; break; }", "if (st > en) { break; }"),
    "e2_extends_with_e": ("int64_t E2 = imax64(Hup - p.q2 - p.e2, E2up - p.e2);",
                          "int64_t E2 = imax64(Hup - p.q2 - p.e2, E2up - p.e);"),
    "no_normalise": ("if (p->q2 <= p->q || p->e2 >= p->e) { p->q2 = p->q; p->e2 = p->e; }", ""),
}


def _compile(mutant_src, d):
    src = os.path.join(d, "m.c")
    lib = os.path.join(d, "m.so")
    with open(src, "w") as fh:
        fh.write(mutant_src)
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-pthread", src, "-o", lib])
    L = ctypes.CDLL(lib)
    L.orc_align_pair.restype = None
    L.orc_align_pair.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32,
                                 ctypes.c_void_p, ctypes.c_void_p]
    L.orc_normalise.argtypes = [ctypes.c_void_p]
    return L


def _run(L, T, Q, p):
    par = (ctypes.c_int32 * 9)(p["a"], p["b"], p["q"], p["e"], p["q2"], p["e2"], p["w"],
                               p["zdrop"], p["end_bonus"])
    L.orc_normalise(par)
    out = np.zeros(1, dtype=oracle.RESULT_DTYPE)
    T = np.ascontiguousarray(T, np.uint8)
    Q = np.ascontiguousarray(Q, np.uint8)
    L.orc_align_pair(T.ctypes.data, len(T), Q.ctypes.data, len(Q), par, out.ctypes.data)
    return {f: int(out[0][f]) for f in oracle.COMPARE_FIELDS}


def _corpus():
    """Pinned cases: inputs plus the result fixed by brute-force enumeration."""
    rng = np.random.default_rng(4242)
    psets = [
        dict(a=2, b=4, q=4, e=2, q2=24, e2=1, w=3, zdrop=5, end_bonus=0),
        dict(a=2, b=3, q=2, e=3, q2=5, e2=1, w=2, zdrop=1, end_bonus=0),
        dict(a=3, b=2, q=4, e=4, q2=6, e2=1, w=1, zdrop=0, end_bonus=0),
        dict(a=2, b=1, q=0, e=1, q2=3, e2=0, w=5, zdrop=4, end_bonus=3),
        dict(a=2, b=4, q=4, e=2, q2=24, e2=1, w=-1, zdrop=-1, end_bonus=0),
    ]
    cases = []
    for p in psets:
        for k in range(25):
            alphabet = 2 if k % 2 else 4
            T = rng.integers(0, alphabet, int(rng.integers(1, 7))).astype(np.uint8)
            Q = rng.integers(0, alphabet, int(rng.integers(1, 7))).astype(np.uint8)
            cases.append((T, Q, p, pins.reference_result(list(T), list(Q), p, "brute")))
    # targeted inputs: large mismatch penalty near the virtual edge, a band that
    # leaves the table, q2 < q (collapses to one piece), equal-score cells on one
    # anti-diagonal, and a two-piece drop whose best cell lies up-right of the max
    targeted = [
        ([0, 0, 1, 1, 0], [1], dict(a=3, b=2, q=0, e=1, q2=2, e2=0, w=2, zdrop=2, end_bonus=0)),
        ([0, 0], [0, 0, 0, 0, 0], dict(a=3, b=2, q=0, e=1, q2=2, e2=0, w=2, zdrop=2, end_bonus=0)),
        ([3, 0, 2, 1], [3, 1, 2], dict(a=2, b=4, q=4, e=2, q2=2, e2=1, w=2, zdrop=3, end_bonus=0)),
        ([0, 1, 1, 1], [1, 0, 1, 1], dict(a=1, b=1, q=1, e=1, q2=1, e2=1, w=4, zdrop=1, end_bonus=0)),
        ([0, 1, 0, 1, 0], [1, 1], dict(a=2, b=1, q=5, e=3, q2=6, e2=0, w=4, zdrop=4, end_bonus=0)),
    ]
    for T, Q, p in targeted:
        T = np.array(T, np.uint8)
        Q = np.array(Q, np.uint8)
        cases.append((T, Q, p, pins.reference_result(list(T), list(Q), p, "brute")))
    return cases


@pytest.fixture(scope="module")
def corpus():
    return _corpus()


def test_unmutated_oracle_passes_corpus(corpus):
    with tempfile.TemporaryDirectory() as d:
        L = _compile(open(SRC).read(), d)
        for T, Q, p, ref in corpus:
            assert _run(L, T, Q, p) == ref


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, corpus):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    # the mistakes are planted in the score path (orc_align_pair), ahead of
    # the local variant and the traceback (which repeat some of its lines)
    cut = src.index("Local extension from an initial score")
    head, tail = src[:cut], src[cut:]
    assert head.count(old) == 1, f"mutation site for {name} not found exactly once"
    with tempfile.TemporaryDirectory() as d:
        L = _compile(head.replace(old, new) + tail, d)
        caught = any(_run(L, T, Q, p) != ref for T, Q, p, ref in corpus)
    assert caught, f"planted mistake {name!r} is not caught by any pinned case"
