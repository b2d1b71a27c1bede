"""Pins of the oracle's traceback (the CIGAR of an extension).

* hand-derived cases (tests/golden/traceback_cases.txt) fix the tie rule;
* every path it returns is checked for validity and re-scored run by run
  (pins.cigar_score), and that score must equal the brute-force optimum over
  all paths to the same cell (pins.brute_force_H) on tiny inputs, and the
  score oracle's max / mqe on larger ones;
* planted mistakes in the traceback code are caught by these cases.
"""
import ctypes
import os
import subprocess
import tempfile

import numpy as np
import pytest

import pins
from oracle import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "traceback_cases.txt")
ENC = {"A": 0, "C": 1, "G": 2, "T": 3}
KEYS = ("a", "b", "q", "e", "q2", "e2", "w", "zdrop", "end_bonus")


def _codes(s):
    return np.array([ENC[c] for c in s], np.uint8)


def _cases():
    out = []
    with open(GOLDEN) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            cid, T, Q, ps, end, exp = line.split("|")
            p = dict(zip(KEYS, (int(x) for x in ps.split())))
            cig, score = exp.split()
            out.append((cid, T, Q, p, end, cig, int(score)))
    return out


def _scoring(p):
    return tuple(p[k] for k in KEYS)


def _end(T, Q, p, end):
    if end == "ext":
        r = oracle.align_pair(T, Q, _scoring(p))
        return oracle.end_cell(r, len(Q))
    t, q = end.split(",")
    return int(t), int(q)


@pytest.mark.parametrize("case", _cases(), ids=lambda c: c[0])
def test_hand_traceback_cases(case):
    cid, T, Q, p, end, cig, score = case
    T, Q = _codes(T), _codes(Q)
    et, eq = _end(T, Q, p, end)
    ops, sc = oracle.traceback_pair(T, Q, _scoring(p), et, eq)
    assert oracle.cigar_string(ops) == cig
    assert sc == score
    assert pins.cigar_score(ops, T, Q, p, et, eq) == score


PSETS = [
    dict(a=2, b=4, q=4, e=2, q2=24, e2=1, w=3, zdrop=-1, end_bonus=0),
    dict(a=2, b=3, q=2, e=3, q2=5, e2=1, w=2, zdrop=-1, end_bonus=0),
    dict(a=3, b=2, q=4, e=4, q2=6, e2=1, w=1, zdrop=-1, end_bonus=0),
    dict(a=2, b=1, q=0, e=1, q2=3, e2=0, w=5, zdrop=-1, end_bonus=0),
    dict(a=1, b=1, q=0, e=1, q2=0, e2=1, w=-1, zdrop=-1, end_bonus=0),
    dict(a=2, b=4, q=4, e=2, q2=24, e2=1, w=-1, zdrop=-1, end_bonus=0),
]


@pytest.mark.parametrize("pi", range(len(PSETS)))
def test_traceback_is_optimal_to_every_band_cell(pi):
    """For every band cell of tiny random pairs, the returned path is valid and
    its run-by-run score equals the best over all paths to that cell."""
    p = PSETS[pi]
    rng = np.random.default_rng(900 + pi)
    for k in range(12):
        alphabet = 2 if k % 2 else 4
        T = rng.integers(0, alphabet, int(rng.integers(1, 6))).astype(np.uint8)
        Q = rng.integers(0, alphabet, int(rng.integers(1, 6))).astype(np.uint8)
        best = pins.brute_force_H(list(T), list(Q), p)
        for (et, eq), h in best.items():
            ops, sc = oracle.traceback_pair(T, Q, _scoring(p), et, eq)
            assert sc == h, (T, Q, et, eq)
            assert pins.cigar_score(ops, T, Q, p, et, eq) == h, (T, Q, et, eq, oracle.cigar_string(ops))


def test_empty_and_out_of_band_end_cells():
    T, Q = _codes("ACGTACGT"), _codes("ACGT")
    p = dict(a=2, b=4, q=4, e=2, q2=4, e2=2, w=2, zdrop=-1, end_bonus=0)
    ops, sc = oracle.traceback_pair(T, Q, _scoring(p), -1, -1)
    assert ops.size == 0 and sc == 0
    with pytest.raises(ValueError):
        oracle.traceback_pair(T, Q, _scoring(p), 7, 3)        # |t - q| = 4 > w
    with pytest.raises(ValueError):
        oracle.traceback_pair(T, Q, _scoring(p), 8, 3)        # outside the table


SCORINGS = [
    (2, 4, 4, 2, 24, 1, 50, 400, 0),       # two-piece, Z-drop on
    (1, 2, 2, 1, 32, 0, 40, 100, 5),       # two-piece with end bonus
    (2, 4, 4, 2, 4, 2, 30, -1, 0),         # single piece, no Z-drop
    (5, 30, 40, 3, 80, 1, 60, 200, 0),     # steep penalties
]


@pytest.mark.parametrize("si", range(len(SCORINGS)))
def test_extension_traceback_scores_match_score_oracle(si):
    """Random pairs with indels: the path to the extension's end cell scores
    exactly the score oracle's max (or mqe when the query end was reached)."""
    sc = SCORINGS[si]
    p = dict(zip(KEYS, sc))
    rng = np.random.default_rng(77 + si)
    for _ in range(20):
        n = int(rng.integers(20, 300))
        T = rng.integers(0, 4, n).astype(np.uint8)
        Q = []
        for b in T:                                   # ~8% substitutions / indels
            u = rng.random()
            if u < 0.04:
                Q.append((b + 1) % 4)
            elif u < 0.06:
                continue
            elif u < 0.08:
                Q.extend([b, int(rng.integers(0, 4))])
            else:
                Q.append(b)
        Q = np.array(Q[: int(rng.integers(10, len(Q) + 1))], np.uint8)
        r = oracle.align_pair(T, Q, sc)
        et, eq = oracle.end_cell(r, len(Q))
        ops, h = oracle.traceback_pair(T, Q, sc, et, eq)
        want = int(r["mqe"]) if r["reach_end"] else int(r["max"])
        assert h == want
        if et >= 0:
            assert pins.cigar_score(ops, T, Q, p, et, eq) == want


# ---------------------------------------------------------------- mutants

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "oracle", "agatha_oracle.c")

MUTANTS = {
    "tie_prefers_last_source": ("if (cand[k] > cand[src]) src = k;",
                                "if (cand[k] >= cand[src]) src = k;"),
    "leading_insertions_short": ("orc_push(&runs, ORC_OP_I, (uint32_t)(q + 1));",
                                 "orc_push(&runs, ORC_OP_I, (uint32_t)q);"),
    "leading_deletions_short": ("orc_push(&runs, ORC_OP_D, (uint32_t)(t + 1));",
                                "orc_push(&runs, ORC_OP_D, (uint32_t)t);"),
    "insertion_as_deletion": ("orc_push(&runs, ORC_OP_I, 1);", "orc_push(&runs, ORC_OP_D, 1);"),
    "e_reads_f_bit": ("const int extended = (st == S_E) ? (d & 8) : (d & 32);",
                      "const int extended = (st == S_E) ? (d & 16) : (d & 32);"),
    "f2_reads_f_bit": ("const int extended = (st == S_F) ? (d & 16) : (d & 64);",
                       "const int extended = (st == S_F) ? (d & 16) : (d & 16);"),
    "no_reverse": ("for (int64_t i = 0; i < n / 2; ++i) {", "for (int64_t i = 0; i < 0; ++i) {"),
    "diag_from_above": ("else Hdiag = row_prev[q - 1].H;", "else Hdiag = row_prev[q].H;"),
    "e_opens_with_e2": ("int64_t open = Hup - p.q - p.e, ext = Eup - p.e;",
                        "int64_t open = Hup - p.q2 - p.e2, ext = Eup - p.e;"),
}


def _compile(src_text, d):
    src = os.path.join(d, "m.c")
    lib = os.path.join(d, "m.so")
    with open(src, "w") as fh:
        fh.write(src_text)
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-pthread", src, "-o", lib])
    L = ctypes.CDLL(lib)
    L.orc_traceback_pair.restype = ctypes.c_int64
    L.orc_traceback_pair.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32,
                                     ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                     ctypes.c_int64, ctypes.c_void_p]
    L.orc_normalise.argtypes = [ctypes.c_void_p]
    return L


def _tb(L, T, Q, p, et, eq):
    par = (ctypes.c_int32 * 9)(*[p[k] for k in KEYS])
    L.orc_normalise(par)
    cap = len(T) + len(Q) + 2
    ops = np.zeros(cap, np.uint32)
    score = ctypes.c_int64(0)
    n = L.orc_traceback_pair(T.ctypes.data, len(T), Q.ctypes.data, len(Q), par, et, eq,
                             ops.ctypes.data, cap, ctypes.byref(score))
    return (tuple(ops[:max(n, 0)]), int(score.value), int(n))


def _mutant_corpus():
    """(T, Q, p, end cell, expected ops or None, expected score)."""
    cases = []
    for cid, T, Q, p, end, cig, score in _cases():
        T, Q = _codes(T), _codes(Q)
        et, eq = _end(T, Q, p, end)
        ops, _ = oracle.traceback_pair(T, Q, _scoring(p), et, eq)
        assert oracle.cigar_string(ops) == cig
        cases.append((T, Q, p, et, eq, ops, score))
    rng = np.random.default_rng(31)
    for p in PSETS:
        for k in range(6):
            T = rng.integers(0, 2 + 2 * (k % 2), int(rng.integers(2, 6))).astype(np.uint8)
            Q = rng.integers(0, 2 + 2 * (k % 2), int(rng.integers(2, 6))).astype(np.uint8)
            for (et, eq), h in pins.brute_force_H(list(T), list(Q), p).items():
                cases.append((T, Q, p, et, eq, None, h))
    return cases


def _caught(L, case):
    T, Q, p, et, eq, ops, score = case
    got_ops, got_score, n = _tb(L, T, Q, p, et, eq)
    if n < 0 or got_score != score:
        return True
    if ops is not None and got_ops != tuple(ops):
        return True
    try:
        return pins.cigar_score(got_ops, T, Q, p, et, eq) != score
    except AssertionError:
        return True


@pytest.fixture(scope="module")
def mutant_corpus():
    return _mutant_corpus()


def test_unmutated_traceback_passes_corpus(mutant_corpus):
    with tempfile.TemporaryDirectory() as d:
        L = _compile(open(SRC).read(), d)
        assert not any(_caught(L, c) for c in mutant_corpus)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_traceback_mutant_is_caught(name, mutant_corpus):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not found exactly once"
    with tempfile.TemporaryDirectory() as d:
        L = _compile(src.replace(old, new), d)
        assert any(_caught(L, c) for c in mutant_corpus), f"planted mistake {name!r} not caught"
