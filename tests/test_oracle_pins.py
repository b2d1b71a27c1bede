"""Pins for the CPU oracle: it must agree with computations that reach the same
answer by a different road (brute force over alignment paths, the textbook
unbanded Gotoh table, a row-major banded table) and with hand-derived and
closed-form results (paper Section 2.1, Eq. 1-7)."""
import itertools
import os

import numpy as np
import pytest

import pins
from oracle import oracle
from paper_2403_06478_gb300 import workload as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hand_cases.txt")
FIELDS = oracle.COMPARE_FIELDS


def _params(a, b, q, e, q2, e2, w, zdrop, end_bonus=0):
    return dict(a=a, b=b, q=q, e=e, q2=q2, e2=e2, w=w, zdrop=zdrop, end_bonus=end_bonus)


def _tuple(p):
    return (p["a"], p["b"], p["q"], p["e"], p["q2"], p["e2"], p["w"], p["zdrop"], p["end_bonus"])


def _codes(s):
    return np.array(["ACGT".index(c) for c in s], dtype=np.uint8)


def _oracle(T, Q, p):
    r = oracle.align_pair(T, Q, _tuple(p))
    return {f: int(r[f]) for f in FIELDS}


def _load_golden():
    cases = []
    with open(GOLDEN) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            cid, T, Q, par, exp = line.split("|")
            p = _params(*[int(x) for x in par.split()])
            expected = {k: int(v) for k, v in (kv.split("=") for kv in exp.split())}
            cases.append((cid, T, Q, p, expected))
    return cases


# ------------------------------------------------------------------ golden

@pytest.mark.parametrize("case", _load_golden(), ids=lambda c: c[0])
def test_hand_derived_cases(case):
    cid, T, Q, p, expected = case
    got = _oracle(_codes(T), _codes(Q), p)
    for k, v in expected.items():
        assert got[k] == v, (cid, k, got)


@pytest.mark.parametrize("case", _load_golden(), ids=lambda c: c[0])
def test_hand_cases_agree_with_brute_force(case):
    # the hand derivations themselves are checked by path enumeration
    cid, T, Q, p, expected = case
    ref = pins.reference_result(list(_codes(T)), list(_codes(Q)), p, "brute")
    for k, v in expected.items():
        assert ref[k] == v, (cid, k, ref)


# ------------------------------------------------------------ brute force

PARAM_SETS = [
    _params(2, 4, 4, 2, 24, 1, 3, 5),      # minimap2 ONT-like, tight band, small zdrop
    _params(2, 4, 2, 2, 2, 2, 2, 3),       # paper's example scoring (single piece)
    _params(1, 4, 6, 2, 26, 1, 4, 2),      # HiFi-like
    _params(2, 3, 2, 3, 5, 1, 2, 1),       # piece 2 wins from gap length 2
    _params(3, 2, 4, 4, 6, 1, 1, 0),       # piece 2 wins from length 1, w=1, zdrop 0
    _params(2, 4, 4, 2, 24, 1, -1, -1),    # unbanded, no termination
    _params(2, 1, 0, 1, 3, 0, 5, 4, 3),    # free gap open, end bonus
]


def _random_pairs(rng, n, max_len, alphabet=4):
    for _ in range(n):
        tl = int(rng.integers(0, max_len + 1))
        ql = int(rng.integers(0, max_len + 1))
        yield (rng.integers(0, alphabet, tl).astype(np.uint8),
               rng.integers(0, alphabet, ql).astype(np.uint8))


@pytest.mark.parametrize("pi", range(len(PARAM_SETS)))
def test_oracle_matches_brute_force(pi):
    p = PARAM_SETS[pi]
    rng = np.random.default_rng(1000 + pi)
    # two-letter alphabet: many ties, exercising the lowest-t and strict-> rules
    for T, Q in itertools.chain(_random_pairs(rng, 40, 6, 2), _random_pairs(rng, 40, 6, 4)):
        ref = pins.reference_result(list(T), list(Q), p, "brute")
        got = _oracle(T, Q, p)
        assert got == ref, (p, T.tolist(), Q.tolist(), got, ref)


def test_oracle_matches_brute_force_8x8():
    rng = np.random.default_rng(77)
    for p in (PARAM_SETS[0], PARAM_SETS[3]):
        for _ in range(2):
            T = rng.integers(0, 3, 8).astype(np.uint8)
            Q = T.copy()
            Q[rng.integers(0, 8)] = (Q[rng.integers(0, 8)] + 1) % 4
            ref = pins.reference_result(list(T), list(Q), p, "brute")
            assert _oracle(T, Q, p) == ref


# -------------------------------------------------- textbook Gotoh, no band

def test_unbanded_no_zdrop_matches_gotoh():
    rng = np.random.default_rng(5)
    for p in (_params(2, 4, 4, 2, 24, 1, -1, -1), _params(1, 4, 6, 2, 26, 1, -1, -1),
              _params(2, 4, 2, 2, 2, 2, -1, -1), _params(2, 3, 1, 3, 4, 1, -1, -1)):
        for _ in range(25):
            n = int(rng.integers(1, 40))
            T = rng.integers(0, 4, n).astype(np.uint8)
            if rng.random() < 0.5:
                Q = T[: int(rng.integers(1, n + 1))].copy()
                for _k in range(int(rng.integers(0, 4))):
                    Q[rng.integers(0, len(Q))] = rng.integers(0, 4)
            else:
                Q = rng.integers(0, 4, int(rng.integers(1, 40))).astype(np.uint8)
            H = pins.gotoh_unbanded(list(T), list(Q), p)
            got = _oracle(T, Q, p)
            assert got["gscore"] == H[len(T) - 1][len(Q) - 1]
            # the global maximum over all cells, earliest anti-diagonal then lowest t
            best = (0, -1, -1)
            for r in range(len(T) + len(Q) - 1):
                for t in range(max(0, r - len(Q) + 1), min(len(T) - 1, r) + 1):
                    if H[t][r - t] > best[0]:
                        best = (H[t][r - t], t, r - t)
            assert (got["max"], got["te"], got["qe"]) == best
            assert got["zdropped"] == 0
            assert got["cells"] == len(T) * len(Q)


def test_long_gaps_use_second_piece():
    # a 30-base insertion: two-piece cost min(4+60, 24+30) = 54 (piece 2)
    rng = np.random.default_rng(9)
    T = rng.integers(0, 4, 60).astype(np.uint8)
    ins = rng.integers(0, 4, 30).astype(np.uint8)
    Q = np.concatenate([T[:30], ins, T[30:]])
    p = _params(2, 4, 4, 2, 24, 1, 40, -1)
    H = pins.gotoh_unbanded(list(T), list(Q), dict(p, w=-1))
    got = _oracle(T, Q, p)
    assert got["gscore"] == H[59][89] == 2 * 60 - 54


# ----------------------------------------------- row-major banded + Z-drop

@pytest.mark.parametrize("seed", range(6))
def test_streaming_matches_row_major_banded(seed):
    rng = np.random.default_rng(seed)
    p = [
        _params(2, 4, 4, 2, 24, 1, 8, 30),
        _params(1, 4, 6, 2, 26, 1, 12, 20),
        _params(2, 4, 4, 2, 24, 1, 5, -1),
        _params(2, 4, 2, 2, 2, 2, 3, 10),
        _params(2, 4, 4, 2, 24, 1, 20, 50, 10),
        _params(2, 3, 2, 3, 5, 1, 6, 12),
    ][seed]
    b = W.random_pairs(rng, 30, 120, W.Scoring(*_tuple(p)), min_len=0, related=0.7)
    for i in range(b.n_pairs):
        T, Q = b.target(i), b.query(i)
        ref = pins.reference_result(list(T), list(Q), p, "banded")
        assert _oracle(T, Q, p) == ref, (i, p)


# ----------------------------------------------------------- closed forms

@pytest.mark.parametrize("n", [1, 2, 17, 300, 1000])
def test_identical_sequences_score_a_times_len(n):
    rng = np.random.default_rng(n)
    T = rng.integers(0, 4, n).astype(np.uint8)
    for a in (1, 2):
        p = _params(a, 4, 4, 2, 24, 1, 100, 400)
        got = _oracle(T, T, p)
        assert got["max"] == a * n and got["gscore"] == a * n
        assert got["te"] == n - 1 and got["qe"] == n - 1
        assert got["zdropped"] == 0


@pytest.mark.parametrize("pos", [0, 5, 150, 299])
def test_single_substitution(pos):
    rng = np.random.default_rng(pos)
    n = 300
    T = rng.integers(0, 4, n).astype(np.uint8)
    Q = T.copy()
    Q[pos] = (Q[pos] + 1) % 4
    p = _params(2, 4, 4, 2, 24, 1, 50, 400)
    assert _oracle(T, Q, p)["gscore"] == 2 * (n - 1) - 4


@pytest.mark.parametrize("l", [1, 2, 5, 19, 20, 21, 40])
def test_single_insertion_gap_cost(l):
    # Q has l extra bases, so any alignment pays for >= l inserted bases and
    # scores at most n matches; gap cost is subadditive, so one run is cheapest:
    # the optimum is exactly a*n - min(q + l*e, q2 + l*e2) when w >= l.
    rng = np.random.default_rng(100 + l)
    n = 400
    T = rng.integers(0, 4, n).astype(np.uint8)
    ins = rng.integers(0, 4, l).astype(np.uint8)
    Q = np.concatenate([T[:200], ins, T[200:]])
    p = _params(2, 4, 4, 2, 24, 1, 60, -1)
    assert _oracle(T, Q, p)["gscore"] == 2 * n - min(4 + 2 * l, 24 + l)
    assert _oracle(Q, T, p)["gscore"] == 2 * n - min(4 + 2 * l, 24 + l)


def test_unrelated_sequences_trigger_zdrop():
    rng = np.random.default_rng(3)
    T = rng.integers(0, 4, 5000).astype(np.uint8)
    Q = rng.integers(0, 4, 5000).astype(np.uint8)
    got = _oracle(T, Q, _params(2, 4, 4, 2, 24, 1, 500, 400))
    assert got["zdropped"] == 1
    assert got["cells"] < 5000 * 1001


def test_empty_inputs():
    p = _params(2, 4, 4, 2, 24, 1, 10, 100)
    for T, Q in ((np.zeros(0, np.uint8), np.zeros(0, np.uint8)),
                 (np.zeros(0, np.uint8), np.ones(5, np.uint8)),
                 (np.ones(5, np.uint8), np.zeros(0, np.uint8))):
        got = _oracle(T, Q, p)
        assert got == dict(max=0, qe=-1, te=-1, gscore=pins.NEG_OUT, mqe=pins.NEG_OUT,
                           mqe_t=-1, mte=pins.NEG_OUT, mte_q=-1, cells=0,
                           zdropped=0, reach_end=0)


# -------------------------------------------------------------- invariants

def _small_batch(seed, n=20, max_len=300):
    rng = np.random.default_rng(seed)
    return W.random_pairs(rng, n, max_len, W.ONT_SCORING, min_len=1, related=0.8)


def test_zdrop_off_equals_infinite_zdrop():
    b = _small_batch(1)
    for i in range(b.n_pairs):
        T, Q = b.target(i), b.query(i)
        x = _oracle(T, Q, _params(2, 4, 4, 2, 24, 1, 50, -1))
        y = _oracle(T, Q, _params(2, 4, 4, 2, 24, 1, 50, 1 << 28))
        assert x == y


def test_full_band_equals_unbanded():
    b = _small_batch(2)
    for i in range(b.n_pairs):
        T, Q = b.target(i), b.query(i)
        wide = max(len(T), len(Q))
        for z in (-1, 100):
            x = _oracle(T, Q, _params(2, 4, 4, 2, 24, 1, wide, z))
            y = _oracle(T, Q, _params(2, 4, 4, 2, 24, 1, -1, z))
            assert x == y


def test_cells_non_decreasing_in_w_without_zdrop():
    b = _small_batch(3)
    for i in range(b.n_pairs):
        T, Q = b.target(i), b.query(i)
        prev = -1
        for w in (1, 2, 5, 10, 40, 400):
            c = _oracle(T, Q, _params(2, 4, 4, 2, 24, 1, w, -1))["cells"]
            assert c >= prev
            prev = c


def test_two_piece_collapses_when_second_piece_never_cheaper():
    b = _small_batch(4)
    for i in range(b.n_pairs):
        T, Q = b.target(i), b.query(i)
        x = _oracle(T, Q, _params(2, 4, 4, 2, 4, 2, 50, 100))
        y = _oracle(T, Q, _params(2, 4, 4, 2, 3, 1, 50, 100))     # q2 <= q: collapses
        z = _oracle(T, Q, _params(2, 4, 4, 2, 30, 2, 50, 100))    # e2 >= e: collapses
        assert x == y == z


def test_batch_driver_matches_single_calls_any_thread_count():
    b = _small_batch(5, n=30)
    ref = [_oracle(b.target(i), b.query(i), dict(zip(
        ("a", "b", "q", "e", "q2", "e2", "w", "zdrop", "end_bonus"), b.scoring.as_tuple())))
        for i in range(b.n_pairs)]
    for threads in (1, 3, 8):
        out = oracle.align_batch(b, threads=threads)
        for i in range(b.n_pairs):
            assert {f: int(out[i][f]) for f in FIELDS} == ref[i]
    sub = oracle.align_batch(b, idx=[4, 2, 9])
    assert {f: int(sub[1][f]) for f in FIELDS} == ref[2]
