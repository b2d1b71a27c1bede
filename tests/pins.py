"""Independent reference computations used to pin the CPU oracle.

Nothing here is imported by the oracle or by the CUDA library.  Each routine
reaches the same quantity by a different road than the oracle's anti-diagonal
streaming loop:

* ``brute_force_H`` enumerates every alignment path from the origin and scores
  each maximal gap run with the two-piece cost, so it knows nothing of the
  E/F/E2/F2 recurrence (paper Section 2.1, Eq. 1-3).
* ``gotoh_unbanded`` is the textbook row-major affine-gap table without band.
* ``banded_table_H`` fills the band row by row (row-major, not by anti-diagonal).
* ``scan_antidiagonals`` applies the termination rule (Eq. 4-7) to any complete
  table of H values, one anti-diagonal after the other.
"""
from __future__ import annotations

import sys
from typing import Dict, Optional, Tuple

NEG_OUT = -0x40000000
MINUS_INF = float("-inf")


def normalise(p: Dict) -> Dict:
    p = dict(p)
    if p["q2"] <= p["q"] or p["e2"] >= p["e"]:
        p["q2"], p["e2"] = p["q"], p["e"]
    return p


def gap(p: Dict, l: int) -> int:
    return min(p["q"] + l * p["e"], p["q2"] + l * p["e2"])


def eff_w(p: Dict, tlen: int, qlen: int) -> int:
    w = p["w"]
    if w < 0 or w > max(tlen, qlen):
        w = max(tlen, qlen)
    return w


def brute_force_H(T, Q, p: Dict) -> Dict[Tuple[int, int], int]:
    """Best score of every band cell by enumerating all paths (tiny inputs only).

    A path starts at the origin (-1,-1) and moves by M (both indices +1, scores
    the substitution of the cell it enters), D (t+1) or I (q+1).  Cells with
    t == -1 or q == -1 are the virtual edge and may be visited freely; every
    real cell on the path must satisfy |t - q| <= w.  A maximal run of D moves
    (or of I moves) is one gap of that length.
    """
    p = normalise(p)
    tlen, qlen = len(T), len(Q)
    w = eff_w(p, tlen, qlen)
    best: Dict[Tuple[int, int], int] = {}
    sys.setrecursionlimit(10000)

    def ok(t, q):
        if t >= tlen or q >= qlen:
            return False
        if t < 0 or q < 0:
            return True            # virtual edge cell
        return abs(t - q) <= w

    def visit(t, q, closed, run_dir, run_len):
        score = closed - (gap(p, run_len) if run_len else 0)
        if t >= 0 and q >= 0:
            if score > best.get((t, q), MINUS_INF):
                best[(t, q)] = score
        # M: closes any open run
        if ok(t + 1, q + 1) and t + 1 >= 0 and q + 1 >= 0:
            s = p["a"] if T[t + 1] == Q[q + 1] else -p["b"]
            visit(t + 1, q + 1, score + s, None, 0)
        for d, (dt, dq) in (("D", (1, 0)), ("I", (0, 1))):
            nt, nq = t + dt, q + dq
            if not ok(nt, nq):
                continue
            if run_dir == d:
                visit(nt, nq, closed, d, run_len + 1)
            else:
                visit(nt, nq, score, d, 1)

    visit(-1, -1, 0, None, 0)
    return best


def gotoh_unbanded(T, Q, p: Dict):
    """Textbook two-piece affine global alignment table, row-major, no band.

    Returns the full H table as a list of lists (H[t][q]).
    """
    p = normalise(p)
    n, m = len(T), len(Q)
    NEG = -10 ** 12
    # row -1 / column -1 are leading gaps
    H = [[NEG] * (m + 1) for _ in range(n + 1)]
    E = [[NEG] * (m + 1) for _ in range(n + 1)]    # ends with a step in t
    E2 = [[NEG] * (m + 1) for _ in range(n + 1)]
    F = [[NEG] * (m + 1) for _ in range(n + 1)]    # ends with a step in q
    F2 = [[NEG] * (m + 1) for _ in range(n + 1)]
    H[0][0] = 0
    for j in range(1, m + 1):
        H[0][j] = -gap(p, j)
    for i in range(1, n + 1):
        H[i][0] = -gap(p, i)
    for i in range(1, n + 1):
        for j in range(1, m + 1):
            E[i][j] = max(H[i - 1][j] - p["q"] - p["e"], E[i - 1][j] - p["e"])
            E2[i][j] = max(H[i - 1][j] - p["q2"] - p["e2"], E2[i - 1][j] - p["e2"])
            F[i][j] = max(H[i][j - 1] - p["q"] - p["e"], F[i][j - 1] - p["e"])
            F2[i][j] = max(H[i][j - 1] - p["q2"] - p["e2"], F2[i][j - 1] - p["e2"])
            s = p["a"] if T[i - 1] == Q[j - 1] else -p["b"]
            H[i][j] = max(H[i - 1][j - 1] + s, E[i][j], F[i][j], E2[i][j], F2[i][j])
    return [[H[i + 1][j + 1] for j in range(m)] for i in range(n)]


def banded_table_H(T, Q, p: Dict) -> Dict[Tuple[int, int], int]:
    """Band cells filled row by row (t outer, q inner)."""
    p = normalise(p)
    tlen, qlen = len(T), len(Q)
    w = eff_w(p, tlen, qlen)
    H: Dict[Tuple[int, int], int] = {}
    E: Dict[Tuple[int, int], float] = {}
    E2: Dict[Tuple[int, int], float] = {}
    for t in range(tlen):
        lo, hi = max(0, t - w), min(qlen - 1, t + w)
        f = f2 = MINUS_INF
        for q in range(lo, hi + 1):
            # F from the left neighbour (t, q-1)
            if q == lo:
                h_left = -gap(p, t + 1) if q == 0 else MINUS_INF
                f_prev = f2_prev = MINUS_INF
            else:
                h_left, f_prev, f2_prev = H[(t, q - 1)], f, f2
            f = max(h_left - p["q"] - p["e"], f_prev - p["e"])
            f2 = max(h_left - p["q2"] - p["e2"], f2_prev - p["e2"])
            # E from the cell above
            if t == 0:
                h_up, e_up, e2_up = -gap(p, q + 1), MINUS_INF, MINUS_INF
            elif (t - 1, q) in H:
                h_up, e_up, e2_up = H[(t - 1, q)], E[(t - 1, q)], E2[(t - 1, q)]
            else:
                h_up = e_up = e2_up = MINUS_INF
            e = max(h_up - p["q"] - p["e"], e_up - p["e"])
            e2 = max(h_up - p["q2"] - p["e2"], e2_up - p["e2"])
            if t == 0 and q == 0:
                h_diag = 0
            elif t == 0:
                h_diag = -gap(p, q)
            elif q == 0:
                h_diag = -gap(p, t)
            else:
                h_diag = H[(t - 1, q - 1)]
            s = p["a"] if T[t] == Q[q] else -p["b"]
            h = max(h_diag + s, e, f, e2, f2)
            H[(t, q)] = h
            E[(t, q)] = e
            E2[(t, q)] = e2
    return H


def scan_antidiagonals(H: Dict[Tuple[int, int], int], tlen: int, qlen: int,
                       p: Dict) -> Dict:
    """Apply the exact termination rule to a complete table of band H values."""
    p = normalise(p)
    res = dict(max=0, qe=-1, te=-1, gscore=NEG_OUT, mqe=NEG_OUT, mqe_t=-1,
               mte=NEG_OUT, mte_q=-1, cells=0, zdropped=0, reach_end=0)
    if tlen == 0 or qlen == 0:
        return res
    gmax, gt, gq = 0, -1, -1
    mqe = mte = None
    zdropped = 0
    last = tlen + qlen - 2
    for r in range(last + 1):
        ts = [t for t in range(tlen) if (t, r - t) in H]
        if not ts:
            zdropped = 1
            break
        res["cells"] += len(ts)
        m, mt = None, None
        for t in ts:                          # ascending t: keep the first maximum
            if m is None or H[(t, r - t)] > m:
                m, mt = H[(t, r - t)], t
        if (tlen - 1, r - tlen + 1) in H:
            v = H[(tlen - 1, r - tlen + 1)]
            if mte is None or v > mte:
                mte, res["mte_q"] = v, r - tlen + 1
        if (r - qlen + 1, qlen - 1) in H:
            v = H[(r - qlen + 1, qlen - 1)]
            if mqe is None or v > mqe:
                mqe, res["mqe_t"] = v, r - qlen + 1
        mq = r - mt
        if m > gmax:
            gmax, gt, gq = m, mt, mq
        elif mt >= gt and mq >= gq and p["zdrop"] >= 0:
            l = abs((mt - gt) - (mq - gq))
            if gmax - m > p["zdrop"] + l * p["e2"]:
                zdropped = 1
                break
        if r == last and (tlen - 1, qlen - 1) in H:
            res["gscore"] = H[(tlen - 1, qlen - 1)]
    res.update(max=gmax, te=gt, qe=gq, zdropped=zdropped)
    if mqe is not None:
        res["mqe"] = mqe
    if mte is not None:
        res["mte"] = mte
    res["reach_end"] = int(not zdropped and mqe is not None and mqe + p["end_bonus"] > gmax)
    return res


def reference_result(T, Q, p: Dict, method: str = "brute") -> Dict:
    if method == "brute":
        H = brute_force_H(T, Q, p)
    elif method == "banded":
        H = banded_table_H(T, Q, p)
    else:
        raise ValueError(method)
    return scan_antidiagonals(H, len(T), len(Q), p)


def cigar_score(ops, T, Q, p: Dict, end_t: int, end_q: int) -> int:
    """Score of an alignment given as CIGAR runs ((length << 4) | op, op
    M=0, I=1, D=2), checked for validity along the way.

    The path starts at the origin (-1,-1); it must end at (end_t, end_q),
    visit only band cells once both indices are >= 0, and use maximal runs
    (no two adjacent runs of one op).  Each run of I or D is one gap, scored
    with the two-piece cost; M scores the substitution of the cell it enters.
    Knows nothing of the E/F/E2/F2 recurrence or of the traceback rule.
    """
    p = normalise(p)
    w = eff_w(p, len(T), len(Q))
    t = q = -1
    score = 0
    prev = None
    for x in ops:
        n, op = int(x) >> 4, int(x) & 15
        assert n >= 1 and op in (0, 1, 2), f"bad run {x:#x}"
        assert op != prev, "adjacent runs of one op"
        prev = op
        if op == 0:
            for _ in range(n):
                t += 1
                q += 1
                score += p["a"] if T[t] == Q[q] else -p["b"]
                assert abs(t - q) <= w, f"({t},{q}) outside the band"
        else:
            for _ in range(n):
                if op == 1:
                    q += 1
                else:
                    t += 1
                if t >= 0 and q >= 0:
                    assert abs(t - q) <= w, f"({t},{q}) outside the band"
            score -= gap(p, n)
        assert t < len(T) and q < len(Q), "path leaves the table"
    assert (t, q) == (end_t, end_q), f"path ends at ({t},{q}), not ({end_t},{end_q})"
    return score


# --------------------------------------------------------------------------
# The local extension from an initial score (the BWA-MEM variant)
# --------------------------------------------------------------------------

def brute_force_H_local(T, Q, p: Dict, h0: int) -> Dict[Tuple[int, int], int]:
    """Best score of every band cell over the paths that start at the origin
    with score h0 and whose score is positive after every move (tiny inputs).

    Moves and gap costs are those of ``brute_force_H``; a path whose score
    reaches zero or below is dropped, so a cell no path reaches is absent.
    Knows nothing of the E/F/E2/F2 recurrence or of its floors at zero.
    """
    p = normalise(p)
    tlen, qlen = len(T), len(Q)
    w = eff_w(p, tlen, qlen)
    best: Dict[Tuple[int, int], int] = {}
    sys.setrecursionlimit(10000)

    def ok(t, q):
        if t >= tlen or q >= qlen:
            return False
        if t < 0 or q < 0:
            return True
        return abs(t - q) <= w

    def visit(t, q, closed, run_dir, run_len):
        score = closed - (gap(p, run_len) if run_len else 0)
        if score <= 0:
            return
        if t >= 0 and q >= 0 and score > best.get((t, q), MINUS_INF):
            best[(t, q)] = score
        if ok(t + 1, q + 1) and t + 1 >= 0 and q + 1 >= 0:
            s = p["a"] if T[t + 1] == Q[q + 1] else -p["b"]
            visit(t + 1, q + 1, score + s, None, 0)
        for d, (dt, dq) in (("D", (1, 0)), ("I", (0, 1))):
            nt, nq = t + dt, q + dq
            if not ok(nt, nq):
                continue
            if run_dir == d:
                visit(nt, nq, closed, d, run_len + 1)
            else:
                visit(nt, nq, score, d, 1)

    visit(-1, -1, h0, None, 0)
    return best


def scan_rows_local(H: Dict[Tuple[int, int], int], tlen: int, qlen: int, p: Dict,
                    h0: int) -> Dict:
    """Apply the local variant's row-by-row rules (one query position at a
    time) to a table of positive band scores (absent: no live path)."""
    p = normalise(p)
    res = dict(max=h0, qe=-1, te=-1, gscore=NEG_OUT, mqe=NEG_OUT, mqe_t=-1,
               mte=NEG_OUT, mte_q=-1, cells=0, zdropped=0, reach_end=0)
    if tlen == 0 or qlen == 0:
        return res
    w = eff_w(p, tlen, qlen)
    best, bt, bq = h0, -1, -1
    mqe = mte = None
    zdropped = 0
    for q in range(qlen):
        ts = [t for t in range(tlen) if abs(t - q) <= w]
        if not ts:
            zdropped = 1
            break
        res["cells"] += len(ts)
        row, rt = 0, -1
        for t in ts:                        # ascending t: the first of equal maxima
            v = H.get((t, q), 0)
            if v > row:
                row, rt = v, t
        v = H.get((tlen - 1, q), 0)
        if ts[-1] == tlen - 1 and v > 0 and (mte is None or v > mte):
            mte, res["mte_q"] = v, q
        if q == qlen - 1 and row > 0:
            mqe, res["mqe_t"] = row, rt
        if row == 0:
            zdropped = 1
            break
        if row > best:
            best, bt, bq = row, rt, q
        elif p["zdrop"] >= 0:
            l = abs((q - bq) - (rt - bt))
            if best - row > p["zdrop"] + l * p["e2"]:
                zdropped = 1
                break
        if q == qlen - 1 and ts[-1] == tlen - 1 and v > 0:
            res["gscore"] = v
    res.update(max=best, te=bt, qe=bq, zdropped=zdropped)
    if mqe is not None:
        res["mqe"] = mqe
    if mte is not None:
        res["mte"] = mte
    res["reach_end"] = int(not zdropped and mqe is not None and mqe + p["end_bonus"] > best)
    return res
