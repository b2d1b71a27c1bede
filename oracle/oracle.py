"""Python access to the CPU oracle (``agatha_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by the
benchmark's CPU-baseline leg.  The product library never loads it.

Every function here marshals arguments; the arithmetic is in the C file, which
restates the paper's recurrence (Section 2.1, Eq. 1-3, two-piece extension) and
termination rule (Eq. 4-7), and the traceback of an extension.  Results are
numpy structured arrays with the same fields as the library's result struct.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "agatha_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")

OUT_NEG_INF = -0x40000000

RESULT_DTYPE = np.dtype([
    ("max", np.int32), ("qe", np.int32), ("te", np.int32), ("gscore", np.int32),
    ("mqe", np.int32), ("mqe_t", np.int32), ("mte", np.int32), ("mte_q", np.int32),
    ("cells", np.int64), ("zdropped", np.uint8), ("reach_end", np.uint8),
    ("pad", np.uint8, (6,)),
])
assert RESULT_DTYPE.itemsize == 48

COMPARE_FIELDS = ("max", "qe", "te", "gscore", "mqe", "mqe_t", "mte", "mte_q",
                  "cells", "zdropped", "reach_end")


class _Params(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in
                ("a", "b", "q", "e", "q2", "e2", "w", "zdrop", "end_bonus")]


_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with the host C compiler (portable flags only)."""
    with _lock:
        if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
            tmp = LIB + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O3", "-std=c11", "-fPIC", "-shared",
                                   "-pthread", SRC, "-o", tmp])
            os.replace(tmp, LIB)
    return LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(LIB)
        lib.orc_align_pair.restype = None
        lib.orc_align_pair.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                       ctypes.c_int32, ctypes.POINTER(_Params), ctypes.c_void_p]
        lib.orc_normalise.restype = None
        lib.orc_normalise.argtypes = [ctypes.POINTER(_Params)]
        lib.orc_align_batch.restype = ctypes.c_int
        lib.orc_align_batch.argtypes = [ctypes.c_void_p] * 7 + [
            ctypes.c_int64, ctypes.POINTER(_Params), ctypes.c_void_p, ctypes.c_int]
        lib.orc_align_pair_local.restype = None
        lib.orc_align_pair_local.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                             ctypes.c_int32, ctypes.POINTER(_Params), ctypes.c_int32,
                                             ctypes.c_void_p]
        lib.orc_align_batch_local.restype = ctypes.c_int
        lib.orc_align_batch_local.argtypes = [ctypes.c_void_p] * 7 + [
            ctypes.c_int64, ctypes.POINTER(_Params), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
        lib.orc_result_size.restype = ctypes.c_int
        lib.orc_traceback_pair.restype = ctypes.c_int64
        lib.orc_traceback_pair.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                           ctypes.c_int32, ctypes.POINTER(_Params), ctypes.c_int32,
                                           ctypes.c_int32, ctypes.c_void_p, ctypes.c_int64,
                                           ctypes.POINTER(ctypes.c_int64)]
        assert lib.orc_result_size() == RESULT_DTYPE.itemsize
        _lib = lib
    return _lib


def _params(scoring) -> _Params:
    t = scoring.as_tuple() if hasattr(scoring, "as_tuple") else tuple(scoring)
    return _Params(*[int(x) for x in t])


def align_pair(target: np.ndarray, query: np.ndarray, scoring) -> np.void:
    """Align one pair (codes 0..3); parameters are normalised first."""
    lib = _load()
    t = np.ascontiguousarray(target, dtype=np.uint8)
    q = np.ascontiguousarray(query, dtype=np.uint8)
    p = _params(scoring)
    lib.orc_normalise(ctypes.byref(p))
    out = np.zeros(1, dtype=RESULT_DTYPE)
    lib.orc_align_pair(t.ctypes.data, len(t), q.ctypes.data, len(q), ctypes.byref(p),
                       out.ctypes.data)
    return out[0]


def align_pair_local(target: np.ndarray, query: np.ndarray, scoring, h0: int) -> np.void:
    """Local extension of one pair from the initial score h0 (the BWA-MEM
    variant); parameters are normalised first."""
    lib = _load()
    t = np.ascontiguousarray(target, dtype=np.uint8)
    q = np.ascontiguousarray(query, dtype=np.uint8)
    p = _params(scoring)
    lib.orc_normalise(ctypes.byref(p))
    out = np.zeros(1, dtype=RESULT_DTYPE)
    lib.orc_align_pair_local(t.ctypes.data if len(t) else None, len(t),
                             q.ctypes.data if len(q) else None, len(q), ctypes.byref(p), int(h0),
                             out.ctypes.data)
    return out[0]


def align_batch(batch, idx: Optional[np.ndarray] = None, threads: Optional[int] = None,
                longest_first: bool = True, h0: Optional[np.ndarray] = None) -> np.ndarray:
    """Align every pair of ``batch`` (or the pairs ``idx``) on host threads;
    with ``h0`` (one initial score per pair of the batch) the local extension
    (the BWA-MEM variant) instead."""
    lib = _load()
    if idx is not None:
        idx = np.asarray(idx, dtype=np.int64)
        q_off = np.ascontiguousarray(batch.q_off[idx])
        t_off = np.ascontiguousarray(batch.t_off[idx])
        q_len = np.ascontiguousarray(batch.q_len[idx])
        t_len = np.ascontiguousarray(batch.t_len[idx])
    else:
        q_off, t_off, q_len, t_len = batch.q_off, batch.t_off, batch.q_len, batch.t_len
    q_off = np.ascontiguousarray(q_off, dtype=np.int64)
    t_off = np.ascontiguousarray(t_off, dtype=np.int64)
    q_len = np.ascontiguousarray(q_len, dtype=np.int32)
    t_len = np.ascontiguousarray(t_len, dtype=np.int32)
    n = int(q_len.shape[0])
    out = np.zeros(n, dtype=RESULT_DTYPE)
    if n == 0:
        return out
    order = None
    if longest_first:
        order = np.ascontiguousarray(np.argsort(-(q_len.astype(np.int64) + t_len), kind="stable"),
                                     dtype=np.int64)
    qc = np.ascontiguousarray(batch.q_codes, dtype=np.uint8)
    tc = np.ascontiguousarray(batch.t_codes, dtype=np.uint8)
    if qc.size == 0:
        qc = np.zeros(1, np.uint8)
    if tc.size == 0:
        tc = np.zeros(1, np.uint8)
    p = _params(batch.scoring)
    nt = threads if threads is not None else (os.cpu_count() or 1)
    if h0 is not None:
        h = np.asarray(h0, dtype=np.int32)
        h = np.ascontiguousarray(h[idx] if idx is not None else h)
        rc = lib.orc_align_batch_local(qc.ctypes.data, tc.ctypes.data, q_off.ctypes.data,
                                       t_off.ctypes.data, q_len.ctypes.data, t_len.ctypes.data,
                                       order.ctypes.data if order is not None else None,
                                       n, ctypes.byref(p), h.ctypes.data, out.ctypes.data, int(nt))
    else:
        rc = lib.orc_align_batch(qc.ctypes.data, tc.ctypes.data, q_off.ctypes.data,
                                 t_off.ctypes.data, q_len.ctypes.data, t_len.ctypes.data,
                                 order.ctypes.data if order is not None else None,
                                 n, ctypes.byref(p), out.ctypes.data, int(nt))
    if rc != 0:
        raise RuntimeError("oracle batch failed")
    return out


CIGAR_OPS = "MID"       # op codes 0, 1, 2 of a run (length << 4 | op)


def end_cell(result, qlen: int):
    """Where the traceback of an extension starts: the query end when the
    extension reached it (reach_end), else the cell of the maximum."""
    if result["reach_end"]:
        return int(result["mqe_t"]), int(qlen) - 1
    return int(result["te"]), int(result["qe"])


def traceback_pair(target: np.ndarray, query: np.ndarray, scoring, end_t: int, end_q: int):
    """Run-length encoded operations of the best path from the origin to
    (end_t, end_q), and H there (0 for an empty path)."""
    lib = _load()
    t = np.ascontiguousarray(target, dtype=np.uint8)
    q = np.ascontiguousarray(query, dtype=np.uint8)
    p = _params(scoring)
    lib.orc_normalise(ctypes.byref(p))
    cap = len(t) + len(q) + 2
    ops = np.zeros(cap, dtype=np.uint32)
    score = ctypes.c_int64(0)
    n = lib.orc_traceback_pair(t.ctypes.data if len(t) else None, len(t),
                               q.ctypes.data if len(q) else None, len(q), ctypes.byref(p),
                               int(end_t), int(end_q), ops.ctypes.data, cap, ctypes.byref(score))
    if n < 0:
        raise ValueError(f"no traceback to ({end_t}, {end_q})")
    return ops[:n].copy(), int(score.value)


def traceback_batch(batch, results, idx=None):
    """CIGAR runs of every pair (or of the pairs ``idx``), from the end cells
    the score oracle's ``results`` give.  Returns a list of uint32 arrays and
    the H value at each end cell."""
    idx = range(batch.n_pairs) if idx is None else idx
    cig, scores = [], []
    for i in idx:
        i = int(i)
        t = batch.t_codes[batch.t_off[i]:batch.t_off[i] + batch.t_len[i]]
        q = batch.q_codes[batch.q_off[i]:batch.q_off[i] + batch.q_len[i]]
        et, eq = end_cell(results[i], int(batch.q_len[i]))
        if batch.t_len[i] <= 0 or batch.q_len[i] <= 0:
            et = eq = -1
        ops, sc = traceback_pair(t, q, batch.scoring, et, eq)
        cig.append(ops)
        scores.append(sc)
    return cig, scores


def cigar_string(ops) -> str:
    return "".join(f"{int(x) >> 4}{CIGAR_OPS[int(x) & 15]}" for x in ops)


def band_cells_full(tlen: int, qlen: int, w: int) -> int:
    """Band cells of the whole table (no termination): the work estimate."""
    if tlen <= 0 or qlen <= 0:
        return 0
    if w < 0 or w > max(tlen, qlen):
        w = max(tlen, qlen)
    total = 0
    for t in range(tlen):
        lo = max(0, t - w)
        hi = min(qlen - 1, t + w)
        if hi >= lo:
            total += hi - lo + 1
    return total
