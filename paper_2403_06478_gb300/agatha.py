"""Python binding of ``libagatha.so`` (ctypes).  Argument marshalling only.

Every name mirrors the C ABI in ``include/agatha.h``: ``agatha_init``,
``agatha_align_batch``, ``agatha_pack_codes`` ...  The alignment itself runs
in the library's CUDA kernels; this module never computes a score.  If the
library is missing the import of a function fails loudly; there is no
fallback of any kind.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libagatha.so")

AGATHA_OK = 0
AGATHA_EINVAL = -1
AGATHA_ENOMEM = -2
AGATHA_ECUDA = -3
AGATHA_ETIMEDOUT = -4
AGATHA_EAGAIN = -5
AGATHA_ECANCELED = -6
AGATHA_EDEVICE = -7
AGATHA_ENOTSUP = -8
AGATHA_ERANGE = -9

AGATHA_HOST_PTRS = 0x00
AGATHA_DEVICE_PTRS = 0x01
AGATHA_PLAIN = 0x02
AGATHA_ASYNC = 0x04
AGATHA_NO_SORT = 0x08
AGATHA_FORCE32 = 0x10
AGATHA_NO_GRAPH = 0x20
AGATHA_EDGE_PATH_ONLY = 0x40
AGATHA_REGS_HIGH = 0x80
AGATHA_NO_TUNE = 0x100
AGATHA_TB_TWO_PASS = 0x200
AGATHA_WARPS2 = 0x400
AGATHA_WARPS4 = 0x800
AGATHA_HALF_WARP = 0x1000
AGATHA_ONE_FRAME = 0x2000

AGATHA_CFG_TIMING = 0x1
AGATHA_CFG_AUTOTUNE = 0x2

# CIGAR run op codes ((length << 4) | op)
AGATHA_CIGAR_M = 0
AGATHA_CIGAR_I = 1
AGATHA_CIGAR_D = 2
CIGAR_OPS = "MID"

# kernel variants the autotuner chooses between, per length class
VARIANT_NAMES = ("int16x2", "int16x2-highreg", "int32", "int16x2-2warps", "int16x2-4warps",
                 "int16x2-halfwarp")

NEG_INF = -0x40000000

RESULT_DTYPE = np.dtype([
    ("max", np.int32), ("qe", np.int32), ("te", np.int32), ("gscore", np.int32),
    ("mqe", np.int32), ("mqe_t", np.int32), ("mte", np.int32), ("mte_q", np.int32),
    ("cells", np.int64), ("zdropped", np.uint8), ("reach_end", np.uint8),
    ("lane16", np.uint8), ("pad", np.uint8, (5,)),
])
assert RESULT_DTYPE.itemsize == 48

RESULT_FIELDS = ("max", "qe", "te", "gscore", "mqe", "mqe_t", "mte", "mte_q", "cells",
                 "zdropped", "reach_end")


class AgathaError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{msg} (code {code})")
        self.code = code


class agatha_params(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in
                ("a", "b", "q", "e", "q2", "e2", "w", "zdrop", "end_bonus")]


class agatha_batch(ctypes.Structure):
    _fields_ = [("n_pairs", ctypes.c_int64),
                ("q_packed", ctypes.c_void_p), ("t_packed", ctypes.c_void_p),
                ("q_words", ctypes.c_int64), ("t_words", ctypes.c_int64),
                ("q_off", ctypes.c_void_p), ("t_off", ctypes.c_void_p),
                ("q_len", ctypes.c_void_p), ("t_len", ctypes.c_void_p)]


class agatha_config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("mem_budget_bytes", ctypes.c_int64), ("max_pairs", ctypes.c_int64),
                ("tune_cache_path", ctypes.c_char_p)]


class agatha_serve_config(ctypes.Structure):
    _fields_ = [("mem_budget_bytes", ctypes.c_int64), ("max_inflight", ctypes.c_int32),
                ("max_batch_pairs", ctypes.c_int32), ("linger_us", ctypes.c_int32),
                ("launch_flags", ctypes.c_uint32)]


class agatha_serve_stats(ctypes.Structure):
    _fields_ = [("requests_done", ctypes.c_int64), ("pairs_done", ctypes.c_int64),
                ("cells_done", ctypes.c_int64), ("launches", ctypes.c_int64),
                ("bytes_in_flight", ctypes.c_int64), ("peak_bytes_in_flight", ctypes.c_int64),
                ("busy_seconds", ctypes.c_double), ("p50_latency_ms", ctypes.c_double),
                ("p99_latency_ms", ctypes.c_double), ("max_launches_in_flight", ctypes.c_int64),
                ("max_device_concurrency", ctypes.c_int64), ("overlap_seconds", ctypes.c_double)]


class agatha_tb_info(ctypes.Structure):
    _fields_ = [("pairs16", ctypes.c_int64), ("pairs32", ctypes.c_int64), ("waves", ctypes.c_int64),
                ("fused", ctypes.c_int64)]


_lib = None

# every function the header declares, with its ctypes signature
_SIGS = {
    "agatha_init": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(agatha_config)]),
    "agatha_destroy": (None, [ctypes.c_void_p]),
    "agatha_align_batch": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(agatha_batch),
                                          ctypes.POINTER(agatha_params), ctypes.c_void_p,
                                          ctypes.c_uint32, ctypes.c_void_p]),
    "agatha_align_batch_local": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(agatha_batch),
                                                ctypes.POINTER(agatha_params), ctypes.c_void_p,
                                                ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p]),
    "agatha_check_params": (ctypes.c_int, [ctypes.POINTER(agatha_params), ctypes.POINTER(agatha_params)]),
    "agatha_pack_codes": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]),
    "agatha_pack_ascii": (ctypes.c_int, [ctypes.c_char_p, ctypes.c_int64, ctypes.c_void_p]),
    "agatha_band_cells": (ctypes.c_int64, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]),
    "agatha_last_kernel_ms": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_float)]),
    "agatha_align_batch_noalloc": (ctypes.c_int, [ctypes.POINTER(agatha_batch),
                                                  ctypes.POINTER(agatha_params), ctypes.c_void_p,
                                                  ctypes.c_void_p]),
    "agatha_serve_start": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(agatha_serve_config)]),
    "agatha_serve_submit": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(agatha_batch),
                                           ctypes.POINTER(agatha_params), ctypes.c_void_p,
                                           ctypes.POINTER(ctypes.c_uint64)]),
    "agatha_serve_poll": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64]),
    "agatha_serve_wait": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int32]),
    "agatha_serve_stats_get": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(agatha_serve_stats)]),
    "agatha_serve_stop": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    "agatha_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "agatha_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "agatha_version": (ctypes.c_int32, []),
    "agatha_tune_variants": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(agatha_params),
                                            ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]),
    "agatha_align_cigar": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(agatha_batch),
                                          ctypes.POINTER(agatha_params), ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                          ctypes.c_uint32, ctypes.c_void_p]),
    "agatha_last_traceback_ms": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_float)]),
    "agatha_last_traceback_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(agatha_tb_info)]),
}


def lib():
    """The loaded library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: run __graft_entry__.build() "
                              "(or python -m paper_2403_06478_gb300.build) first")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def declared_symbols():
    return tuple(_SIGS)


def _check(code: int, ctx=None, what: str = "agatha"):
    if code != AGATHA_OK:
        msg = lib().agatha_strerror(code).decode()
        if ctx is not None:
            detail = lib().agatha_last_error(ctx)
            if detail:
                msg += ": " + detail.decode()
        raise AgathaError(code, f"{what}: {msg}")


def make_params(scoring) -> agatha_params:
    t = scoring.as_tuple() if hasattr(scoring, "as_tuple") else tuple(scoring)
    return agatha_params(*[int(x) for x in t])


def agatha_check_params(scoring) -> agatha_params:
    out = agatha_params()
    _check(lib().agatha_check_params(ctypes.byref(make_params(scoring)), ctypes.byref(out)))
    return out


def agatha_band_cells(tlen: int, qlen: int, w: int) -> int:
    return int(lib().agatha_band_cells(int(tlen), int(qlen), int(w)))


def agatha_pack_codes(codes: np.ndarray) -> np.ndarray:
    """Pack codes 0..3 into 16-base uint32 words (runs in the library)."""
    codes = np.ascontiguousarray(codes, dtype=np.uint8)
    n = int(codes.shape[0])
    out = np.zeros(max(1, (n + 15) // 16), dtype=np.uint32)
    _check(lib().agatha_pack_codes(codes.ctypes.data if n else None, n, out.ctypes.data),
           what="agatha_pack_codes")
    return out


def agatha_pack_ascii(s: bytes) -> np.ndarray:
    n = len(s)
    out = np.zeros(max(1, (n + 15) // 16), dtype=np.uint32)
    _check(lib().agatha_pack_ascii(s, n, out.ctypes.data), what="agatha_pack_ascii")
    return out


@dataclass
class PackedBatch:
    """Host arrays of a batch in the library's input format."""
    q_packed: np.ndarray
    t_packed: np.ndarray
    q_off: np.ndarray
    t_off: np.ndarray
    q_len: np.ndarray
    t_len: np.ndarray

    @property
    def n_pairs(self) -> int:
        return int(self.q_len.shape[0])

    def nbytes(self) -> int:
        return sum(int(a.nbytes) for a in (self.q_packed, self.t_packed, self.q_off,
                                             self.t_off, self.q_len, self.t_len))


def pack_batch(batch) -> PackedBatch:
    """Pack a workload batch (concatenated codes) with the library's packer."""
    return PackedBatch(agatha_pack_codes(batch.q_codes), agatha_pack_codes(batch.t_codes),
                       np.ascontiguousarray(batch.q_off, dtype=np.int64),
                       np.ascontiguousarray(batch.t_off, dtype=np.int64),
                       np.ascontiguousarray(batch.q_len, dtype=np.int32),
                       np.ascontiguousarray(batch.t_len, dtype=np.int32))


def _host_batch(pb: PackedBatch) -> agatha_batch:
    return agatha_batch(pb.n_pairs, pb.q_packed.ctypes.data, pb.t_packed.ctypes.data,
                        int(pb.q_packed.shape[0]), int(pb.t_packed.shape[0]),
                        pb.q_off.ctypes.data, pb.t_off.ctypes.data,
                        pb.q_len.ctypes.data, pb.t_len.ctypes.data)


class Context:
    """An ``agatha_ctx`` on one device."""

    def __init__(self, device: int = 0, mem_budget_bytes: int = 0, max_pairs: int = 0,
                 tune_cache_path: Optional[str] = None, timing: bool = False,
                 autotune: bool = False):
        self._ptr = ctypes.c_void_p()
        flags = (AGATHA_CFG_TIMING if timing else 0) | (AGATHA_CFG_AUTOTUNE if autotune else 0)
        cfg = agatha_config(device, flags, mem_budget_bytes, max_pairs,
                            tune_cache_path.encode() if tune_cache_path else None)
        _check(lib().agatha_init(ctypes.byref(self._ptr), ctypes.byref(cfg)), what="agatha_init")

    @property
    def handle(self):
        return self._ptr

    def close(self):
        if self._ptr:
            lib().agatha_destroy(self._ptr)
            self._ptr = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def last_kernel_ms(self) -> float:
        ms = ctypes.c_float()
        _check(lib().agatha_last_kernel_ms(self._ptr, ctypes.byref(ms)), self._ptr,
               "agatha_last_kernel_ms")
        return float(ms.value)

    def last_error(self) -> str:
        return lib().agatha_last_error(self._ptr).decode()

    def tune_variants(self, scoring, w_max: Optional[int] = None):
        """The autotuner's variant per length class (indices into
        VARIANT_NAMES) followed by the split flag, or None if these parameters
        were not tuned yet."""
        v = (ctypes.c_int32 * 5)()
        p = make_params(scoring)
        rc = lib().agatha_tune_variants(self._ptr, ctypes.byref(p),
                                        ctypes.c_int32(scoring.w if w_max is None else w_max), v)
        if rc == AGATHA_EAGAIN:
            return None
        _check(rc, self._ptr, "agatha_tune_variants")
        return [int(x) for x in v]

    # -- alignment ---------------------------------------------------------
    def align_host(self, pb: PackedBatch, scoring, flags: int = 0, stream: int = 0,
                   out: Optional[np.ndarray] = None) -> np.ndarray:
        """agatha_align_batch with host arrays; returns the result records."""
        n = pb.n_pairs
        if out is None:
            out = np.zeros(n, dtype=RESULT_DTYPE)
        b = _host_batch(pb)
        p = make_params(scoring)
        rc = lib().agatha_align_batch(self._ptr, ctypes.byref(b), ctypes.byref(p),
                                      out.ctypes.data if n else None,
                                      ctypes.c_uint32(flags & ~AGATHA_DEVICE_PTRS),
                                      ctypes.c_void_p(stream) if stream else None)
        _check(rc, self._ptr, "agatha_align_batch")
        return out

    def align_local(self, pb: PackedBatch, scoring, h0, flags: int = 0, stream: int = 0,
                    out: Optional[np.ndarray] = None) -> np.ndarray:
        """agatha_align_batch_local with host arrays: the local extension
        from the initial scores h0 (one per pair); returns the result records."""
        n = pb.n_pairs
        if out is None:
            out = np.zeros(n, dtype=RESULT_DTYPE)
        h = np.ascontiguousarray(h0, dtype=np.int32)
        if h.shape[0] != n:
            raise ValueError("one initial score per pair")
        b = _host_batch(pb)
        p = make_params(scoring)
        rc = lib().agatha_align_batch_local(self._ptr, ctypes.byref(b), ctypes.byref(p),
                                            h.ctypes.data if n else None, out.ctypes.data if n else None,
                                            ctypes.c_uint32(flags & ~AGATHA_DEVICE_PTRS),
                                            ctypes.c_void_p(stream) if stream else None)
        _check(rc, self._ptr, "agatha_align_batch_local")
        return out

    def align_cigar(self, pb: PackedBatch, scoring, flags: int = 0, stream: int = 0,
                    cigar_cap: Optional[int] = None):
        """agatha_align_cigar with host arrays.  Returns (results, cigar_off,
        cigar): pair i's runs are cigar[cigar_off[i]:cigar_off[i + 1]].  The
        default capacity (t_len + q_len summed) always suffices."""
        n = pb.n_pairs
        out = np.zeros(n, dtype=RESULT_DTYPE)
        off = np.zeros(n + 1, dtype=np.int64)
        if cigar_cap is None:
            cigar_cap = int(np.asarray(pb.t_len, np.int64).sum() + np.asarray(pb.q_len, np.int64).sum())
        cigar = np.empty(max(int(cigar_cap), 1), dtype=np.uint32)
        b = _host_batch(pb)
        p = make_params(scoring)
        rc = lib().agatha_align_cigar(self._ptr, ctypes.byref(b), ctypes.byref(p),
                                      out.ctypes.data if n else None, off.ctypes.data,
                                      cigar.ctypes.data, ctypes.c_int64(int(cigar_cap)),
                                      ctypes.c_uint32(flags), ctypes.c_void_p(stream) if stream else None)
        _check(rc, self._ptr, "agatha_align_cigar")
        return out, off, cigar[: int(off[-1])]

    def last_traceback_info(self) -> dict:
        info = agatha_tb_info()
        _check(lib().agatha_last_traceback_info(self._ptr, ctypes.byref(info)), self._ptr,
               "agatha_last_traceback_info")
        return {"pairs16": int(info.pairs16), "pairs32": int(info.pairs32), "waves": int(info.waves),
                "fused": int(info.fused)}

    def last_traceback_ms(self) -> float:
        ms = ctypes.c_float()
        _check(lib().agatha_last_traceback_ms(self._ptr, ctypes.byref(ms)), self._ptr,
               "agatha_last_traceback_ms")
        return float(ms.value)

    def align_device(self, q_packed, t_packed, q_off, t_off, q_len, t_len, out, scoring,
                     flags: int = 0, stream: int = 0) -> None:
        """agatha_align_batch on device tensors (torch CUDA tensors or raw pointers).

        ``out`` is a uint8 device tensor of n_pairs * 48 bytes."""
        def ptr(x):
            return int(x.data_ptr()) if hasattr(x, "data_ptr") else int(x)

        def numel(x):
            return int(x.numel()) if hasattr(x, "numel") else int(len(x))

        n = numel(q_len)
        b = agatha_batch(n, ptr(q_packed), ptr(t_packed), numel(q_packed), numel(t_packed),
                         ptr(q_off), ptr(t_off), ptr(q_len), ptr(t_len))
        p = make_params(scoring)
        rc = lib().agatha_align_batch(self._ptr, ctypes.byref(b), ctypes.byref(p),
                                      ctypes.c_void_p(ptr(out)),
                                      ctypes.c_uint32(flags | AGATHA_DEVICE_PTRS),
                                      ctypes.c_void_p(stream) if stream else None)
        _check(rc, self._ptr, "agatha_align_batch")


AGATHA_NOALLOC_MAX_PAIRS = 65536


def agatha_align_batch_noalloc(q_packed, t_packed, q_off, t_off, q_len, t_len, out, scoring,
                               stream: int = 0, n_pairs: Optional[int] = None,
                               words: Optional[tuple] = None) -> None:
    """The allocation-free entry point on device tensors (torch CUDA tensors or
    raw pointers).  ``out`` holds n_pairs * 48 bytes of device memory;
    ``words`` = (q_words, t_words) overrides the stream sizes taken from the
    tensors."""
    def ptr(x):
        if x is None:
            return None
        return int(x.data_ptr()) if hasattr(x, "data_ptr") else int(x)

    def numel(x):
        return 0 if x is None else (int(x.numel()) if hasattr(x, "numel") else int(len(x)))

    n = numel(q_len) if n_pairs is None else int(n_pairs)
    qw, tw = words if words is not None else (numel(q_packed), numel(t_packed))
    b = agatha_batch(n, ptr(q_packed), ptr(t_packed), qw, tw,
                     ptr(q_off), ptr(t_off), ptr(q_len), ptr(t_len))
    p = make_params(scoring)
    _check(lib().agatha_align_batch_noalloc(ctypes.byref(b), ctypes.byref(p),
                                            ctypes.c_void_p(ptr(out)) if out is not None else None,
                                            ctypes.c_void_p(stream) if stream else None),
           what="agatha_align_batch_noalloc")


class Server:
    """The serving loop of a context: ``agatha_serve_start`` ... ``agatha_serve_stop``.

    ``submit`` copies the request's inputs before it returns; the result array
    it hands back is filled by the library when the ticket completes and must
    not be read before ``wait`` (or ``poll``) reports completion."""

    def __init__(self, ctx: Context, mem_budget_bytes: int = 0, max_inflight: int = 0,
                 max_batch_pairs: int = 0, linger_us: int = 0, launch_flags: int = 0):
        self.ctx = ctx
        cfg = agatha_serve_config(int(mem_budget_bytes), int(max_inflight), int(max_batch_pairs),
                                  int(linger_us), int(launch_flags))
        _check(lib().agatha_serve_start(ctx.handle, ctypes.byref(cfg)), ctx.handle,
               "agatha_serve_start")
        self._out = {}          # ticket -> result array the library writes into

    def submit(self, pb: PackedBatch, scoring) -> int:
        n = pb.n_pairs
        out = np.zeros(max(n, 1), dtype=RESULT_DTYPE)
        b = _host_batch(pb)
        p = make_params(scoring)
        t = ctypes.c_uint64()
        _check(lib().agatha_serve_submit(self.ctx.handle, ctypes.byref(b), ctypes.byref(p),
                                         out.ctypes.data, ctypes.byref(t)),
               self.ctx.handle, "agatha_serve_submit")
        self._out[int(t.value)] = out[:n]
        return int(t.value)

    def poll(self, ticket: int) -> int:
        """AGATHA_OK, AGATHA_EAGAIN, AGATHA_ECANCELED ... (the raw code)."""
        return int(lib().agatha_serve_poll(self.ctx.handle, ctypes.c_uint64(ticket)))

    def wait_code(self, ticket: int, timeout_ms: int = -1) -> int:
        """agatha_serve_wait's raw code; the ticket's results stay reachable
        through ``result`` after AGATHA_OK."""
        return int(lib().agatha_serve_wait(self.ctx.handle, ctypes.c_uint64(ticket),
                                           ctypes.c_int32(timeout_ms)))

    def result(self, ticket: int) -> np.ndarray:
        return self._out.pop(ticket)

    def wait(self, ticket: int, timeout_ms: int = -1) -> np.ndarray:
        """Wait for a ticket and return its results; raises AgathaError otherwise."""
        rc = self.wait_code(ticket, timeout_ms)
        if rc != AGATHA_OK:
            if rc != AGATHA_ETIMEDOUT:
                self._out.pop(ticket, None)
            _check(rc, self.ctx.handle, "agatha_serve_wait")
        return self._out.pop(ticket)

    def stats(self) -> dict:
        st = agatha_serve_stats()
        _check(lib().agatha_serve_stats_get(self.ctx.handle, ctypes.byref(st)), self.ctx.handle,
               "agatha_serve_stats_get")
        return {name: getattr(st, name) for name, _ in agatha_serve_stats._fields_}

    def stop(self, drain: bool = True) -> None:
        _check(lib().agatha_serve_stop(self.ctx.handle, ctypes.c_int32(1 if drain else 0)),
               self.ctx.handle, "agatha_serve_stop")


def agatha_init(device: int = 0, **kw) -> Context:
    return Context(device, **kw)


def agatha_align_batch(ctx: Context, batch, scoring=None, flags: int = 0, stream: int = 0):
    """Align a workload batch (or a PackedBatch) on the GPU; host in, host out."""
    pb = batch if isinstance(batch, PackedBatch) else pack_batch(batch)
    if scoring is None:
        scoring = batch.scoring
    return ctx.align_host(pb, scoring, flags=flags, stream=stream)


def results_equal(a: np.ndarray, b: np.ndarray, fields: Sequence[str] = RESULT_FIELDS):
    """Indices of records that differ in any compared field."""
    bad = np.zeros(a.shape[0], dtype=bool)
    for f in fields:
        bad |= a[f] != b[f]
    return np.flatnonzero(bad)


def cigar_string(runs) -> str:
    """SAM-style text of CIGAR runs ((length << 4) | op)."""
    return "".join(f"{int(x) >> 4}{CIGAR_OPS[int(x) & 15]}" for x in runs)
