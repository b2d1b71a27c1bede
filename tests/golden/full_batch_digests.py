"""Digests of the CPU oracle's results on the full-size workloads.

Running this file as a script aligns every pair of the ONT-like, HiFi-like and
skewed batches (20,000 / 20,000 / 100,000 pairs, seeded as in the workload
module) with the oracle only, on all host cores, and writes
``full_batch_oracle.txt`` beside it:

    name  n_pairs  input_sha256  result_sha256  cells  zdropped  chunk  chunk digests

The GPU test of every pair (``tests/test_gpu_full_parity.py``) compares the
library's results with these digests, chunk by chunk, and recomputes the
oracle for a chunk whose digest differs to name the pairs.  When the seeded
inputs themselves differ (another numpy on the machine running the test: the
input digest tells), the test runs the oracle on the whole batch instead.

Nothing here computes an alignment: the digests are of the oracle's output
(and of the generator's input), in a fixed byte layout.
"""
from __future__ import annotations

import hashlib
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
GOLDEN = os.path.join(HERE, "full_batch_oracle.txt")
CONFIGS = ("ont", "hifi", "skewed")
CHUNK = 1000

# the compared result fields in a fixed little-endian layout (the oracle's
# and the library's result records share these names)
_CANON = np.dtype([("max", "<i4"), ("qe", "<i4"), ("te", "<i4"), ("gscore", "<i4"),
                   ("mqe", "<i4"), ("mqe_t", "<i4"), ("mte", "<i4"), ("mte_q", "<i4"),
                   ("cells", "<i8"), ("zdropped", "u1"), ("reach_end", "u1")])


def canonical(results: np.ndarray) -> np.ndarray:
    out = np.zeros(results.shape[0], dtype=_CANON)
    for f in _CANON.names:
        out[f] = results[f]
    return out


def result_digest(results: np.ndarray) -> str:
    return hashlib.sha256(canonical(results).tobytes()).hexdigest()


def chunk_digests(results: np.ndarray, chunk: int = CHUNK) -> list:
    c = canonical(results)
    return [hashlib.sha256(c[i:i + chunk].tobytes()).hexdigest()[:16]
            for i in range(0, c.shape[0], chunk)]


def input_digest(batch) -> str:
    h = hashlib.sha256()
    for a in (batch.q_len, batch.t_len, batch.q_off, batch.t_off, batch.q_codes, batch.t_codes):
        h.update(np.ascontiguousarray(a).tobytes())
    h.update(repr(batch.scoring.as_tuple()).encode())
    return h.hexdigest()


def read_golden(path: str = GOLDEN) -> dict:
    recs = {}
    if not os.path.exists(path):
        return recs
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        f = line.split()
        recs[f[0]] = {"n_pairs": int(f[1]), "input": f[2], "result": f[3], "cells": int(f[4]),
                      "zdropped": int(f[5]), "chunk": int(f[6]), "chunks": f[7].split(",")}
    return recs


def main(names=CONFIGS) -> int:
    sys.path.insert(0, ROOT)
    from oracle import oracle as O
    from paper_2403_06478_gb300 import workload as W
    lines = ["# Oracle results of the full-size workloads (tests/golden/full_batch_digests.py).",
             "# name n_pairs input_sha256 result_sha256 cells zdropped chunk chunk_digests",
             f"# written with numpy {np.__version__}, oracle on {os.cpu_count()} host threads"]
    old = read_golden()
    for name in CONFIGS:
        if name not in names and name in old:
            r = old[name]
            lines.append(f"{name} {r['n_pairs']} {r['input']} {r['result']} {r['cells']} "
                         f"{r['zdropped']} {r['chunk']} {','.join(r['chunks'])}")
            continue
        batch = W.make_config(name)
        t0 = time.perf_counter()
        res = O.align_batch(batch)
        dt = time.perf_counter() - t0
        print(f"{name}: {batch.n_pairs} pairs, {int(res['cells'].sum())} cells, {dt:.1f} s",
              flush=True)
        lines.append(f"{name} {batch.n_pairs} {input_digest(batch)} {result_digest(res)} "
                     f"{int(res['cells'].sum())} {int(res['zdropped'].sum())} {CHUNK} "
                     f"{','.join(chunk_digests(res))}")
    with open(GOLDEN, "w") as fh:
        fh.write("\n".join(lines) + "\n")
    return 0


if __name__ == "__main__":
    sys.exit(main(tuple(sys.argv[1:]) or CONFIGS))
