"""How much could predicting the termination point gain?  One JSON line per workload.

The paper's discussion proposes predicting, before execution, where the
termination test (Eq. 4-7) will fire, so that the scheduler knows each pair's
real work.  The device queue here orders pairs by the Section 4.5 estimate
(anti-diagonals x band width), an upper bound that ignores termination.  This
study bounds what any predictor could add: it aligns each batch once, then
times the kernel with the queue in three orders, all through the same
persistent kernel and results checked identical:
  predicted   the default: longest predicted work first (device-side ordering)
  ideal       longest *actual* work first: the cells each pair really computed,
              known only after aligning it (a perfect predictor)
  input       the order of the batch (AGATHA_NO_SORT)

    python -m paper_2403_06478_gb300.termination_study [--workloads ont,skewed,hifi]
"""
from __future__ import annotations

import argparse
import json
import statistics

import numpy as np

from . import agatha as A
from . import build as B
from . import workload as W


def _permuted(pb: A.PackedBatch, idx: np.ndarray) -> A.PackedBatch:
    return A.PackedBatch(pb.q_packed, pb.t_packed, np.ascontiguousarray(pb.q_off[idx]),
                         np.ascontiguousarray(pb.t_off[idx]), np.ascontiguousarray(pb.q_len[idx]),
                         np.ascontiguousarray(pb.t_len[idx]))


def _time(ctx, pb, scoring, flags, reps):
    ms = []
    res = None
    for _ in range(reps):
        res = ctx.align_host(pb, scoring, flags=flags)
        ms.append(ctx.last_kernel_ms())
    return statistics.median(ms), res


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--workloads", default="ont,skewed,hifi")
    ap.add_argument("--repeat", type=int, default=3)
    ap.add_argument("--device", type=int, default=0)
    args = ap.parse_args(argv)
    B.build()
    with A.Context(args.device, timing=True) as ctx:
        for name in args.workloads.split(","):
            batch = W.make_config(name)
            pb = A.pack_batch(batch)
            sc = batch.scoring
            ctx.align_host(pb, sc)                                  # warm-up
            t_pred, res = _time(ctx, pb, sc, 0, args.repeat)
            ideal = np.argsort(-res["cells"], kind="stable")
            t_ideal, res_i = _time(ctx, _permuted(pb, ideal), sc, A.AGATHA_NO_SORT, args.repeat)
            t_input, res_n = _time(ctx, pb, sc, A.AGATHA_NO_SORT, args.repeat)
            if A.results_equal(res_i, res[ideal]).size or A.results_equal(res_n, res).size:
                raise AssertionError(f"{name}: results depend on the order")
            cells = int(res["cells"].sum())
            terminated = res["zdropped"] == 1
            line = {
                "workload": name, "pairs": batch.n_pairs, "cells": cells,
                "pairs_terminated_early": int(terminated.sum()),
                "kernel_ms": {"predicted": round(t_pred, 3), "ideal": round(t_ideal, 3),
                              "input": round(t_input, 3)},
                "gcups": {"predicted": round(cells / t_pred / 1e6, 1), "ideal": round(cells / t_ideal / 1e6, 1),
                          "input": round(cells / t_input / 1e6, 1)},
                "ideal_gain_over_predicted": round(t_pred / t_ideal, 4),
            }
            print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
