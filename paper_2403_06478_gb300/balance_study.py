"""Load-balancing study on two-length mixes (the paper's 4096 bp / 128 bp
experiment, Section 5.6), one JSON line per long-pair fraction.

The paper compares its uneven bucketing against sorting and the original
order.  Here the persistent kernel always pulls pairs from a device queue;
the comparison is between that queue in longest-predicted-first order (the
default batched path), the same queue in input order (AGATHA_NO_SORT), and
the plain kernel (one block per pair, input order).  Results of all three are
checked to be identical.

    python -m paper_2403_06478_gb300.balance_study [--fractions 0.01,0.05,0.1,0.25,0.5]
"""
from __future__ import annotations

import argparse
import json
import statistics

from . import agatha as A
from . import build as B
from . import workload as W


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--fractions", default="0.01,0.05,0.1,0.25,0.5,0.75")
    ap.add_argument("--pairs", type=int, default=20000)
    ap.add_argument("--repeat", type=int, default=3)
    ap.add_argument("--device", type=int, default=0)
    args = ap.parse_args(argv)
    B.build()
    with A.Context(args.device, timing=True) as ctx:
        for f in [float(x) for x in args.fractions.split(",")]:
            batch = W.make_long_ratio(f, n_pairs=args.pairs)
            pb = A.pack_batch(batch)
            line = {"long_fraction": f, "pairs": batch.n_pairs,
                    "workload": f"{args.pairs} pairs, {f:.0%} of 4096 bp, the rest 128 bp, "
                                "5% sub / 2.5% ins / 2.5% del, ONT-like scoring (w=500)"}
            ref = None
            for label, flags, reps in (("lpt_queue", 0, args.repeat),
                                       ("input_order_queue", A.AGATHA_NO_SORT, args.repeat),
                                       ("plain", A.AGATHA_PLAIN, 1)):
                ms = []
                for _ in range(reps):
                    res = ctx.align_host(pb, batch.scoring, flags=flags)
                    ms.append(ctx.last_kernel_ms())
                if ref is None:
                    ref = res
                elif A.results_equal(res, ref).size:
                    raise AssertionError(f"{label} differs from the batched path at fraction {f}")
                cells = int(res["cells"].sum())
                t = statistics.median(ms)
                line[label] = {"kernel_ms": round(t, 3), "gcups": round(cells / t / 1e6, 1)}
            line["lpt_vs_input_order"] = round(line["input_order_queue"]["kernel_ms"] /
                                               line["lpt_queue"]["kernel_ms"], 3)
            line["lpt_vs_plain"] = round(line["plain"]["kernel_ms"] / line["lpt_queue"]["kernel_ms"], 3)
            print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
