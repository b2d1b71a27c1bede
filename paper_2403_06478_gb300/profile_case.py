"""Profiling driver: align the first ``--pairs`` pairs of a workload a few times.

A small, self-contained case for ``ncu`` captures of one kernel (the full
benchmark is too long to replay under a profiler).  Prints the cell count.
"""
import argparse
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

from paper_2403_06478_gb300 import agatha as A  # noqa: E402
from paper_2403_06478_gb300 import build as B  # noqa: E402
from paper_2403_06478_gb300 import workload as W  # noqa: E402

FLAGS = {"batched": 0, "plain": A.AGATHA_PLAIN, "force32": A.AGATHA_FORCE32,
         "edge": A.AGATHA_EDGE_PATH_ONLY, "regs_high": A.AGATHA_REGS_HIGH,
         "two_pass": A.AGATHA_TB_TWO_PASS}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="ont")
    ap.add_argument("--pairs", type=int, default=2000)
    ap.add_argument("--repeat", type=int, default=2)
    ap.add_argument("--length", type=int, default=20000,
                    help="pair length of --workload identical / fixed")
    ap.add_argument("--path", default="batched", choices=sorted(FLAGS))
    ap.add_argument("--traceback", action="store_true", help="agatha_align_cigar instead")
    args = ap.parse_args()
    B.build()
    if args.workload == "identical":
        # long identical pairs: every anti-diagonal after the first w+2 is a bulk step
        import numpy as np
        rng = np.random.default_rng(5)
        xs = [rng.integers(0, 4, args.length).astype(np.uint8) for _ in range(args.pairs)]
        batch = W.from_pairs(xs, [x.copy() for x in xs], W.ONT_SCORING, name="identical")
    elif args.workload == "fixed":
        # pairs of one length with small-config errors and ONT-like scoring
        batch = W.make_long_ratio(1.0, n_pairs=args.pairs, long_len=args.length)
    else:
        batch = W.make_config(args.workload, n_pairs=args.pairs)
    pb = A.pack_batch(batch)
    with A.Context(0) as ctx:
        for _ in range(args.repeat):
            if args.traceback:
                res, off, _ = ctx.align_cigar(pb, batch.scoring, flags=FLAGS[args.path])
            else:
                res = ctx.align_host(pb, batch.scoring, flags=FLAGS[args.path])
    print(f"ok {args.workload} pairs={batch.n_pairs} cells={int(res['cells'].sum())}")


if __name__ == "__main__":
    main()
