"""Serving benchmark: Poisson request arrivals into the continuous-batching
loop (``agatha_serve_*``), one JSON line per arrival rate.

Requests carry 1-512 pairs drawn uniformly from the ONT-like mix (20,000
pairs, w=500, Z-drop 400); the server has a 16 GB arena.  At each rate the
arrivals run until 2,000 requests or 10 s of arrivals, whichever comes first
(at least 50 requests).  Latency = completion - scheduled arrival, where
completion is seen by a thread that waits on the tickets in submission order
(a request that completes before an earlier one is counted when the earlier
one is done, so tail figures are, if anything, pessimistic).  The library's
own submit-to-completion percentiles are reported beside them.

    python -m paper_2403_06478_gb300.serve_bench [--rates 10,100,1000] [--budget-gb 16]
        [--tune-cache FILE]

Each line also carries the overlap figures of the server (launches in
flight at once, and from the device's global timer the most launches whose
kernels ran at one instant and the device time with two or more), the tuned
plan the merged launches used, and the GPU clocks sampled during the point.
"""
from __future__ import annotations

import argparse
import json
import threading
import time

import numpy as np

from . import agatha as A
from . import build as B
from . import workload as W
from .clocks import ClockSampler


def _point(ctx, pool_pb, pool, rate, args, rng):
    n_req = int(max(50, min(args.max_requests, round(rate * args.max_seconds))))
    reqs = W.poisson_requests(rng, rate, n_req, pool.n_pairs, args.max_pairs)
    # each request references the pool's packed streams: submission copies
    # only the words its pairs touch
    batches = [A.PackedBatch(pool_pb.q_packed, pool_pb.t_packed, pool_pb.q_off[r.pair_idx],
                             pool_pb.t_off[r.pair_idx], pool_pb.q_len[r.pair_idx],
                             pool_pb.t_len[r.pair_idx]) for r in reqs]
    srv = A.Server(ctx, mem_budget_bytes=int(args.budget_gb * (1 << 30)),
                   max_inflight=args.max_inflight, max_batch_pairs=args.max_batch_pairs,
                   linger_us=args.linger_us, launch_flags=LAUNCH_PLANS[args.plan])
    tickets = [None] * n_req
    done_at = [0.0] * n_req
    submitted = threading.Semaphore(0)

    def waiter():
        for i in range(n_req):
            submitted.acquire()
            srv.wait(tickets[i])
            done_at[i] = time.perf_counter()

    th = threading.Thread(target=waiter)
    th.start()
    sampler = ClockSampler(args.device)
    sampler.start()
    t0 = time.perf_counter()
    for i, r in enumerate(reqs):
        delay = t0 + r.arrival_s - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        tickets[i] = srv.submit(batches[i], pool.scoring)
        submitted.release()
    th.join()
    t_end = max(done_at)
    clocks = sampler.stop()
    st = srv.stats()
    srv.stop(drain=True)
    lat = np.array([done_at[i] - (t0 + reqs[i].arrival_s) for i in range(n_req)]) * 1e3
    pairs = int(sum(len(r.pair_idx) for r in reqs))
    wall = t_end - t0
    return {
        "rate_req_s": rate, "requests": n_req, "pairs": pairs,
        "offered_pairs_per_s": pairs / reqs[-1].arrival_s,
        "pairs_per_s": pairs / wall, "gcups": st["cells_done"] / wall / 1e9,
        "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
        "lib_p50_ms": st["p50_latency_ms"], "lib_p99_ms": st["p99_latency_ms"],
        "launches": st["launches"], "busy_s": st["busy_seconds"], "wall_s": wall,
        "peak_bytes_in_flight": st["peak_bytes_in_flight"],
        "max_launches_in_flight": st["max_launches_in_flight"],
        "max_device_concurrency": st["max_device_concurrency"],
        "device_overlap_s": st["overlap_seconds"],
        "clocks": clocks,
    }


# launch plans the server can run: the context's autotuned plan, or several
# warps per pair (shorter latency for the long pairs of a request)
LAUNCH_PLANS = {"tuned": 0, "warps2": A.AGATHA_WARPS2 | A.AGATHA_REGS_HIGH,
                "warps4": A.AGATHA_WARPS4 | A.AGATHA_REGS_HIGH}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--rates", default="10,20,50,100,200,500,1000,2000")
    ap.add_argument("--max-requests", type=int, default=2000)
    ap.add_argument("--max-seconds", type=float, default=10.0)
    ap.add_argument("--max-pairs", type=int, default=512)
    ap.add_argument("--budget-gb", type=float, default=16.0)
    ap.add_argument("--max-inflight", type=int, default=2)
    ap.add_argument("--max-batch-pairs", type=int, default=8192)
    ap.add_argument("--linger-us", type=int, default=0)
    ap.add_argument("--plan", default="tuned", choices=sorted(LAUNCH_PLANS),
                    help="plan of the server's launches: the autotuned one, or 2 or 4 warps per pair")
    ap.add_argument("--device", type=int, default=0)
    ap.add_argument("--tune-cache", default=None,
                    help="autotuner cache file (the benchmark's, to serve with the same plan)")
    args = ap.parse_args(argv)
    B.build()
    pool = W.make_config("ont")
    pool_pb = A.pack_batch(pool)
    ctx = A.Context(args.device, autotune=True, tune_cache_path=args.tune_cache)
    # the autotuner measures its plan on one host batch of the scoring; the
    # server's merged launches then use it
    ctx.align_host(pool_pb, pool.scoring)
    tuned = ctx.tune_variants(pool.scoring)
    rng = np.random.default_rng(W.SEED_BASE + 5)
    for rate in [float(x) for x in args.rates.split(",")]:
        line = _point(ctx, pool_pb, pool, rate, args, rng)
        line["config"] = {"workload": "serving: Poisson arrivals, 1-512 ONT-like pairs per request",
                          "budget_gb": args.budget_gb, "max_inflight": args.max_inflight,
                          "max_batch_pairs": args.max_batch_pairs, "linger_us": args.linger_us,
                          "plan": args.plan,
                          "tuned_plan": None if tuned is None else
                          {"variants": [A.VARIANT_NAMES[v] for v in tuned[:4]], "split": bool(tuned[4])}}
        print(json.dumps(line), flush=True)
    ctx.close()


if __name__ == "__main__":
    main()
