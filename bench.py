#!/usr/bin/env python
"""Benchmark of banded two-piece-affine Z-drop extension alignment on GB300.

One step = one pass of the whole hot path (validation, longest-first ordering,
the batched warp kernel) over one batch of synthetic ONT-like pairs (20,000
pairs, log-normal lengths with median 5 kbp, 12% errors, 10% divergent tails,
w=500, zdrop=400).  Printed as one JSON line:

  value       GCUPS of the batched kernel path, inputs resident in HBM, CUDA
              events on the launching stream, L2 flushed between steps
  e2e         the same metric through agatha_align_batch with pinned HOST
              buffers (host->device copies and result read-back included)
  plain       the plain one-pair-per-block kernel on the same batch
  roofline    the warp kernel against the integer issue rate of the GPU
  cpu_baseline the CPU oracle on a bounded sample of the same workload

``--workload hifi|skewed|small`` measures another configuration with the same
metric (the ONT-like batch is the default and the headline).
``--traceback`` measures the path with its CIGARs (agatha_align_cigar): the
score kernels plus the direction-recording traceback kernel.
``--impl reference`` times the CPU oracle as the reference arm instead.
Multi-GPU (torchrun): every rank aligns its own batch (weak scaling, no
collective on the data path); rank 0 prints the aggregate.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_2403_06478_gb300.clocks import ClockSampler  # noqa: E402

METRIC = "GCUPS & pairs/s on ONT-like mix: batched vs plain GPU kernel, bit-exact"
WORKLOADS = {
    "ont": ("ont: 20000 pairs, query log-normal (median 5 kbp, sigma 0.8, clip 500-50k), "
            "target 5% sub / 4% del / 3% ins, 10% divergent tails, a=2 b=4 q=4 e=2 q2=24 e2=1, "
            "w=500, zdrop=400"),
    "hifi": ("hifi: 20000 pairs, query Normal(15 kbp, 3 kbp) min 2 kbp, 1% errors "
             "(0.5 sub / 0.25 ins / 0.25 del), 2% divergent tails, a=1 b=4 q=6 e=2 q2=26 e2=1, "
             "w=500, zdrop=200"),
    "skewed": ("skewed: 100000 pairs, query Pareto(alpha 1.5, min 500 bp, cap 100 kbp), 8% errors "
               "(4 sub / 2 ins / 2 del), 20% divergent tails, a=2 b=4 q=4 e=2 q2=24 e2=1, w=750, "
               "zdrop=400"),
    "small": ("small: 256 pairs of 1000 bp, 5% sub / 2.5% ins / 2.5% del, a=2 b=4 q=4 e=2 "
              "q2=24 e2=1, w=100, zdrop=400"),
    "short": ("short: 200000 pairs of 150 bp, 1% errors (0.8 sub / 0.1 ins / 0.1 del), 5% divergent "
              "tails, BWA-MEM default parameters a=1 b=4 q=6 e=1 (single piece), w=100, zdrop=100, "
              "end_bonus=5, this method's extension rules"),
}
L2_FLUSH_BYTES = 512 << 20          # > 129 MB of L2
# algorithmic integer lane-ops per band cell (substitution score 2, five-way
# max 3, two gap openings 2, four gap add-max 4, max tracking 2); a packed
# 16x2 lane op serves two cells
OPS_PER_CELL_I32 = 13.0
OPS_PER_CELL_I16X2 = 6.5
# traceback kernel: the cell ops plus the direction byte (four equality and
# four gap-continuation comparisons, one byte insert); halved on 16x2 lanes
OPS_PER_CELL_TB = OPS_PER_CELL_I32 + 9.0
OPS_PER_CELL_TB16 = OPS_PER_CELL_TB / 2
CPU_SAMPLE_PAIRS = 6000
CPU_SAMPLE_CELLS = 4e10             # about 12 s of the oracle on 16 cores
CPU_SAMPLE_CELLS_1T = 2e9           # about 10 s on one core
REF_STEP_PAIRS = 300


def _env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            return json.load(fh), "measured"
    return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


def traffic_from_profile(kernel, input_bytes):
    """DRAM bytes per launch of the dominant kernel, from the committed ncu
    capture of a smaller case of the same kernel scaled by input bytes (the
    kernel reads its inputs once; band state never leaves the SM); null if
    the capture was taken on another kernel or build."""
    path = os.path.join(ROOT, "profiles", "warp16_kernel_ont_traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        d = json.load(fh)
    if d.get("kernel") != kernel or d.get("kernel_digest") != _kernel_digest():
        return None
    return int(d["dram_bytes_per_input_byte"] * input_bytes)


def traffic_tb16(kernel, table_bytes):
    """DRAM bytes of one traceback launch, scaled from the committed capture
    of a smaller case by direction-table bytes (null for another build)."""
    name = "tbf16_kernel_traffic.json" if kernel.startswith("tbf16") else "tb16_kernel_traffic.json"
    path = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        d = json.load(fh)
    if d.get("kernel") != kernel or d.get("kernel_digest") != _kernel_digest(
            ("kernel_tb.cuh", "kernel_warp16.cuh", "kernel_warp16_c16.cu", "agatha_dev.cuh")):
        return None
    return int(d["dram_bytes_per_table_byte"] * table_bytes)


def _kernel_digest(files=None):
    """Digest of the 16-bit kernel's sources: a traffic figure is only valid
    for the build it was measured on."""
    import hashlib
    h = hashlib.sha256()
    for f in files or ("kernel_warp16.cuh", "kernel_warp16_c4.cu", "kernel_warp16_c8.cu",
                       "kernel_warp16_c16.cu", "kernel_warp16_c24.cu", "agatha_dev.cuh"):
        with open(os.path.join(ROOT, "paper_2403_06478_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def cpu_baseline(batch, n_sample: int, gpu_res=None, seed: int = 7):
    """The oracle on a bounded random sample of the batch, all host cores, and
    one core on part of it.  With ``gpu_res`` (the timed step's results), the
    sample's oracle results are also compared with them pair by pair."""
    from oracle import oracle as O      # the CPU oracle: timed here as a reported baseline
    from paper_2403_06478_gb300 import shard as S
    rng = np.random.default_rng(seed)
    idx = rng.permutation(batch.n_pairs)[:n_sample]
    # bounded: stop adding pairs once the predicted work reaches CPU_SAMPLE_CELLS
    est = np.cumsum(S.predicted_cells(batch.q_len[idx], batch.t_len[idx], batch.scoring.w))
    idx = np.sort(idx[:max(1, int(np.searchsorted(est, CPU_SAMPLE_CELLS)) + 1)])
    cores = os.cpu_count() or 1
    O.align_batch(batch, idx=idx[:8], threads=cores)     # load + warm
    t0 = time.perf_counter()
    res = O.align_batch(batch, idx=idx, threads=cores)
    dt = time.perf_counter() - t0
    cells = int(res["cells"].sum())
    # one thread on a smaller part of the same sample (about 10 s)
    est1 = np.cumsum(S.predicted_cells(batch.q_len[idx], batch.t_len[idx], batch.scoring.w))
    one = idx[:max(1, int(np.searchsorted(est1, CPU_SAMPLE_CELLS_1T)) + 1)]
    t0 = time.perf_counter()
    res1 = O.align_batch(batch, idx=one, threads=1)
    dt1 = time.perf_counter() - t0
    cells1 = int(res1["cells"].sum())
    out = {"value": round(cells / dt / 1e9, 4), "unit": "GCUPS", "cores": cores, "kind": "oracle",
           "sample": f"{idx.size} seeded random pairs of the workload ({cells} cells, {dt:.1f} s)",
           "single_thread": {"value": round(cells1 / dt1 / 1e9, 4), "unit": "GCUPS", "cores": 1,
                             "sample": f"{one.size} of those pairs ({cells1} cells, {dt1:.1f} s)"}}
    if gpu_res is not None:
        fields = O.COMPARE_FIELDS
        sub = gpu_res[idx]
        bad = [int(idx[k]) for k in
               np.flatnonzero(np.any([sub[f] != res[f] for f in fields], axis=0))]
        out["oracle_checked_pairs"] = int(idx.size)
        out["oracle_checked_cells"] = cells
        out["oracle_exact"] = not bad
        if bad:
            out["oracle_mismatches"] = bad[:20]
    return out


PROFILE_PATHS = ("batched", "plain", "force32", "edge", "regs_high", "two_pass")


def run_profile_case(args):
    """A small case for ncu captures of one kernel (the timed benchmark is too
    long to replay under a profiler): the first --pairs pairs of the workload
    (or --pairs pairs of one --length: ``identical`` sequences, every
    anti-diagonal after the first w+2 a bulk step, or ``fixed``-length pairs
    with the small configuration's errors and ONT-like scoring), aligned
    --repeat times on the chosen path.  Prints the cell count, not a bench line."""
    from paper_2403_06478_gb300 import agatha as A
    from paper_2403_06478_gb300 import build as B
    from paper_2403_06478_gb300 import workload as W
    flags = {"batched": 0, "plain": A.AGATHA_PLAIN, "force32": A.AGATHA_FORCE32,
             "edge": A.AGATHA_EDGE_PATH_ONLY, "regs_high": A.AGATHA_REGS_HIGH,
             "two_pass": A.AGATHA_TB_TWO_PASS}[args.path]
    B.build()
    if args.workload == "identical":
        rng = np.random.default_rng(5)
        xs = [rng.integers(0, 4, args.length).astype(np.uint8) for _ in range(args.pairs)]
        batch = W.from_pairs(xs, [x.copy() for x in xs], W.ONT_SCORING, name="identical")
    elif args.workload == "fixed":
        batch = W.make_long_ratio(1.0, n_pairs=args.pairs, long_len=args.length)
    else:
        batch = W.make_config(args.workload, n_pairs=args.pairs)
    pb = A.pack_batch(batch)
    with A.Context(0) as ctx:
        for _ in range(args.repeat):
            if args.traceback:
                res, _, _ = ctx.align_cigar(pb, batch.scoring, flags=flags)
            else:
                res = ctx.align_host(pb, batch.scoring, flags=flags)
    print(f"ok {args.workload} pairs={batch.n_pairs} cells={int(res['cells'].sum())}")
    return 0


def run_reference(args):
    """Reference arm: the CPU oracle on bounded samples of the same workload."""
    rank = _env_int("RANK", 0)
    if rank != 0:
        return 0
    from paper_2403_06478_gb300 import workload as W
    from oracle import oracle as O
    batch = W.make_config(args.workload)
    cores = os.cpu_count() or 1
    rng = np.random.default_rng(11)
    perm = rng.permutation(batch.n_pairs)

    def sample(k):
        lo = (k * REF_STEP_PAIRS) % batch.n_pairs
        return np.sort(perm[lo:lo + REF_STEP_PAIRS])

    O.build()
    for k in range(args.warmup):
        O.align_batch(batch, idx=sample(k), threads=cores)
    total_cells, total_s, total_pairs = 0, 0.0, 0
    for k in range(args.steps):
        idx = sample(args.warmup + k)
        t0 = time.perf_counter()
        res = O.align_batch(batch, idx=idx, threads=cores)
        total_s += time.perf_counter() - t0
        total_cells += int(res["cells"].sum())
        total_pairs += idx.size
    gcups = total_cells / total_s / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": round(gcups, 4), "unit": "GCUPS",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(total_s / max(args.steps, 1) * 1e3, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload],
                   "step": f"{REF_STEP_PAIRS} pairs per step (bounded sample)"},
        "pairs_per_s": round(total_pairs / total_s, 2),
        "cpu_baseline": {"value": round(gcups, 4), "unit": "GCUPS", "cores": cores, "kind": "oracle",
                         "sample": f"{args.steps} steps x {REF_STEP_PAIRS} seeded random pairs"},
        "e2e": {"value": round(gcups, 4), "unit": "GCUPS", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def traceback_cells(res, batch):
    """Band cells on anti-diagonals 0..r_end of every pair's traceback (the
    cells the traceback kernel computes), r_end the end cell's anti-diagonal."""
    w_all = batch.scoring.w
    total = 0
    for i in range(batch.n_pairs):
        tl, ql = int(batch.t_len[i]), int(batch.q_len[i])
        r = res[i]
        et, eq = (int(r["mqe_t"]), ql - 1) if r["reach_end"] else (int(r["te"]), int(r["qe"]))
        if tl <= 0 or ql <= 0 or et < 0 or eq < 0:
            continue
        w = w_all if 0 <= w_all <= max(tl, ql) else max(tl, ql)
        rr = np.arange(et + eq + 1, dtype=np.int64)
        st = np.maximum(np.maximum(0, rr - ql + 1), -((w - rr) // 2))
        en = np.minimum(np.minimum(tl - 1, rr), (rr + w) // 2)
        total += int(np.maximum(0, en - st + 1).sum())
    return total


# local extension (the BWA-MEM variant): the int32 cell update (13), the
# row accumulator riding with E (max and its t: 2) and the floors of the
# four gap states at zero (4)
OPS_PER_CELL_LOCAL = 19.0


def run_local(args):
    """The BWA-MEM variant of the extension through agatha_align_batch_local:
    local extension of every pair from its seed score (uniform 19-60, the
    workload module's seed_scores), one query row at a time.

    value = cells / local-kernel time (CUDA events the library records
    around the kernel on the call's stream); e2e = the same cells / the whole
    call from pinned host buffers (copies both ways included).  Weak scaling
    under torchrun like the score path."""
    import torch
    from paper_2403_06478_gb300 import agatha as A
    from paper_2403_06478_gb300 import build as B
    from paper_2403_06478_gb300 import shard as S
    from paper_2403_06478_gb300 import workload as W
    rank, world, local = _env_int("RANK", 0), _env_int("WORLD_SIZE", 1), _env_int("LOCAL_RANK", 0)
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    B.build()
    batch = W.make_config(args.workload, seed=None if rank == 0 else W.SEED_BASE + 2 + 1000 * rank)
    h0 = W.seed_scores(batch.n_pairs, seed=None if rank == 0 else W.SEED_BASE + 8 + 1000 * rank)
    pb = A.pack_batch(batch)
    pin = {k: torch.from_numpy(getattr(pb, k)).pin_memory() for k in
           ("q_packed", "t_packed", "q_off", "t_off", "q_len", "t_len")}
    pin_pb = A.PackedBatch(*[pin[k].numpy() for k in
                             ("q_packed", "t_packed", "q_off", "t_off", "q_len", "t_len")])
    h0_pin = torch.from_numpy(h0).pin_memory().numpy()
    n = pb.n_pairs
    host_out = torch.empty(n * 48, dtype=torch.uint8).pin_memory().numpy().view(A.RESULT_DTYPE)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    ctx = A.Context(local, timing=True)
    for _ in range(args.warmup):
        ctx.align_local(pin_pb, batch.scoring, h0_pin, stream=stream.cuda_stream, out=host_out)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    k_ms, e2e_ms = [], []
    for k in range(args.steps):
        flush.fill_(k & 0xff)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.align_local(pin_pb, batch.scoring, h0_pin, stream=stream.cuda_stream, out=host_out)
        e1.record(stream)
        e1.synchronize()
        e2e_ms.append(e0.elapsed_time(e1))
        k_ms.append(ctx.last_kernel_ms())
    torch.cuda.synchronize()
    clocks = sampler.stop()
    res = host_out.copy()
    cells = int(res["cells"].sum())
    (all_cells, all_pairs), (k_tot, e2e_tot) = S.reduce_step_stats(
        [cells, n], [sum(k_ms), sum(e2e_ms)], device="cuda")
    if rank != 0:
        ctx.close()
        if dist is not None:
            dist.destroy_process_group()
        return 0
    peaks, peak_kind = measured_peaks()
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    sm_max_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    int_peak = n_sm * 128 * sm_max_mhz * 1e6 / 1e12
    t_ms = statistics.mean(k_ms)
    achieved = cells * OPS_PER_CELL_LOCAL / (t_ms / 1e3) / 1e12
    w = batch.scoring.w
    C = next(c for c in (4, 8, 16) if 32 * c - 1 >= w)
    line = {
        "metric": "GCUPS of the local extension from seed scores (BWA-MEM variant), exact",
        "value": round(all_cells * args.steps / (k_tot / 1e3) / 1e9, 3), "unit": "GCUPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(k_tot / args.steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload], "pairs_per_gpu": n, "cells_per_step": cells,
                   "h0": "seed scores uniform in [19, 60]", "l2": "flushed between steps (512 MB write)",
                   "value_basis": "local kernel, CUDA events on the call's stream"},
        "pairs_per_s": round(all_pairs * args.steps / (k_tot / 1e3), 1),
        "zdropped": int(res["zdropped"].sum()), "reach_end": int(res["reach_end"].sum()),
        "e2e": {"value": round(all_cells * args.steps / (e2e_tot / 1e3) / 1e9, 3), "unit": "GCUPS",
                "h2d_bytes_per_step": int(pin_pb.nbytes() + 4 * n), "d2h_bytes_per_step": int(n * 48 + 64),
                "ms_per_step": round(e2e_tot / args.steps, 3)},
        "gpu_launches": args.steps * 4,          # prep classify / scan / scatter, local kernel
        "roofline": {"bound": "alu", "achieved": round(achieved, 3), "peak": round(int_peak, 3),
                     "unit": "Tops/s", "frac": round(achieved / int_peak, 4), "traffic": None,
                     "kernel": f"local_align_kernel<{C}>", "kernel_ms": round(t_ms, 3),
                     "ops_per_cell": OPS_PER_CELL_LOCAL,
                     "peak_basis": f"{n_sm} SMs x 128 int32 lanes x {sm_max_mhz:.0f} MHz ({peak_kind})"},
        "clocks": clocks,
    }
    if world == 1 and not args.no_cpu_baseline:
        from oracle import oracle as O     # the CPU oracle: timed as a reported baseline and checked
        # the whole batch: about 4e9 cells, a few seconds on the host cores,
        # and every pair checked against the timed results
        idx = np.arange(n)
        cores = os.cpu_count() or 1
        t0 = time.perf_counter()
        ref = O.align_batch(batch, idx=idx, threads=cores, h0=h0)
        dt = time.perf_counter() - t0
        sub = res[idx]
        bad = np.flatnonzero(np.any([sub[f] != ref[f] for f in O.COMPARE_FIELDS], axis=0))
        line["cpu_baseline"] = {"value": round(int(ref["cells"].sum()) / dt / 1e9, 4), "unit": "GCUPS",
                                "cores": cores, "kind": "oracle",
                                "sample": f"all {idx.size} pairs ({int(ref['cells'].sum())} cells, {dt:.1f} s)",
                                "oracle_checked_pairs": int(idx.size), "oracle_exact": bool(bad.size == 0)}
        line["oracle_exact"] = bool(bad.size == 0)
        line["oracle_checked_pairs"] = int(idx.size)
    print(json.dumps(line), flush=True)
    ctx.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_traceback(args):
    """The path with CIGARs through agatha_align_cigar (host buffers only).

    value = score cells / (score kernels + traceback kernels), CUDA events on
    the call's stream; e2e = the same cells / the whole call (copies both
    ways, host planning between the passes), both from pinned host buffers.
    Under torchrun each rank traces its own batch (weak scaling); rank 0
    prints the units of all ranks over the slowest rank's time."""
    import torch
    from paper_2403_06478_gb300 import agatha as A
    from paper_2403_06478_gb300 import build as B
    from paper_2403_06478_gb300 import shard as S
    from paper_2403_06478_gb300 import workload as W
    rank, world, local = _env_int("RANK", 0), _env_int("WORLD_SIZE", 1), _env_int("LOCAL_RANK", 0)
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    B.build()
    batch = W.make_config(args.workload, seed=None if rank == 0 else W.SEED_BASE + 2 + 1000 * rank)
    pb = A.pack_batch(batch)
    pin = {k: torch.from_numpy(getattr(pb, k)).pin_memory() for k in
           ("q_packed", "t_packed", "q_off", "t_off", "q_len", "t_len")}
    pin_pb = A.PackedBatch(*[pin[k].numpy() for k in
                             ("q_packed", "t_packed", "q_off", "t_off", "q_len", "t_len")])
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    ctx = A.Context(local, timing=True, autotune=True, tune_cache_path=args.tune_cache)
    ctx.align_host(pb, batch.scoring)                     # autotune the score path
    for _ in range(args.warmup):
        res, off, cig = ctx.align_cigar(pin_pb, batch.scoring, stream=stream.cuda_stream)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    wall_ms, score_ms, tb_ms = [], [], []
    for k in range(args.steps):
        flush.fill_(k & 0xff)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res, off, cig = ctx.align_cigar(pin_pb, batch.scoring, stream=stream.cuda_stream)
        wall_ms.append((time.perf_counter() - t0) * 1e3)
        score_ms.append(ctx.last_kernel_ms())
        tb_ms.append(ctx.last_traceback_ms())
    torch.cuda.synchronize()
    clocks = sampler.stop()
    alone = A.agatha_align_batch(ctx, batch)
    exact = bool(A.results_equal(res, alone).size == 0)
    cells = int(res["cells"].sum())
    (all_cells, all_pairs), (k_tot, wall_tot) = S.reduce_step_stats(
        [cells, pb.n_pairs], [sum(score_ms) + sum(tb_ms), sum(wall_ms)], device="cuda")
    if rank != 0:
        ctx.close()
        if dist is not None:
            dist.destroy_process_group()
        return 0
    tcells = traceback_cells(res, batch)
    n = pb.n_pairs
    peaks, peak_kind = measured_peaks()
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    sm_max_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    int_peak = n_sm * 128 * sm_max_mhz * 1e6 / 1e12
    t_ms = statistics.mean(tb_ms)
    info = ctx.last_traceback_info()
    packed = info["pairs16"] > 0 and info["pairs32"] * 2 < info["pairs16"]
    fused = packed and info["fused"] * 2 > info["pairs16"]
    ops_cell = OPS_PER_CELL_TB16 if packed else OPS_PER_CELL_TB
    # the fused kernel computes the score path's cells (up to termination),
    # the two-pass kernels the cells up to each end cell
    units = cells if fused else tcells
    achieved = units * ops_cell / (t_ms / 1e3) / 1e12
    w = batch.scoring.w
    minb = dict([(4, 6), (8, 4), (16, 3), (24, 2)])
    nonempty = (batch.t_len > 0) & (batch.q_len > 0)
    if packed:
        C = next(c for c in (4, 8, 16, 24) if 32 * c - 1 >= w)
        kernel = f"{'tbf16' if fused else 'tb16'}_kernel<{C}, {minb[C]}>"
    else:
        C = next(c for c in (4, 8, 16, 24, 32) if 32 * c - 1 >= w)
        kernel = f"tb_kernel<{C}>"
    if fused:                 # room for every anti-diagonal of each pair
        table_bytes = int((batch.t_len[nonempty].astype(np.int64) + batch.q_len[nonempty] - 1).sum()) * 32 * C
    else:
        table_bytes = sum(((int(r["mqe_t"]) + int(batch.q_len[i]) - 1) if r["reach_end"] else
                           (int(r["te"]) + int(r["qe"]))) + 1 for i, r in enumerate(res)
                          if nonempty[i] and (r["reach_end"] or r["te"] >= 0)) * 32 * C
    line = {
        "metric": "GCUPS with traceback (score path + CIGAR of every extension), bit-exact",
        "value": round(all_cells * args.steps / (k_tot / 1e3) / 1e9, 3), "unit": "GCUPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(k_tot / args.steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "int16x2" if packed else "int32",
        "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload], "pairs_per_gpu": n, "cells_per_step": cells,
                   "traceback_cells_per_step": tcells, "cigar_runs_per_step": int(off[-1]),
                   "direction_table_bytes": int(table_bytes),
                   "l2": "flushed between steps (512 MB write)",
                   "value_basis": "score kernels + traceback kernels, CUDA events"},
        "pairs_per_s": round(all_pairs * args.steps / (k_tot / 1e3), 1),
        "score_kernel_ms": round(statistics.mean(score_ms), 3),
        "traceback_kernel_ms": round(t_ms, 3),
        "results_equal_score_path": exact,
        "e2e": {"value": round(all_cells * args.steps / (wall_tot / 1e3) / 1e9, 3), "unit": "GCUPS",
                "h2d_bytes_per_step": int(pin_pb.nbytes()),
                "d2h_bytes_per_step": int(n * 48 + 4 * n + 4 * int(off[-1])),
                "ms_per_step": round(wall_tot / args.steps, 3)},
        # score path (prep 3, 16-bit kernel, overflow kernel), one traceback
        # launch per wave, the CIGAR gather
        "gpu_launches": args.steps * (5 + info["waves"] + 1),
        "traceback_pairs": {"lanes16": info["pairs16"], "int32": info["pairs32"], "waves": info["waves"],
                            "fused": info["fused"]},
        "roofline": {"bound": "alu", "achieved": round(achieved, 3), "peak": round(int_peak, 3),
                     "unit": "Tops/s", "frac": round(achieved / int_peak, 4),
                     "traffic": traffic_tb16(kernel, table_bytes) if packed else None,
                     "units": "score cells" if fused else "cells up to each end cell",
                     "kernel": kernel, "kernel_ms": round(t_ms, 3),
                     "ops_per_cell": ops_cell,
                     "peak_basis": f"{n_sm} SMs x 128 int32 lanes x {sm_max_mhz:.0f} MHz ({peak_kind})"},
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    ctx.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--plain-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample-pairs", type=int, default=CPU_SAMPLE_PAIRS)
    ap.add_argument("--tune-cache", default=None,
                    help="autotuner cache file: read if present, written after tuning")
    ap.add_argument("--workload", default="ont", choices=sorted(WORKLOADS) + ["identical", "fixed"],
                    help="ont (the headline), or another configuration of the same metric "
                         "(identical / fixed: --profile-case only)")
    ap.add_argument("--profile-case", action="store_true",
                    help="run a small case for an ncu capture instead of the benchmark")
    ap.add_argument("--pairs", type=int, default=2000, help="--profile-case: pairs")
    ap.add_argument("--repeat", type=int, default=2, help="--profile-case: calls")
    ap.add_argument("--length", type=int, default=20000,
                    help="--profile-case: pair length of --workload identical / fixed")
    ap.add_argument("--path", default="batched", choices=PROFILE_PATHS,
                    help="--profile-case: kernel path")
    ap.add_argument("--traceback", action="store_true",
                    help="the path with CIGARs: score kernels + traceback kernel")
    ap.add_argument("--local", action="store_true",
                    help="the BWA-MEM variant: local extension from seed scores (agatha_align_batch_local)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.profile_case:
        return run_profile_case(args)
    if args.workload not in WORKLOADS:
        ap.error(f"--workload {args.workload} is only for --profile-case")
    if args.impl == "reference":
        return run_reference(args)
    if args.traceback:
        return run_traceback(args)
    if args.local:
        return run_local(args)

    import torch
    from paper_2403_06478_gb300 import agatha as A
    from paper_2403_06478_gb300 import build as B
    from paper_2403_06478_gb300 import workload as W

    rank, world, local = _env_int("RANK", 0), _env_int("WORLD_SIZE", 1), _env_int("LOCAL_RANK", 0)
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    B.build()

    # each rank aligns its own batch: rank 0 the standard workload, others reseeded
    batch = W.make_config(args.workload, seed=None if rank == 0 else W.SEED_BASE + 2 + 1000 * rank)
    pb = A.pack_batch(batch)
    n = pb.n_pairs
    ctx = A.Context(local, timing=True, autotune=True, tune_cache_path=args.tune_cache)
    # a dedicated stream: every launch, copy and timing event of the step sits on it
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    sh = stream.cuda_stream
    dev = {k: torch.from_numpy(getattr(pb, k)).to("cuda", non_blocking=False)
           for k in ("q_packed", "t_packed", "q_off", "t_off", "q_len", "t_len")}
    out = torch.empty(n * 48, dtype=torch.uint8, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")

    # the autotuner measures its variants on the first host batch of a scoring
    ctx.align_host(pb, batch.scoring)
    tuned = ctx.tune_variants(batch.scoring)

    def run_dev(flags):
        ctx.align_device(dev["q_packed"], dev["t_packed"], dev["q_off"], dev["t_off"], dev["q_len"],
                         dev["t_len"], out, batch.scoring, flags=flags | A.AGATHA_ASYNC, stream=sh)

    def timed(flags, steps, warmup, sampler=None):
        for _ in range(warmup):
            run_dev(flags)
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        if sampler:
            sampler.start()
        step_ms, kern_ms = [], []
        for k in range(steps):
            flush.fill_(k & 0xff)                      # evict L2 between steps (not timed)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            run_dev(flags)
            e1.record(stream)
            e1.synchronize()
            step_ms.append(e0.elapsed_time(e1))
            kern_ms.append(ctx.last_kernel_ms())
        torch.cuda.synchronize()
        clocks = sampler.stop() if sampler else None
        res = out.cpu().numpy().view(A.RESULT_DTYPE).copy()
        return step_ms, kern_ms, res, clocks

    sampler = ClockSampler(local)
    step_ms, kern_ms, res, clocks = timed(0, args.steps, args.warmup, sampler)
    cells = int(res["cells"].sum())
    plain_ms, plain_kern, plain_res, _ = timed(A.AGATHA_PLAIN, max(1, args.plain_steps), 1)
    bit_exact = bool(A.results_equal(res, plain_res).size == 0)

    # end to end: pinned host buffers through the C ABI, copies inside the timed region
    pin = {k: torch.from_numpy(getattr(pb, k)).pin_memory() for k in
           ("q_packed", "t_packed", "q_off", "t_off", "q_len", "t_len")}
    pin_pb = A.PackedBatch(*[pin[k].numpy() for k in
                             ("q_packed", "t_packed", "q_off", "t_off", "q_len", "t_len")])
    host_out = torch.empty(n * 48, dtype=torch.uint8).pin_memory().numpy().view(A.RESULT_DTYPE)
    for _ in range(args.warmup):
        ctx.align_host(pin_pb, batch.scoring, stream=sh, out=host_out)
    torch.cuda.synchronize()
    e2e_ms = []
    for k in range(args.steps):
        flush.fill_(k & 0xff)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.align_host(pin_pb, batch.scoring, stream=sh, out=host_out)
        e1.record(stream)
        e1.synchronize()
        e2e_ms.append(e0.elapsed_time(e1))
    e2e_exact = bool(A.results_equal(host_out, res).size == 0)
    h2d = pin_pb.nbytes()
    d2h = n * 48 + 32

    # aggregate over ranks: units all ranks processed / the slowest rank's time
    from paper_2403_06478_gb300 import shard as S
    (all_cells, all_pairs), (tot_ms, e2e_tot) = S.reduce_step_stats(
        [cells, n], [sum(step_ms), sum(e2e_ms)], device="cuda")
    value = all_cells * args.steps / (tot_ms / 1e3) / 1e9
    e2e_value = all_cells * args.steps / (e2e_tot / 1e3) / 1e9

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0

    peaks, peak_kind = measured_peaks()
    props = torch.cuda.get_device_properties(local)
    n_sm = props.multi_processor_count
    sm_max_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    int_peak = n_sm * 128 * sm_max_mhz * 1e6 / 1e12         # Tops/s of int32 lanes
    k_ms = statistics.mean(kern_ms)
    lane16 = res["lane16"].astype(bool)
    cells16 = int(res["cells"][lane16].sum())
    ops = cells16 * OPS_PER_CELL_I16X2 + (cells - cells16) * OPS_PER_CELL_I32
    achieved = ops / (k_ms / 1e3) / 1e12
    # the kernel the (tuned) plan launches: slots per lane from the band, the
    # resident blocks per SM from the register budget the tuner chose
    w = batch.scoring.w
    c16 = 4 if 0 < w <= 127 else (8 if 0 < w <= 255 else (16 if 0 < w <= 511 else 24))
    high = bool(tuned) and not tuned[4] and tuned[0] == 1
    minb = {4: (6, 4), 8: (4, 3), 16: (4, 3), 24: (3, 2)}[c16][1 if high else 0]
    kernel = f"warp16_align_kernel<{c16}, {minb}>" if cells16 * 2 > cells else "warp_align_kernel"
    # kernels per step: prep classify/scan/scatter, the warp kernel (one per
    # length class when the autotuner split the queue) and, with 16-bit lanes,
    # the int32 kernel over the (usually empty) overflow list
    split = bool(tuned and tuned[4])
    # on a 24-slot batch run as one launch of one warp per pair, the pairs
    # whose own band fits 640 slots take the 20-slot kernel beside it
    narrow = c16 == 24 and bool(lane16.any()) and not split and (not tuned or tuned[0] in (0, 1))
    weff = np.minimum(np.maximum(batch.t_len, batch.q_len), w if w > 0 else np.iinfo(np.int32).max)
    launches_per_step = 3 + (4 if split else 1) + (1 if narrow else 0) + (1 if lane16.any() else 0)
    line = {
        "metric": METRIC, "value": round(value, 3), "unit": "GCUPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(tot_ms / args.steps, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int16x2" if cells16 * 2 > cells else "int32",
        "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload], "pairs_per_gpu": n, "cells_per_step": cells,
                   "pairs_on_16bit_lanes": int(lane16.sum()),
                   "pairs_on_20_slot_frame": int((weff <= 638).sum()) if narrow else 0,
                   "autotune": None if tuned is None else
                   {"class_variants": [A.VARIANT_NAMES[v] for v in tuned[:4]], "split": split},
                   "l2": "flushed between steps (512 MB write)", "inputs": "resident in HBM"},
        "pairs_per_s": round(all_pairs * args.steps / (tot_ms / 1e3), 1),
        "plain": {"value": round(all_cells / (statistics.mean(plain_ms) / 1e3) / 1e9, 3)
                  if world == 1 else round(cells / (statistics.mean(plain_ms) / 1e3) / 1e9, 3),
                  "unit": "GCUPS", "ms_per_step": round(statistics.mean(plain_ms), 3),
                  "kernel_ms": round(statistics.mean(plain_kern), 3),
                  "pairs_per_s": round(n / (statistics.mean(plain_ms) / 1e3), 1)},
        "batched_vs_plain": round(statistics.mean(plain_ms) / (tot_ms / args.steps), 3),
        "bit_exact_batched_vs_plain": bit_exact,
        "e2e": {"value": round(e2e_value, 3), "unit": "GCUPS", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h), "bit_exact": e2e_exact,
                "ms_per_step": round(e2e_tot / args.steps, 3)},
        "gpu_launches": launches_per_step * args.steps,
        "roofline": {"bound": "alu", "achieved": round(achieved, 3),
                     "peak": round(int_peak, 3), "unit": "Tops/s", "frac": round(achieved / int_peak, 4),
                     "traffic": traffic_from_profile(kernel, h2d), "kernel": kernel,
                     "kernel_ms": round(k_ms, 3), "ops_per_cell": round(ops / max(cells, 1), 3),
                     "peak_basis": f"{n_sm} SMs x 128 int32 lanes x {sm_max_mhz:.0f} MHz ({peak_kind})"},
        "clocks": clocks,
    }
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(batch, args.cpu_sample_pairs, gpu_res=res)
        line["oracle_exact"] = line["cpu_baseline"]["oracle_exact"]
        line["oracle_checked_pairs"] = line["cpu_baseline"]["oracle_checked_pairs"]
    print(json.dumps(line), flush=True)
    ctx.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
