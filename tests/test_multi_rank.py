"""Multi-GPU host logic on CPU: the LPT split, the result gather and the step
statistics reduction, run as two gloo ranks.  The per-rank alignment is done
by the CPU oracle here (this machine has no GPU); on GPUs each rank runs the
library on its own device with the same split and the same gather."""
import os
import socket

import numpy as np
import pytest

from paper_2403_06478_gb300 import shard as S
from paper_2403_06478_gb300 import workload as W


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    try:
        import torch.distributed as dist
        from oracle import oracle as O
        os.environ["MASTER_ADDR"] = "127.0.0.1"
        os.environ["MASTER_PORT"] = str(port)
        dist.init_process_group("gloo", rank=rank, world_size=world)
        batch = W.make_config("small", n_pairs=48)
        idx = S.shard_indices(batch.q_len, batch.t_len, batch.scoring.w, rank, world)
        local = O.align_batch(batch, idx=idx, threads=1)
        full = S.gather_results(local, idx, batch.n_pairs)
        sums, maxes = S.reduce_step_stats([int(local["cells"].sum()), idx.size], [10.0 + rank])
        ok = True
        if rank == 0:
            ref = O.align_batch(batch, threads=1)
            ok &= all(np.array_equal(full[f], ref[f]) for f in O.COMPARE_FIELDS)
            ok &= sums == [float(ref["cells"].sum()), float(batch.n_pairs)]
            ok &= maxes == [10.0 + world - 1]
        dist.barrier()
        dist.destroy_process_group()
        q.put((rank, bool(ok), ""))
    except Exception as e:  # reported to the parent
        q.put((rank, False, repr(e)))


def test_two_gloo_ranks_split_gather_and_reduce():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=240) for _ in procs]
    for p in procs:
        p.join(timeout=60)
    assert all(p.exitcode == 0 for p in procs)
    for rank, ok, err in sorted(out):
        assert ok, f"rank {rank}: {err}"


def test_lpt_split_is_a_partition_and_balanced():
    rng = np.random.default_rng(3)
    for n_items, world in ((0, 2), (5, 8), (100, 2), (1000, 3), (5000, 8)):
        work = rng.pareto(1.5, n_items) * 1000 + 1
        work = work.astype(np.int64)
        parts = S.lpt_partition(work, world)
        assert len(parts) == world
        allidx = np.concatenate(parts) if n_items else np.array([], np.int64)
        assert np.array_equal(np.sort(allidx), np.arange(n_items))
        if n_items:
            loads = [int(work[p].sum()) for p in parts]
            # Graham's bound for LPT: at most 4/3 of the optimum
            assert max(loads) <= 4.0 / 3.0 * S.lower_bound(work, world) + 1


def test_lpt_beats_equal_counts_on_skewed_lengths():
    batch = W.make_config("skewed", n_pairs=4000)
    work = S.predicted_cells(batch.q_len, batch.t_len, batch.scoring.w)
    lpt = S.load_imbalance(work, S.lpt_partition(work, 4))
    equal = S.load_imbalance(work, np.array_split(np.arange(batch.n_pairs), 4))
    assert lpt <= equal
    assert lpt < 1.01


def test_predicted_cells_matches_band_count_shape():
    # the estimate is the band-cell count of a square pair up to the corner triangles
    q = np.array([1000, 0, 10, 5000])
    t = np.array([1000, 5, 10, 4000])
    est = S.predicted_cells(q, t, 100)
    assert est[1] == 0
    assert est[0] == 2000 * 101 // 2
    assert est[2] == 20 * 11 // 2          # band wider than the pair: w becomes the length
    assert est[3] > est[0]


@pytest.mark.gpu
def test_sharded_on_one_gpu_equals_whole_batch():
    from paper_2403_06478_gb300 import agatha as A
    from paper_2403_06478_gb300 import build as B
    B.build()
    batch = W.make_config("skewed", n_pairs=600)
    with A.Context(0) as ctx:
        whole = A.agatha_align_batch(ctx, batch)
        for n in (2, 3, 8):
            assert A.results_equal(S.align_sharded(ctx, batch, n), whole).size == 0
