"""The multi-rank host logic on CPU: two gloo ranks (127.0.0.1) split a global ensemble draw and reduce
their timings, as bench.py does over NCCL with one rank per GPU."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist
    from paper_1107_4650_gb300 import distributed as PD
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        runs, idx, _ = PD.ensemble_shard(24, rank, world)
        cost = sum(PD.run_cost(r) for r in runs)
        gathered = [None] * world
        dist.all_gather_object(gathered, (idx, cost))
        slowest = PD.max_over_ranks(10.0 + rank, world)
        np.save(os.path.join(out_dir, "rank%d.npy" % rank),
                np.array([len(runs), cost, slowest], dtype=np.float64))
        if rank == 0:
            all_idx = sorted(i for ids, _ in gathered for i in ids)
            costs = [c for _, c in gathered]
            np.save(os.path.join(out_dir, "gather.npy"), np.array(all_idx))
            np.save(os.path.join(out_dir, "costs.npy"), np.array(costs))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_split_the_ensemble_and_reduce_timings(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    per_rank = [np.load(tmp_path / ("rank%d.npy" % r)) for r in range(world)]
    all_idx = np.load(tmp_path / "gather.npy")
    costs = np.load(tmp_path / "costs.npy")
    assert list(all_idx) == list(range(24 * world))          # disjoint and complete
    assert all(int(p[0]) == 24 for p in per_rank)             # equal counts
    assert abs(costs[0] - costs[1]) / costs.max() < 0.1       # balanced work
    assert all(p[2] == 11.0 for p in per_rank)                # every rank sees the slowest time


def test_single_rank_shard_is_the_whole_draw():
    from paper_1107_4650_gb300 import distributed as PD
    from paper_1107_4650_gb300 import workloads as W
    runs, idx, _ = PD.ensemble_shard(16, 0, 1)
    ref, _ = W.klein_ensemble(nruns=16)
    assert idx == list(range(16)) and [r.side for r in runs] == [r.side for r in ref]
    with pytest.raises(ValueError):
        PD.ensemble_shard(4, 2, 2)
