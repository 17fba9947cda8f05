"""The multi-rank path of the benchmark on CPU: two gloo ranks (one process
each, 127.0.0.1), every rank with its own replica of the workload.  The
whole job's time is the slowest rank's, its work the sum over ranks, and
the replicas are independent datasets (distinct seeds, no collective on the
data path)."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_1511_07482_gb300 import synthetic
    # rank r: time 10 + r ms, 100 (r + 1) evaluations; e2e 20 - r ms, 7 evaluations
    tot = bench.combine_ranks([10.0 + rank, 100 * (rank + 1), 20.0 - rank, 7], world)
    w = synthetic.small_case(n=50, d=2, M=16, seed=bench.rank_seed(2, rank))
    gathered = [None] * world
    dist.all_gather_object(gathered, float(w.X.sum()))
    out[rank] = (tot, gathered)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_combine_and_shard():
    import torch.multiprocessing as mp
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank_main, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
        res = dict(out)
    for r in range(world):
        tot, gathered = res[r]
        assert tot == [11.0, 300.0, 20.0, 14.0]
        assert gathered[0] != gathered[1]


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.combine_ranks([1.5, 2, 3.5, 4], 1) == [1.5, 2.0, 3.5, 4.0]
    assert bench.rank_seed(2, 0) == 2 and bench.rank_seed(2, 3) == 3002
    assert len({bench.rank_seed(4, r, 100000) for r in range(8)}) == 8
