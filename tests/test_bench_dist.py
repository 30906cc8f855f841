"""bench.py's multi-rank reductions on two gloo ranks (CPU).

Under torchrun every rank times its own share of the work; the reported
figure is the slowest rank's time over all ranks' implicit steps, and only
rank 0 prints.  These tests run the same helpers on two CPU processes.
"""
import json
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, lr = bench.dist_env()
        assert (r, w, lr) == (rank, world, rank)
        # rank k: k+1 implicit steps taking 10*(k+1) ms each
        local_ms = [10.0 * (rank + 1)] * (rank + 1)
        per_step, t_max = bench.aggregate(local_ms, len(local_ms), world)
        mx = bench.reduce_max(float(rank) + 0.5, world)
        sm = bench.reduce_sum(float(rank) + 1.0, world)
        bench.barrier(world)

        class A:
            pass

        a = A()
        a.rank, a.world, a.local_rank = rank, world, rank
        ref_rc = bench.run_reference(a) if rank != 0 else 0  # other ranks exit without work
        with open(os.path.join(out_dir, "rank%d.txt" % rank), "w") as f:
            json.dump([per_step, t_max, mx, sm, ref_rc], f)
    finally:
        dist.destroy_process_group()


def test_aggregate_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp

    world = 2
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    for rank in range(world):
        per_step, t_max, mx, sm, ref_rc = json.load(open(tmp_path / ("rank%d.txt" % rank)))
        # slowest rank: 2 steps x 20 ms = 40 ms; 1 + 2 = 3 steps over the job
        assert t_max == pytest.approx(40.0)
        assert per_step == pytest.approx(40.0 / 3.0)
        assert mx == pytest.approx(1.5)
        assert sm == pytest.approx(3.0)
        assert ref_rc == 0


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.reduce_max(2.5, 1) == 2.5
    assert bench.reduce_sum(2.5, 1) == 2.5
    per_step, t_max = bench.aggregate([1.0, 3.0], 2, 1)
    assert t_max == 4.0 and per_step == 2.0
