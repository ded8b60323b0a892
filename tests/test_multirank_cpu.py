"""The multi-rank host logic of bench.py on CPU: two gloo ranks (one process
each, 127.0.0.1 rendezvous) run the same helpers bench.py runs under NCCL on
the GPUs: the max-over-ranks reduction of the step time, the whole-job
throughput of the replicas, and each rank's own replica seeds."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import sys

    sys.path.insert(0, ROOT)
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import torch.distributed as dist

    import bench
    from paper_2603_09668_gb300 import inputs

    dist.init_process_group("gloo", rank=rank, world_size=world)
    w, r, _ = bench.dist_env()
    ms = 10.0 + 5.0 * rank  # rank 1 is the slow one
    ms_max = bench.reduce_max(ms)
    sc = inputs.sheet_scene(nu=20, nv=14, n_grid=32, n_substeps=10, **bench.replica_seeds(rank))
    out[rank] = (w, r, ms_max, bench.job_value(1000, w, ms_max), sc.n, float(sc.wind.sum()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_max_and_weak_scale():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    assert sorted(res) == [0, 1]
    for rank, (w, r, ms_max, value, n, _) in res.items():
        assert (w, r) == (world, rank)
        assert ms_max == 15.0  # the slowest rank's time on every rank
        assert value == pytest.approx(1000 * world / 15e-3)
    assert res[0][4] == res[1][4]  # the same workload shape
    assert res[0][5] != res[1][5]  # each replica has its own wind field


def test_one_rank_needs_no_process_group(monkeypatch):
    import sys

    sys.path.insert(0, ROOT)
    import bench

    monkeypatch.setenv("WORLD_SIZE", "1")
    assert bench.reduce_max(3.5) == 3.5
    assert bench.job_value(100, 1, 2.0) == pytest.approx(5e4)
    assert np.isfinite(bench.job_value(1, 8, 1.0))
