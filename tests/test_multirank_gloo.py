"""The N > 1 path of bench.py on CPU: two gloo ranks, each with its own
replicate, the slowest rank's time for the whole job, and the reference arm
run by rank 0 alone."""
import os
import socket
import sys

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, local = bench.dist_env()
        ms_local = 100.0 + 37.0 * r            # rank 1 is the slow one
        ms_max = bench.max_over_ranks(ms_local)
        rate = bench.whole_job_rate(w, 5, ms_max)
        from paper_1701_05936_gb300 import synth
        prob = synth.gaussian_ar1(n=40, p=60, k=3, dtype="f32", workload=2, replicate=r)
        dist.barrier()
        out[rank] = (r, w, local, ms_max, rate, float(np.asarray(prob.y).sum()))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_time_the_job_by_the_slowest_rank():
    world = 2
    out = mp.Manager().dict()
    mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
    assert sorted(out.keys()) == [0, 1]
    for rank in range(world):
        r, w, local, ms_max, rate, ysum = out[rank]
        assert (r, w, local) == (rank, world, rank)
        assert ms_max == 137.0                       # the max over ranks, on every rank
        assert rate == world * 5 / 0.137             # units of all ranks / the slowest time
    assert out[0][5] != out[1][5]                    # each rank fits its own replicate


def test_one_rank_is_its_own_max():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5) == 12.5
    assert bench.whole_job_rate(1, 10, 2000.0) == 5.0


def test_reference_arm_exits_on_other_ranks(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1"])
    assert bench.run_reference(bench.parse()) == 0   # returns before any work or output
