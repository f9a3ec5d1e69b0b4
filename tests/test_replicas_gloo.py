"""Multi-GPU path on the CPU: the benchmark runs one independent replica per rank (each rank
its own slice, no data-path collective) and takes the slowest rank's time; two gloo ranks
check the rank-to-slice map, the max-over-ranks timing and the whole-job throughput."""
import os

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
from paper_1608_03589_gb300 import synth


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # each rank's "measured" time; the job time is the maximum
        mine = 10.0 + 5.0 * rank
        total = bench.max_over_ranks(mine, dist, torch.device("cpu"))
        # replicas: each rank its own slice, different data
        wl = synth.SMALL
        g = wl.sinogram(slice_id=bench.replica_slice(rank))
        sums = [torch.zeros(1, dtype=torch.float64) for _ in range(world)]
        dist.all_gather(sums, torch.tensor([float(g.sum())], dtype=torch.float64))
        out[rank] = (total, [float(x) for x in sums])
    finally:
        dist.destroy_process_group()


def test_two_replicas_max_timing_and_distinct_slices():
    world, port = 2, 29500 + (os.getpid() % 2000)
    with mp.get_context("spawn").Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_worker, args=(world, port, out), nprocs=world, start_method="spawn")
        res = dict(out)
    assert res[0][0] == res[1][0] == 15.0           # slowest rank's time on every rank
    s0, s1 = res[0][1]
    assert s0 != s1                                 # the ranks backproject different slices
    # whole-job throughput: all ranks' updates over the slowest time
    upd = synth.LARGE.updates
    assert bench.throughput(upd, world, 4, 15.0) == pytest.approx(upd * 2 * 4 / 0.015 / 1e9)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    # under torchrun the oracle arm is timed by rank 0; other ranks return without work
    called = []

    class Args:
        warmup, steps = 0, 1

    import oracle
    monkeypatch.setattr(oracle, "filter_rows", lambda *a, **k: called.append("f"))
    bench.run_reference(Args(), 2, 1)
    assert called == []
