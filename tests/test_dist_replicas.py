"""The multi-GPU path of bench.py is replicas (one independent scan per rank, no data-path collective):
check its host logic -- the max-over-ranks timing reduction, the whole-job rate and the reference arm
leaving ranks other than 0 without work -- with world_size 2 on the gloo backend, on CPU."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    try:
        assert bench.dist_env() == (rank, world, rank)
        dev_ms, wall, e2e = bench.reduce_timings([10.0 + 5.0 * rank, 1.0 - 0.5 * rank, 2.0 * rank], world,
                                                 torch.device("cpu"))
        out[rank] = (dev_ms, wall, e2e, bench.whole_job_rate(world, 16, 20, dev_ms))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_replica_timing_reduction_with_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_worker, args=(2, _free_port(), out), nprocs=2, start_method="spawn", join=True)
        res = dict(out)
    for rank in (0, 1):
        dev_ms, wall, e2e, rate = res[rank]
        assert dev_ms == 15.0 and wall == 1.0 and e2e == 2.0      # the max of each, on every rank
        assert rate == pytest.approx(2 * 16 * 20 / 0.015)


def test_reference_arm_other_ranks_do_no_work(monkeypatch):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("LOCAL_RANK", "1")

    class A:
        n, steps, warmup, gpus = 100_000, 1, 1, 2
    assert bench.run_reference(A()) is None
