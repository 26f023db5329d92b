"""Multi-process host logic of bench.py on CPU (gloo, world size 2).

Particles are independent (Eq. 1), so N GPUs run N replicas, each with its own
particles, and the only collective is the reduction of the timings: the
maximum of the ranks' timed regions and the sum of their particle-steps.  The
reference arm runs on rank 0 only.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        assert bench.dist_env() == (rank, world, rank)
        elapsed = [100.0, 250.0][rank]
        steps = [1_000_000, 3_000_000][rank]
        out[rank] = bench.reduce_over_ranks(elapsed, steps, torch.device("cpu"))
        # the reference arm does its work on rank 0 only; other ranks return at once
        if rank == 1:
            out["ref_rank1"] = bench.reference_arm(None, 1, world)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_ranks_reduce_max_time_and_sum_of_particle_steps():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
        assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
        assert out[0] == out[1] == (250.0, 4_000_000.0)
        assert out["ref_rank1"] is None


def test_single_process_reduction_is_the_identity():
    import bench
    assert bench.reduce_over_ranks(12.5, 7, torch.device("cpu")) == (12.5, 7.0)
