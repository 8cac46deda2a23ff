"""The N > 1 path of bench.py on CPU: world_size-2 gloo process group (replicas only: every rank
solves its own problem; the only collectives are the barrier and the max-over-ranks timing)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = [120.0, 180.0][rank]          # the ranks' own timed regions
    mx = bench.max_over_ranks(local_ms, dist, "cpu")
    val = bench.whole_job_value(1_000_000, 4, world, mx)
    dist.barrier()
    # the reference arm: rank 0 alone runs it, the others return without work
    ran = None
    if rank != 0:
        class A:  # arguments that would make rank 0 work; rank 1 must not touch them
            steps = 1
            gpus = world
        ran = bench.run_reference(A(), rank, world)
    q.put((rank, mx, val, ran))
    dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_value_with_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, mx, val, ran in res:
        assert mx == 180.0                              # every rank sees the slowest rank's time
        assert val == pytest.approx(1_000_000 * 4 * 2 / 0.18 / 1e9)
    assert res[1][3] is None                            # rank 1 did no reference work


def test_single_process_has_no_collective():
    import bench
    assert bench.max_over_ranks(42.5) == 42.5
    assert bench.whole_job_value(10, 2, 1, 20.0) == pytest.approx(10 * 2 / 0.02 / 1e9)
