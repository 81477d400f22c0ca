"""The benchmark's multi-rank bookkeeping on two gloo ranks (CPU): every rank
strokes its own batch (weak scaling, no collective on the data path) and the job
is timed by the slowest rank."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank-dependent timed regions: the job's time is the slowest rank's
    t = bench.max_over_ranks(10.0 + 5.0 * rank, "cpu")
    v = bench.job_throughput(1000, world, t)
    dist.barrier()
    q.put((rank, t, v))
    dist.destroy_process_group()


def test_two_rank_max_time_and_weak_scaling_throughput():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, v in res:
        assert t == pytest.approx(15.0)
        assert v == pytest.approx(2 * 1000 / 15e-3)


def test_single_process_passthrough():
    import bench
    assert bench.max_over_ranks(3.5, "cpu") == 3.5
    assert bench.job_throughput(100, 1, 10.0) == pytest.approx(1e4)


def _dying_worker(rank, world, port, q):
    import datetime
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=5))
    import bench
    dist.barrier()

    def report(what):
        q.put((rank, what))
        q.close()
        q.join_thread()  # flushed before the hard exit below

    if rank == 1:
        report("left")
        os._exit(0)  # leaves between steps, before the timing collective
    try:
        bench.max_over_ranks(10.0, "cpu")
        report("no error")
    except Exception:
        report("error")
    os._exit(0)


def test_a_rank_that_leaves_ends_the_timing_collective_with_an_error():
    """Failure detection on the host: when one rank exits between steps, the
    other's max-over-ranks collective raises within the process group's timeout
    instead of waiting forever."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_dying_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
    assert res == {0: "error", 1: "left"}
