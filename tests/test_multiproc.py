"""The multi-rank path of bench.py (replicas, no data collective) on CPU: two gloo ranks,
each with its own timed duration; the job value is all steps over the slowest rank."""

import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    total = [2.0, 3.0][rank]  # rank 1 is the slow one
    value, t = bench.combine_ranks(total, 10, world, device="cpu")
    out.put((rank, value, t))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    mp = pytest.importorskip("torch.multiprocessing")
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
    for rank, value, t in res:
        assert t == 3.0
        assert value == pytest.approx(2 * 10 / 3.0)


def test_single_rank_is_plain():
    import bench
    v, t = bench.combine_ranks(4.0, 8, 1)
    assert v == 2.0 and t == 4.0
