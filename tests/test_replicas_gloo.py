"""The replica bookkeeping of bench.py on two CPU ranks (gloo): the barrier
returns on both, the timed region is the slowest rank's, and the job's
throughput counts every replica's columns.  No GPU: the ranks are processes
on the host, rendezvous on 127.0.0.1."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, world: int, port: int, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    bench.rank_barrier(dist)
    seconds = [0.25, 0.5][rank]  # rank 1 is the slower one
    t = bench.rank_max(dist, seconds, "cpu")
    out.put((rank, t, bench.job_throughput(world, 1000, t)))
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    assert [r[1] for r in res] == [0.5, 0.5]
    assert all(r[2] == pytest.approx(2 * 1000 / 0.5) for r in res)


def test_single_process_needs_no_group():
    import bench

    bench.rank_barrier(None)
    assert bench.rank_max(None, 1.5, "cpu") == 1.5
    assert bench.job_throughput(1, 262144, 0.005) == pytest.approx(262144 / 0.005)
