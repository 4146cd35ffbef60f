"""The multi-rank path of bench.py on CPU (gloo, world size 2): every rank
times its own replica, the job's time is the slowest rank's, and the value
counts the simulated seconds of all replicas."""
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


def _rank(rank, ws, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    ms = bench.max_over_ranks(100.0 + 50.0 * rank, dist, "cpu")
    out.put((rank, ms, bench.whole_job_value(ws, 5, 1.0, ms)))
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_take_the_slowest_rank():
    ws = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(ws))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, value in res:
        assert ms == 150.0
        assert value == pytest.approx(2 * 5 * 1.0 / 0.150)
    assert bench_alone() == 100.0


def bench_alone():
    import bench
    return bench.max_over_ranks(100.0, None, "cpu")
