"""The multi-GPU path of the benchmark shards maps across ranks with no
data-path collective; its only exchange is the final reduction of timings and
counts.  Exercised here with two gloo ranks on CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as tdist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank r: its own map took (100 + 50 r) ms mixed, (200 - 10 r) ms plain and
    # converged (1000 + r) / (900 + 2 r) pixels
    times, counts = bench.reduce_over_ranks((100.0 + 50 * rank, 200.0 - 10 * rank),
                                            (1000 + rank, 900 + 2 * rank), "cpu")
    q.put((rank, times, counts))
    tdist.destroy_process_group()


def test_two_rank_reduction():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, times, counts in out:
        assert times == [150.0, 200.0]          # slowest rank
        assert counts == [2001, 1802]           # all ranks' pixels
