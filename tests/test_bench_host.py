"""Host-side logic of bench.py: the max-over-ranks timing reduction used
when one process runs per GPU (checked here with two gloo ranks on CPU) and
the latency percentiles."""
import os
import socket

import numpy as np
import pytest

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # each rank reports its own step time; the job time is the slowest rank's
    got = bench.reduce_max(10.0 + 5.0 * rank, world)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, got))


def test_reduce_max_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert out == {0: 15.0, 1: 15.0}


def test_reduce_max_single_rank_is_identity():
    assert bench.reduce_max(3.5, 1) == 3.5


def test_percentiles():
    xs = np.arange(1, 101, dtype=float)
    p = bench.percentiles(xs)
    assert p["p50"] == pytest.approx(50.5)
    assert p["p99"] == pytest.approx(99.01)
    assert bench.percentiles([])["p50"] is None
