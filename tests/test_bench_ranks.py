"""bench.py's replica reduction across ranks (slowest time, summed codewords), with two gloo
ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=2)
    import bench
    secs, cw = bench.reduce_over_ranks(1.0 + rank, 10 ** 12 * (rank + 1), "cpu")
    out[rank] = (secs, cw)
    dist.destroy_process_group()


def test_reduce_over_two_ranks():
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert out[0] == out[1] == (2.0, 3 * 10 ** 12)


def test_reduce_single_process_is_identity():
    import bench
    assert bench.reduce_over_ranks(3.5, 7, "cpu") == (3.5, 7)
