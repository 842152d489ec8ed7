"""bench.py's multi-rank aggregation (max of times, sum of units over ranks),
run as two gloo ranks on CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t, u = bench.reduce_max_sum((10.0 + rank, 100.0 * (rank + 1)), world, torch.device("cpu"))
    out[rank] = (t, u)
    dist.destroy_process_group()


def test_reduce_max_sum_two_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert out[0] == (11.0, 300.0) and out[1] == (11.0, 300.0)


def test_single_rank_is_identity():
    import bench
    assert bench.reduce_max_sum((3.0, 4.0), 1, None) == (3.0, 4.0)
