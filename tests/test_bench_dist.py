"""The multi-rank path of bench.py on CPU: world size 2 over gloo.  Every
rank runs an independent replica (the chain problems are independent), so
the only collective is the max-over-ranks of the timed duration."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    q.put((rank, bench.max_over_ranks(1.5 + rank, torch.device("cpu")), bench._dist()))
    dist.destroy_process_group()


def test_max_over_ranks_world_size_two():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = [q.get(timeout=120) for _ in ps]
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, m, (world, r, local) in out:
        assert m == 2.5 and world == 2 and r == rank


def test_single_process_max_is_identity():
    import bench
    assert bench.max_over_ranks(3.25, torch.device("cpu")) == 3.25
