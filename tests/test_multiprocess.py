"""N > 1 host logic of bench.py on CPU: two gloo ranks, each a replica with
its own timing; the job rate uses the slowest rank (max over ranks)."""
import os
import socket

import pytest
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
    t_local = 2.0 if rank == 0 else 4.0    # rank 1 is the slow replica
    value, t = bench.aggregate(t_local, steps=10, world=world, device="cpu")
    q.put((rank, value, t))
    dist.destroy_process_group()


def test_two_rank_aggregate_uses_slowest_rank():
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
    for rank, value, t in res:
        assert t == 4.0
        assert value == pytest.approx(2 * 10 / 4.0)


def test_single_rank_aggregate():
    import bench
    value, t = bench.aggregate(2.5, steps=5, world=1)
    assert t == 2.5 and value == pytest.approx(2.0)
