"""The N > 1 bench path on CPU: two gloo ranks, one replica each.

Each rank solves its own instance (no data-path collective); the whole-job
value is the sum of correct solves over the max of the rank times.
"""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    tot_ms = [120.0, 150.0][rank]
    ok = [3, 4][rank]
    v, t, n = bench.aggregate(dist, tot_ms, ok, device="cpu")
    q.put((rank, v, t, n))
    dist.destroy_process_group()


def test_two_rank_aggregate():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for _, v, t, n in res:
        assert t == 150.0 and n == 7
        assert v == pytest.approx(7 / 0.150)
