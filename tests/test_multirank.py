"""The N > 1 host path (q-point sharding, max-over-ranks timing) on CPU with gloo, world size 2."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2509_23018_gb300.shard import max_over_ranks, qpoint_shard  # noqa: E402


def test_shards_disjoint_and_balanced():
    costs = [3000 ** 2, 300 ** 2, 1500 ** 2, 2500 ** 2, 800 ** 2, 1200 ** 2, 2900 ** 2]
    for world in (1, 2, 3, 4):
        got = [qpoint_shard(costs, r, world) for r in range(world)]
        flat = sorted(i for s in got for i in s)
        assert flat == list(range(len(costs)))
        loads = [sum(costs[i] for i in s) for s in got]
        assert max(loads) <= sum(costs) / world + max(costs)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    costs = [5.0, 1.0, 4.0, 2.0, 3.0]
    mine = qpoint_shard(costs, rank, world)
    t = max_over_ranks(10.0 + rank)
    got = [None] * world
    dist.all_gather_object(got, mine)
    out[rank] = (t, got)
    dist.destroy_process_group()


def test_gloo_two_ranks():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    for rank in (0, 1):
        t, shards = res[rank]
        assert t == 11.0  # max over ranks
        assert sorted(shards[0] + shards[1]) == [0, 1, 2, 3, 4]
        assert not set(shards[0]) & set(shards[1])
