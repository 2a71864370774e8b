"""Multi-rank host logic of the sharded ensemble, on CPU with gloo (world size 2)."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2404_17754_gb300 import shard


def test_assign_is_a_balanced_partition():
    costs = [5.6, 0.56, 2.9, 1.1, 1.7, 0.9, 2.2, 0.6, 1.4, 2.95]
    for world in (1, 2, 3, 4):
        shares = shard.assign(costs, world)
        flat = sorted(i for s in shares for i in s)
        assert flat == list(range(len(costs)))
        loads = [sum(costs[i] for i in s) for s in shares]
        assert max(loads) - min(loads) <= max(costs)  # greedy bound
    assert shard.assign(costs, 2) == shard.assign(list(costs), 2)  # deterministic


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, costs, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = shard.assign(costs, world)[rank]
    # each rank "runs" its analyses: time = its load, ERR = a function of the index
    t = sum(costs[i] for i in mine)
    t_max = shard.max_over_ranks(t, dist)
    table = shard.gather_table({i: 0.1 * i for i in mine}, dist)
    q.put((rank, mine, t_max, sorted(table.items())))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_sharding_with_gloo():
    costs = [3.0, 1.0, 2.0, 2.5, 0.5, 1.5]
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, costs, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res.sort()
    shares = [r[1] for r in res]
    assert sorted(shares[0] + shares[1]) == list(range(len(costs)))
    loads = [sum(costs[i] for i in s) for s in shares]
    for r in res:
        assert r[2] == pytest.approx(max(loads))
        assert r[3] == [(i, 0.1 * i) for i in range(len(costs))]
