"""Multi-process (gloo, CPU) test of the batch sharding: every rank computes
its own share of the uneven batch; together the shares cover every instance
exactly once and the loads are balanced.  No GPU."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import synth
from paper_1501_02946_gb300 import shard


def _costs():
    return [shard.instance_cost(n * n, t, n, n, 2 * t) for (n, t) in synth.batch_shapes(1505, 64)]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = shard.shard_for_rank(_costs(), rank, world)
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    load = torch.tensor([sum(_costs()[i] for i in mine)], dtype=torch.float64)
    loads = [torch.zeros(1, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(loads, load)
    if rank == 0:
        out.put((gathered, [float(x.item()) for x in loads]))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_batch_shards_cover_and_balance(world):
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    gathered, loads = q.get()
    flat = sorted(i for part in gathered for i in part)
    costs = _costs()
    assert flat == list(range(len(costs)))
    assert max(loads) - min(loads) <= max(costs)
    assert max(loads) <= sum(costs) / world + max(costs)


def test_partition_single_rank_and_empty():
    assert shard.partition([3.0, 1.0, 2.0], 1) == [[0, 1, 2]]
    assert shard.partition([], 2) == [[], []]
    with pytest.raises(ValueError):
        shard.partition([1.0], 0)
