"""Multi-rank host logic on CPU: two gloo ranks split a batch of holograms.

Each rank takes its share of the instances; all-gathering the shares shows
that together they cover every instance exactly once and that the work is
balanced.  No GPU and no data-path collective is involved.
"""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1309_2734_gb300 import workloads
from paper_1309_2734_gb300.shard import shard_instances


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, costs, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = shard_instances(costs, rank, world)
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    if rank == 0:
        out.put(gathered)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_cover_the_batch():
    batch = workloads.video_batch(n_instances=64)
    costs = [c.evals for c in batch]
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, costs, q)) for r in range(2)]
    for p in procs:
        p.start()
    shares = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    flat = sorted(i for s in shares for i in s)
    assert flat == list(range(64))
    loads = [sum(costs[i] for i in s) for s in shares]
    assert max(loads) / min(loads) < 1.1


def test_shard_single_rank_and_errors():
    assert shard_instances([3, 1, 2], 0, 1) == [0, 1, 2]
    with pytest.raises(ValueError):
        shard_instances([1], 2, 2)
