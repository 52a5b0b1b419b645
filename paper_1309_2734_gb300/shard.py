"""Partition of independent hologram instances over ranks (one GPU per rank).

Holograms of a batch share nothing, so ranks split the instances and need no
collective on the data path.  Instances are assigned greedily, largest
W * H * N first, to the rank with the least work so far; the result is
deterministic and identical on every rank.
"""
from __future__ import annotations

from typing import List, Sequence


def shard_instances(costs: Sequence[float], rank: int, world: int) -> List[int]:
    """Indices of the instances rank `rank` of `world` computes, in ascending order."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    load = [0.0] * world
    owner = [0] * len(costs)
    for i in sorted(range(len(costs)), key=lambda k: (-float(costs[k]), k)):
        r = min(range(world), key=lambda q: (load[q], q))
        owner[i] = r
        load[r] += float(costs[i])
    return [i for i in range(len(costs)) if owner[i] == rank]
