"""Assignment of independent boxes to ranks (one process per GPU).

The batched ensemble has no data exchange between boxes, so it shards with no collective on
the data path: boxes go to ranks by longest-processing-time first on their node counts
(N_b^3), each rank steps its own boxes, and only diagnostics or timings are gathered.
"""
from __future__ import annotations

import heapq


def lpt_assign(costs, nranks: int):
    """Greedy LPT: visit boxes by decreasing cost, give each to the least-loaded rank.

    Returns a list (one per rank) of box indices in increasing order. Ties break on the lower
    rank and the lower box index, so every rank computes the same assignment.
    """
    if nranks < 1:
        raise ValueError("nranks must be >= 1")
    order = sorted(range(len(costs)), key=lambda b: (-costs[b], b))
    heap = [(0, r) for r in range(nranks)]
    out = [[] for _ in range(nranks)]
    for b in order:
        load, r = heapq.heappop(heap)
        out[r].append(b)
        heapq.heappush(heap, (load + costs[b], r))
    return [sorted(v) for v in out]


def box_cost(box) -> int:
    n = box["n"]
    return int(n) * int(box.get("ny", n)) * int(box.get("nz", n))


def shard_boxes(boxes, rank: int, world: int):
    """The boxes (and their global indices) that `rank` of `world` steps."""
    mine = lpt_assign([box_cost(b) for b in boxes], world)[rank]
    return [boxes[b] for b in mine], mine


# ---------------------------------------------------------------- slab decomposition of one box
# A single box split along z into one slab of whole planes per rank. Collision is local; the
# propagation of eq:Egeneral needs, across each slab face, the post-collision populations that
# cross it: the 9 directions with v_z = +1 leave the top plane upwards and the 9 with v_z = -1
# leave the bottom plane downwards (velocity index i = (vx+1) + 3(vy+1) + 9(vz+1)).
UP = tuple(range(18, 27))      # v_z = +1
DOWN = tuple(range(0, 9))      # v_z = -1


def slab_bounds(nz: int, rank: int, world: int):
    """Planes [z0, z1) of `rank`'s slab: nz split as evenly as possible, the first nz % world
    ranks holding one plane more."""
    if world < 1 or not 0 <= rank < world or nz < world:
        raise ValueError("need 0 <= rank < world <= nz")
    q, r = divmod(nz, world)
    z0 = rank * q + min(rank, r)
    return z0, z0 + q + (1 if rank < r else 0)


def slab_neighbours(rank: int, world: int):
    """(rank below, rank above) on the periodic ring of slabs."""
    return (rank - 1) % world, (rank + 1) % world
