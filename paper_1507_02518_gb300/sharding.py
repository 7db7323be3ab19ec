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
