"""Multi-rank host logic on CPU (gloo, world_size 2): box sharding and bench timing reduction."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1507_02518_gb300 import sharding, workloads


def test_lpt_partitions_and_balances():
    boxes = workloads.batch_boxes(96)
    costs = [sharding.box_cost(b) for b in boxes]
    for world in (1, 2, 4, 8):
        parts = sharding.lpt_assign(costs, world)
        flat = sorted(b for p in parts for b in p)
        assert flat == list(range(96))
        loads = [sum(costs[b] for b in p) for p in parts]
        # LPT is within 4/3 of optimal; the mean is a lower bound of the optimum
        assert max(loads) <= 4.0 / 3.0 * (sum(loads) / world) + max(costs)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank), KBC_BENCH_BACKEND="gloo")
    import bench
    r, w, _ = bench.dist_init(world)
    boxes = workloads.batch_boxes(96)
    mine, idx = sharding.shard_boxes(boxes, r, w)
    nodes = float(sum(sharding.box_cost(b) for b in mine))
    total = bench.sum_over_ranks(nodes, w)
    slowest = bench.max_over_ranks(1.0 + r, w)
    import torch
    gathered = [None] * w
    dist.all_gather_object(gathered, idx)
    q.put((r, total, slowest, gathered))
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_without_overlap():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    boxes = workloads.batch_boxes(96)
    expect_total = float(sum(sharding.box_cost(b) for b in boxes))
    for r, total, slowest, gathered in res:
        assert total == expect_total
        assert slowest == 2.0
        flat = sorted(b for part in gathered for b in part)
        assert flat == list(range(96))
