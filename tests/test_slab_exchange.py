"""Routing of the slab faces between ranks (paper_1507_02518_gb300/slab.py) on gloo ranks on
CPU: every rank's top face must land in the receive-from-below buffer of the rank above and its
bottom face in the receive-from-above buffer of the rank below, on a periodic ring of 1, 2 and
3 ranks (with 2 ranks both neighbours are the same rank)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1507_02518_gb300 import slab


class FakeFaces:
    """The four face buffers of a slab, as CPU tensors tagged with their owner and side."""

    def __init__(self, rank, n=5):
        self.send_up = torch.full((n,), 100.0 * rank + 1)
        self.send_down = torch.full((n,), 100.0 * rank + 2)
        self.recv_below = torch.zeros(n)
        self.recv_above = torch.zeros(n)


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
    try:
        f = FakeFaces(rank)
        for _ in range(2):                       # twice: the ordering holds step after step
            for r in dist.batch_isend_irecv(slab.exchange_ops(f, rank, world, dist)):
                r.wait()
        out[rank] = (float(f.recv_below[0]), float(f.recv_above[0]))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_faces_reach_the_neighbours(world):
    out = mp.Manager().dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    for r in range(world):
        below, above = (r - 1) % world, (r + 1) % world
        assert out[r] == (100.0 * below + 1, 100.0 * above + 2)
