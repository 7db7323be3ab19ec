"""The slab decomposition of one box along z (the multi-GPU design for a single box), run as
gloo ranks on CPU with the oracle doing the arithmetic: each rank collides its planes,
exchanges the 9 populations per face that cross it, and propagates with those halo planes.
The gathered result must equal the single-domain oracle bit for bit."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_1507_02518_gb300 import sharding, workloads

V, W = oracle.lattice()
SHAPE = (7, 6, 9)        # nx, ny, nz
STEPS = 5
NU = 2e-3


def initial_state():
    nx, ny, nz = SHAPE
    return W.reshape(27, 1, 1, 1) * (1 + 0.02 * workloads.population_noise(nx, ny, nz, 13))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _slab_step(f, beta, rank, world):
    """One collide-and-propagate step of a slab f[27, nloc, ny, nx] with halo exchange."""
    import torch
    fpost, _, _ = oracle.collide_field(f, beta)
    down, up = sharding.slab_neighbours(rank, world)
    nloc, ny, nx = f.shape[1:]
    send_up = torch.from_numpy(np.ascontiguousarray(fpost[list(sharding.UP), -1]))
    send_down = torch.from_numpy(np.ascontiguousarray(fpost[list(sharding.DOWN), 0]))
    from_down = torch.empty_like(send_up)       # the plane below, directions moving up
    from_up = torch.empty_like(send_down)       # the plane above, directions moving down
    reqs = [dist.isend(send_up, up), dist.isend(send_down, down),
            dist.irecv(from_down, down), dist.irecv(from_up, up)]
    for q in reqs:
        q.wait()
    ext = np.zeros((27, nloc + 2, ny, nx))
    ext[:, 1:-1] = fpost
    ext[list(sharding.UP), 0] = from_down.numpy()
    ext[list(sharding.DOWN), -1] = from_up.numpy()
    out = np.empty_like(f)
    for i in range(27):
        vx, vy, vz = V[i]
        shifted = np.roll(ext[i], shift=(vy, vx), axis=(1, 2))     # periodic in y and x
        out[i] = shifted[1 - vz: 1 - vz + nloc]                    # f_i(z) = f'_i(z - v_z)
    return out


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    nz = SHAPE[2]
    z0, z1 = sharding.slab_bounds(nz, rank, world)
    f = np.ascontiguousarray(initial_state()[:, z0:z1])
    beta = oracle.beta(NU)
    for _ in range(STEPS):
        f = _slab_step(f, beta, rank, world)
    slabs = [None] * world
    dist.all_gather_object(slabs, (z0, z1, f))
    q.put((rank, slabs))
    dist.destroy_process_group()


def test_slab_bounds_cover_the_box():
    for nz in (3, 8, 9, 100):
        for world in range(1, min(nz, 8) + 1):
            bounds = [sharding.slab_bounds(nz, r, world) for r in range(world)]
            assert bounds[0][0] == 0 and bounds[-1][1] == nz
            assert all(a[1] == b[0] for a, b in zip(bounds, bounds[1:]))
            sizes = [b - a for a, b in bounds]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        sharding.slab_bounds(2, 0, 3)


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_ranks_reproduce_the_single_domain_bitwise(world):
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=180) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    ref, _, _ = oracle.run(initial_state(), STEPS, oracle.beta(NU))
    for _, slabs in res:
        got = np.concatenate([f for _, _, f in sorted(slabs, key=lambda s: s[0])], axis=1)
        assert np.array_equal(got, ref)
