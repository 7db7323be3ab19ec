"""One periodic box split along z over several GPUs (or several contexts on one GPU).

Each rank holds a slab of whole z-planes in a slab context of the library (``lb_slab_create``):
its planes plus one halo plane per side. The collision is local; eq:Egeneral's propagation
carries the 9 populations with v_z = +1 (-1) through the top (bottom) face of every slab each
step, so after each step a slab sends one 9-plane face to each neighbour and receives one from
each (9 nx ny stored values per face). The library steps the two boundary planes first and
packs the outgoing faces (``lb_slab_step_faces``), steps the other planes while the faces travel
(``lb_slab_step_interior``) and scatters the received faces (``lb_slab_unpack``); this module
only moves the face buffers: ``torch.distributed`` point-to-point (NCCL between GPUs) for one
slab per process, or device copies between slabs that live in the same process.

``slab_bounds`` (``sharding.py``) decides which planes each rank holds.
"""
from __future__ import annotations

import numpy as np

from . import lb
from .sharding import slab_bounds


class Slab:
    """Planes z0 .. z0 + nz_local - 1 of a periodic nx x ny x nz box; device memory is one torch
    uint8 tensor owned by this object, and the face buffers are views into it."""

    def __init__(self, nx, ny, nz, z0, nz_local, nu=1e-3, variant="d+t+q", gamma="estimate",
                 storage="f32", scheme="pull", stream=None, device=None):
        torch = lb._torch()
        self.cfg = lb.make_config(nx, ny, nz, nu, variant, gamma, storage, scheme)
        self.z0, self.nz_local = int(z0), int(nz_local)
        self.shape = (self.nz_local, ny, nx)
        self.nbytes = lb.lb_slab_required_bytes(self.cfg, nz_local)
        if self.nbytes == 0:
            raise lb.LBError(lb.LB_ERR_INVALID_ARG, "invalid slab")
        self.device = torch.device(device or "cuda")
        self.stream = stream or torch.cuda.current_stream(self.device)
        self.buf = lb._device_buffer(torch, self.nbytes, self.device, self.stream)
        self.ctx = lb.lb_slab_create(self.cfg, z0, nz_local, self.buf.data_ptr(), self.nbytes,
                                     self.stream.cuda_stream)
        ptrs, fb = lb.lb_slab_faces(self.ctx)
        base = self.buf.data_ptr()
        self.send_up, self.send_down, self.recv_below, self.recv_above = [
            self.buf[p - base:p - base + fb] for p in ptrs]

    def close(self):
        if getattr(self, "ctx", None):
            lb.lb_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def t(self) -> int:
        return lb.lb_time(self.ctx)

    def set_kernel(self, kind):
        lb.lb_set_kernel(self.ctx, lb.KERNEL[kind] if isinstance(kind, str) else kind)

    def step_faces(self, record=False):
        lb.lb_slab_step_faces(self.ctx, record)

    def step_interior(self):
        lb.lb_slab_step_interior(self.ctx)

    def unpack(self):
        lb.lb_slab_unpack(self.ctx)

    def init_field(self, rho, u):
        """rho [nz_local, ny, nx] (or None), u [3, nz_local, ny, nx]: this slab's planes."""
        torch = lb._torch()
        if isinstance(u, torch.Tensor) and u.is_cuda:
            u = u.to(torch.float64).contiguous()
            r = None if rho is None else rho.to(torch.float64).contiguous()
            lb.lb_init_field(self.ctx, 0 if r is None else r.data_ptr(), u.data_ptr(), True)
        else:
            u = np.ascontiguousarray(u, dtype=np.float64)
            r = None if rho is None else np.ascontiguousarray(rho, dtype=np.float64)
            lb.lb_init_field(self.ctx, 0 if r is None else r.ctypes.data, u.ctypes.data, False)

    def set_populations(self, f):
        f = np.ascontiguousarray(f, dtype=np.float64)
        assert f.shape == (27,) + self.shape
        lb.lb_set_populations(self.ctx, f.ctypes.data, False)

    def get_populations(self) -> np.ndarray:
        f = np.empty((27,) + self.shape)
        lb.lb_get_populations(self.ctx, f.ctypes.data, False)
        return f

    def moments(self):
        rho = np.empty(self.shape)
        u = np.empty((3,) + self.shape)
        lb.lb_moments(self.ctx, rho.ctypes.data, u.ctypes.data, False)
        return rho, u


def make_slabs(nx, ny, nz, parts, **kw):
    """All slabs of one box in this process (on one GPU: the single-GPU form of the split)."""
    bounds = [slab_bounds(nz, r, parts) for r in range(parts)]
    return [Slab(nx, ny, nz, z0, z1 - z0, **kw) for z0, z1 in bounds]


def step_local(slabs, n=1, record=False):
    """n steps of slabs that live in this process: faces, then interior, then each slab's
    outgoing faces copied into its neighbours' receive buffers (stream-ordered device copies;
    all slabs must share one stream), then unpack."""
    k = len(slabs)
    for _ in range(n):
        for s in slabs:
            s.step_faces(record)
        for s in slabs:
            s.step_interior()
        for j, s in enumerate(slabs):
            slabs[(j + 1) % k].recv_below.copy_(s.send_up)
            slabs[(j - 1) % k].recv_above.copy_(s.send_down)
        for s in slabs:
            s.unpack()


def exchange_ops(slab, rank, world, dist):
    """The point-to-point operations of one face exchange of rank `rank`: its top face goes to
    the rank above (periodic), its bottom face to the rank below; it receives the rank below's
    top face and the rank above's bottom face. With two ranks both neighbours are the same rank;
    each pair of messages keeps its order (sends and receives are posted in the same order)."""
    up, down = (rank + 1) % world, (rank - 1) % world
    return [dist.P2POp(dist.isend, slab.send_up, up),
            dist.P2POp(dist.irecv, slab.recv_below, down),
            dist.P2POp(dist.isend, slab.send_down, down),
            dist.P2POp(dist.irecv, slab.recv_above, up)]


def step_distributed(slab, rank, world, dist, n=1, record=False):
    """n steps of this rank's slab, one slab per process: the faces travel (NCCL between GPUs)
    while the interior planes are stepped."""
    for _ in range(n):
        slab.step_faces(record)
        if world == 1:
            slab.step_interior()
            slab.recv_below.copy_(slab.send_up)
            slab.recv_above.copy_(slab.send_down)
        else:
            reqs = dist.batch_isend_irecv(exchange_ops(slab, rank, world, dist))
            slab.step_interior()
            for r in reqs:
                r.wait()
        slab.unpack()
