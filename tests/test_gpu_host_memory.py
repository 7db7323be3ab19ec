"""Host-memory transfers of the C ABI: page-locked host buffers are read and written in place by
the kernels, pageable ones go through the staging area in chunks. Both routes (and the device
route) must give bitwise the same state and the same exported values, on ragged boxes and at
interior offsets of a page-locked allocation."""
import numpy as np
import pytest

from paper_1507_02518_gb300 import lb, workloads

from test_gpu_parity import lattice, seeded_state

pytestmark = pytest.mark.gpu

SHAPES = [(20, 13, 7), (33, 4, 5)]


def pinned_like(a, offset=0):
    """A page-locked copy of the float64 array a, starting `offset` values into a pinned
    allocation (an interior pointer); returns (numpy view, owner tensor)."""
    import torch
    owner = torch.empty(a.size + offset, dtype=torch.float64).pin_memory()
    view = owner.numpy()[offset:offset + a.size].reshape(a.shape)
    view[...] = a
    return view, owner


def pinned_empty(shape, offset=0):
    return pinned_like(np.zeros(shape), offset)


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("storage,scheme", [("f64", "pull"), ("f32", "aa"), ("f16", "aa")])
@pytest.mark.parametrize("offset", [0, 3])
def test_init_and_moments_through_pinned_memory(kbc, shape, storage, scheme, offset):
    nx, ny, nz = shape
    u = 0.05 * workloads.population_noise(nx, ny, nz, 5)[:3]
    rho = 1.0 + 0.01 * workloads.population_noise(nx, ny, nz, 6)[0]
    a = lattice(shape, storage=storage, scheme=scheme)
    b = lattice(shape, storage=storage, scheme=scheme)
    a.init_field(rho, u)                              # pageable: staged copies
    rho_p, _o1 = pinned_like(rho, offset)
    u_p, _o2 = pinned_like(u, offset)
    b.init_field(rho_p, u_p)                          # page-locked: read in place
    fa, fb = a.get_populations(), b.get_populations()
    assert np.array_equal(fa, fb)
    for lat in (a, b):
        lat.step(3)
    ra, ua = np.empty((nz, ny, nx)), np.empty((3, nz, ny, nx))
    lb.lb_moments(a.ctx, ra.ctypes.data, ua.ctypes.data, False)
    rb, _o3 = pinned_empty((nz, ny, nx), offset)
    ub, _o4 = pinned_empty((3, nz, ny, nx), offset)
    lb.lb_moments(b.ctx, rb.ctypes.data, ub.ctypes.data, False)
    assert np.array_equal(ra, rb) and np.array_equal(ua, ub)
    # rho = NULL (unit density) with a page-locked u
    b.init_field(None, u_p)
    a.init_field(None, u)
    assert np.array_equal(a.get_populations(), b.get_populations())


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("storage,scheme", [("f64", "aa"), ("f32", "pull"), ("f16", "aa")])
def test_populations_through_pinned_memory(kbc, shape, storage, scheme):
    import torch
    nx, ny, nz = shape
    f = seeded_state(nx, ny, nz, seed=8)
    a = lattice(shape, storage=storage, scheme=scheme)
    b = lattice(shape, storage=storage, scheme=scheme)
    lb.lb_set_time(a.ctx, 5)
    lb.lb_set_time(b.ctx, 5)                          # odd time: the AA export permutes
    a.set_populations(f)
    f_p, _o = pinned_like(f, 1)
    lb.lb_set_populations(b.ctx, f_p.ctypes.data, False)
    ga = a.get_populations()
    gb, _o2 = pinned_empty(f.shape, 2)
    lb.lb_get_populations(b.ctx, gb.ctypes.data, False)
    assert np.array_equal(ga, gb)
    # and the device route agrees
    gd = torch.empty((27, nx * ny * nz), dtype=torch.float64, device="cuda")
    lb.lb_get_populations(b.ctx, gd.data_ptr(), True)
    assert np.array_equal(gd.cpu().numpy().reshape(f.shape), ga)


@pytest.mark.parametrize("max_iters", [0, 6])
def test_presolve_from_pinned_velocity(kbc, max_iters):
    shape = (12, 10, 9)
    nx, ny, nz = shape
    u = 0.04 * workloads.population_noise(nx, ny, nz, 11)[:3]
    a = lattice(shape, storage="f32", scheme="aa")
    b = lattice(shape, storage="f32", scheme="aa")
    ia, resa = a.presolve(u, max_iters=max_iters, tol=-1.0)
    u_p, _o = pinned_like(u, 0)
    ib, resb = lb.lb_presolve(b.ctx, u_p.ctypes.data, False, 1.0 / 6.0, max_iters, -1.0, False)
    assert ia == ib == max_iters
    assert (np.isnan(resa) and np.isnan(resb)) or resa == resb
    assert np.array_equal(a.get_populations(), b.get_populations())
