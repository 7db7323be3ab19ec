"""One box split along z into 2 and 3 slab contexts on one GPU (the single-GPU form of the
multi-GPU split): after each step the library packs the 9 populations that cross each face,
the faces are copied into the neighbours' receive buffers, and the library unpacks them. The
slabs' gathered populations must equal the single-box run bit for bit (the collision is local
and the exchange moves stored values unchanged), in pull and AA, FP64, FP32 and FP16, with the
default and the row-staged kernels. The neighbour ring is periodic."""
import numpy as np
import pytest

import oracle
from paper_1507_02518_gb300 import lb, slab, workloads

from test_gpu_parity import lattice, seeded_state

pytestmark = pytest.mark.gpu


def gather(slabs):
    return np.concatenate([s.get_populations() for s in slabs], axis=1)


@pytest.mark.parametrize("storage", ["f64", "f32", "f16"])
@pytest.mark.parametrize("scheme", ["pull", "aa"])
@pytest.mark.parametrize("parts", [1, 2, 3])
@pytest.mark.parametrize("steps", [10, 11])
def test_slabs_equal_the_single_box_bitwise(kbc, storage, scheme, parts, steps):
    shape = (24, 16, 9)                     # slabs of 9, 5+4 and 3+3+3 planes
    f0 = seeded_state(*shape, seed=31)
    ref = lattice(shape, storage=storage, scheme=scheme)
    ref.set_populations(f0)
    ref.step(steps)
    slabs = slab.make_slabs(*shape, parts, storage=storage, scheme=scheme)
    for s in slabs:
        s.set_populations(f0[:, s.z0:s.z0 + s.nz_local])
    slab.step_local(slabs, steps)
    assert all(s.t == steps for s in slabs)
    assert np.array_equal(gather(slabs), ref.get_populations())


@pytest.mark.parametrize("storage", ["f32", "f16"])
@pytest.mark.parametrize("scheme", ["pull", "aa"])
@pytest.mark.parametrize("kind", ["packed", "rows", "adj"])
def test_slabs_with_each_fp32_kernel(kbc, storage, scheme, kind):
    shape = (64, 8, 12)                     # the rows kernel takes 4 rows of 64 nodes per tile
    f0 = seeded_state(*shape, seed=32)
    ref = lattice(shape, storage=storage, scheme=scheme)
    ref.set_kernel(kind)
    ref.set_populations(f0)
    ref.step(10)
    slabs = slab.make_slabs(*shape, 3, storage=storage, scheme=scheme)
    for s in slabs:
        s.set_kernel(kind)
        s.set_populations(f0[:, s.z0:s.z0 + s.nz_local])
    slab.step_local(slabs, 10)
    assert np.array_equal(gather(slabs), ref.get_populations())


@pytest.mark.parametrize("scheme", ["pull", "aa"])
@pytest.mark.parametrize("kind", ["packed", "adj"])
def test_slabs_with_nodes_recollided_in_fp64(kbc, scheme, kind):
    """1e-7 (relative) from equilibrium every FP32 node is re-collided in FP64 by the pass
    that follows each step kernel, the boundary planes' pass before their faces are packed:
    populations and gammas equal the single box's bit for bit."""
    n = 12
    rho, u = workloads.random_spectrum(n, 3, 0.04, seed=33)
    f0 = oracle.init_equilibrium(rho, u) * (1 + 1e-7 * workloads.population_noise(n, n, n, 34))
    ref = lattice((n, n, n), storage="f32", scheme=scheme)
    ref.set_kernel(kind)
    ref.set_populations(f0)
    ref.step(4)
    slabs = slab.make_slabs(n, n, n, 3, storage="f32", scheme=scheme)
    for s in slabs:
        s.set_kernel(kind)
        s.set_populations(f0[:, s.z0:s.z0 + s.nz_local])
    slab.step_local(slabs, 3)
    slab.step_local(slabs, 1, record=True)
    assert np.array_equal(gather(slabs), ref.get_populations())
    g = np.concatenate([lb_gamma(s) for s in slabs], axis=0)
    assert np.array_equal(g, ref.gamma())


def test_slab_init_moments_gamma_and_one_plane_slabs(kbc):
    """init_field and moments address the slab's own planes; slabs of one plane (both
    boundaries the same plane, no interior) work; gamma is recorded on request."""
    n = 12
    rho, u = workloads.random_spectrum(n, 3, 0.04, seed=5)
    ref = lattice((n, n, n), storage="f32", scheme="aa")
    ref.init_field(rho, u)
    ref.step(6)
    bounds = [(0, 1), (1, 5), (6, 1), (7, 5)]
    slabs = [slab.Slab(n, n, n, z0, k, storage="f32", scheme="aa") for z0, k in bounds]
    for s in slabs:
        s.init_field(rho[s.z0:s.z0 + s.nz_local], u[:, s.z0:s.z0 + s.nz_local])
    slab.step_local(slabs, 5)
    slab.step_local(slabs, 1, record=True)
    assert np.array_equal(gather(slabs), ref.get_populations())
    r_ref, u_ref = ref.moments()
    r = np.concatenate([s.moments()[0] for s in slabs], axis=0)
    assert np.array_equal(r, r_ref)
    g = np.concatenate([lb_gamma(s) for s in slabs], axis=0)
    assert np.array_equal(g, ref.gamma())


def lb_gamma(s):
    g = np.empty(s.shape, dtype=np.float32)
    lb.lb_get_gamma(s.ctx, g.ctypes.data, False)
    return g


def test_slab_call_order_is_enforced(kbc):
    s = slab.Slab(8, 8, 8, 0, 8, storage="f32", scheme="pull")
    with pytest.raises(lb.LBError):
        s.step_interior()                   # faces first
    s.step_faces()
    with pytest.raises(lb.LBError):
        s.get_populations()                 # the step is not complete
    with pytest.raises(lb.LBError):
        s.step_faces()
    s.step_interior()
    with pytest.raises(lb.LBError):
        s.step_faces()                      # unpack first
    s.recv_below.copy_(s.send_up)
    s.recv_above.copy_(s.send_down)
    s.unpack()
    with pytest.raises(lb.LBError):
        lb.lb_step(s.ctx, 1)                # whole-box calls
    with pytest.raises(lb.LBError):
        lb.lb_diagnostics(s.ctx)
    assert s.t == 1
