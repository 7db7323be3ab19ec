"""Density pre-solve on the GPU (lb_presolve) against the oracle's iteration, and its steady
state against the closed-form pressure of the Taylor-Green vortex (Sec. "Numerical
Simulations": consistent initial density and higher moments)."""
import math

import numpy as np
import pytest

import oracle
from paper_1507_02518_gb300 import lb, workloads

from test_gpu_parity import FP64_TOL, lattice

pytestmark = pytest.mark.gpu
NU_PRE = 1.0 / 6.0


@pytest.mark.parametrize("shape", [(12, 12, 12), (10, 9, 8), (33, 5, 4)])
@pytest.mark.parametrize("scheme", ["pull", "aa"])
@pytest.mark.parametrize("nu_pre", [NU_PRE, 0.01])
def test_fp64_iterations_match_oracle(kbc, shape, scheme, nu_pre):
    nx, ny, nz = shape
    rho, u0 = workloads.random_spectrum(nx, 2.0, 0.05, seed=4) if nx == ny == nz else (
        None, workloads.population_noise(nx, ny, nz, 9)[:3] * 0.05)
    iters = 40
    lat = lattice(shape, storage="f64", scheme=scheme)
    it, res = lat.presolve(u0, nu_pre=nu_pre, max_iters=iters, tol=-1.0)
    assert it == iters and lat.t == 0
    ref, it_ref, res_ref = oracle.presolve(u0, oracle.beta(nu_pre), iters)
    assert it_ref == iters
    err = np.max(np.abs(lat.get_populations() - ref))
    assert err <= FP64_TOL, err
    # the change is measured on rho - 1 rounded to FP32: two roundings of |rho - 1|
    r_ref, _ = oracle.macroscopic(ref)
    assert abs(res - res_ref) <= 2 * 2.0 ** -24 * 1.5 * float(np.max(np.abs(r_ref - 1))) + 1e-15


@pytest.mark.parametrize("storage,tol", [("f32", 2e-6), ("f16", 2e-4)])
def test_reduced_precision_iterations_track_oracle(kbc, storage, tol):
    _, u0 = workloads.taylor_green(16, 0.05)
    lat = lattice((16, 16, 16), storage=storage, scheme="aa")
    lat.presolve(u0, max_iters=64, tol=-1.0)
    ref, _, _ = oracle.presolve(u0, oracle.beta(NU_PRE), 64)
    W = oracle.lattice()[1].reshape(27, 1, 1, 1)
    err = np.max(np.abs(lat.get_populations() - ref) / W)
    assert err <= tol, err


@pytest.mark.parametrize("scheme", ["pull", "aa"])
def test_converges_to_taylor_green_pressure(kbc, scheme):
    N, nz, U = 32, 3, 0.005
    _, u0 = workloads.taylor_green_2d(N, nz, U)
    lat = lattice((N, N, nz), storage="f64", scheme=scheme)
    it, res = lat.presolve(u0, max_iters=6000, tol=1e-13)
    assert res <= 1e-13 and it < 6000 and it % 2 == 0
    f = lat.get_populations()
    r, _ = oracle.macroscopic(f)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(N), np.arange(N), indexing="ij")
    k = 2 * math.pi / N
    expect = 0.75 * U * U * (np.cos(2 * k * x) + np.cos(2 * k * y))
    assert np.max(np.abs(r - r.mean() - expect)) <= 0.02 * np.max(np.abs(expect))
    ref, _, _ = oracle.presolve(u0, oracle.beta(NU_PRE), 6000, tol=1e-14)
    assert np.max(np.abs(f - ref)) <= 1e-11


def test_host_and_device_u0_agree_and_state_steps(kbc):
    import torch
    _, u0 = workloads.kida(12, 0.05)
    a = lattice((12, 12, 12), storage="f32", scheme="pull")
    b = lattice((12, 12, 12), storage="f32", scheme="pull")
    ia = a.presolve(u0, max_iters=7, tol=-1.0)
    ib = b.presolve(torch.from_numpy(u0).cuda(), max_iters=7, tol=-1.0)
    assert ia == ib and ia[0] == 8                 # rounded up to an even count
    assert np.array_equal(a.get_populations(), b.get_populations())
    d = a.diagnostics()
    assert d["step"] == 0 and np.isnan(d["gamma_mean"])
    a.step(3)
    assert a.t == 3 and a.diagnostics()["nonfinite_count"] == 0


def test_arguments_are_validated(kbc):
    lat = lattice((8, 8, 8), storage="f64", scheme="aa")
    u0 = np.zeros((3, 8, 8, 8))
    for kw in ({"nu_pre": 0.0}, {"nu_pre": -1.0}, {"max_iters": -1}, {"tol": float("nan")}):
        with pytest.raises(lb.LBError) as e:
            lat.presolve(u0, **kw)
        assert e.value.status == lb.LB_ERR_INVALID_ARG
    it, res = lat.presolve(u0, max_iters=0)
    assert it == 0 and np.isnan(res)


def test_continuing_from_the_current_state_is_the_same_iteration(kbc):
    _, u0 = workloads.kida(12, 0.05)
    a = lattice((12, 12, 12), storage="f64", scheme="aa")
    a.presolve(u0, max_iters=20, tol=-1.0)
    b = lattice((12, 12, 12), storage="f64", scheme="aa")
    b.presolve(u0, max_iters=10, tol=-1.0)
    b.presolve(u0, max_iters=10, tol=-1.0, from_current=True)
    assert np.array_equal(a.get_populations(), b.get_populations())
    b.step(1)
    with pytest.raises(lb.LBError) as e:
        b.presolve(u0, max_iters=2, from_current=True)
    assert e.value.status == lb.LB_ERR_INVALID_ARG


def test_interpolated_density_start_converges_to_the_same_state(kbc):
    """The coarse-to-fine start of the pre-solve (table2.presolved_density) reaches the state a
    cold start reaches."""
    import torch
    from paper_1507_02518_gb300 import table2
    n = 32
    _, u = workloads.kida(n, 0.05)
    cold = lattice((n, n, n), storage="f64", scheme="aa")
    it_cold, _ = cold.presolve(u, max_iters=100000, tol=1e-13)
    rho_c = table2.presolved_density(16, "f64", 1e-13, min_n=16, log=lambda *a: None)
    warm = lattice((n, n, n), storage="f64", scheme="aa")
    warm.init_field(table2.interpolate_periodic(rho_c, n), torch.from_numpy(u).cuda())
    it_warm, _ = warm.presolve(u, max_iters=100000, tol=1e-13, from_current=True)
    print("cold %d iterations, warm %d" % (it_cold, it_warm))
    assert it_warm < it_cold
    assert np.max(np.abs(warm.get_populations() - cold.get_populations())) <= 1e-10
