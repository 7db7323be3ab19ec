"""Pins of the oracle's density pre-solve (Sec. "Numerical Simulations": the initial density and
higher moments come from an iteration run to steady state with the velocity held at u0)."""
import math

import numpy as np
import pytest

import oracle
from paper_1507_02518_gb300 import workloads as wl

NU_PRE = 1.0 / 6.0          # beta_pre = 1/2: every iteration relaxes fully to f_eq(rho, u0)


def test_mass_is_conserved():
    rho, u0 = wl.kida(12, 0.05)
    f, it, res = oracle.presolve(u0, oracle.beta(NU_PRE), 40)
    assert it == 40 and res > 0
    r, _ = oracle.macroscopic(f)
    assert float(r.sum()) == pytest.approx(12 ** 3, rel=1e-14)


def test_uniform_velocity_is_a_fixed_point():
    u0 = np.zeros((3, 4, 5, 6))
    u0[0], u0[1], u0[2] = 0.03, -0.02, 0.01
    f0 = oracle.init_equilibrium(np.ones((4, 5, 6)), u0)
    f, it, res = oracle.presolve(u0, oracle.beta(NU_PRE), 10, tol=0.0)
    assert it == 1 and res <= 1e-15        # converged after the first measured change
    assert np.max(np.abs(f - f0)) <= 1e-16


def test_parallel_shear_flow_needs_no_pressure():
    """u0 = U sin(k y) x: u.grad u = 0, so the density stays uniform (each y-level of the
    product-form equilibrium sums to W(v_y))."""
    _, u0 = wl.shear_wave(5, 16, 4, 0.04)
    f, it, res = oracle.presolve(u0, oracle.beta(0.02), 25)
    r, _ = oracle.macroscopic(f)
    assert np.max(np.abs(r - 1.0)) <= 1e-13     # round-off of 25 iterations; U^2 = 1.6e-3


@pytest.mark.parametrize("U,bound", [(0.005, 0.02), (0.02, 0.06)])
def test_taylor_green_converges_to_the_incompressible_pressure(U, bound):
    """2D Taylor-Green u0 = U (sin kx cos ky, -cos kx sin ky): the incompressible pressure is
    p - <p> = (U^2/4)(cos 2kx + cos 2ky), so rho - <rho> = 3 p' (c_s^2 = 1/3). The iteration's
    steady state approaches it as U -> 0 (its mass balance carries O(U/(D k)) advection terms)."""
    N, nz = 32, 3
    _, u0 = wl.taylor_green_2d(N, nz, U)
    f, it, res = oracle.presolve(u0, oracle.beta(NU_PRE), 4000, tol=1e-14)
    assert res <= 1e-14 and it < 4000
    r, _ = oracle.macroscopic(f)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(N), np.arange(N), indexing="ij")
    k = 2 * math.pi / N
    expect = 0.75 * U * U * (np.cos(2 * k * x) + np.cos(2 * k * y))
    err = np.max(np.abs(r - r.mean() - expect)) / np.max(np.abs(expect))
    assert err <= bound, err


def test_stops_at_tolerance_and_reports_the_change():
    _, u0 = wl.taylor_green_2d(16, 3, 0.01)
    _, it_a, res_a = oracle.presolve(u0, oracle.beta(NU_PRE), 5000, tol=1e-9)
    _, it_b, res_b = oracle.presolve(u0, oracle.beta(NU_PRE), 5000, tol=1e-12)
    assert res_a <= 1e-9 and res_b <= 1e-12
    assert it_a < it_b
    _, it_c, res_c = oracle.presolve(u0, oracle.beta(NU_PRE), it_a - 1, tol=1e-9)
    assert it_c == it_a - 1 and res_c > 1e-9
