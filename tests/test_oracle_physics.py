"""Physics pins of the oracle: decay rates the viscosity relation fixes, and closed-form
diagnostics on the discrete grid (arXiv:1507.02518, eq:viscosity, Sec. "Numerical Simulations").
"""
import math

import numpy as np
import pytest

import oracle
from paper_1507_02518_gb300 import workloads as wl


def shear_amplitude(f, ny):
    rho, u = oracle.macroscopic(f)
    y = np.arange(ny)
    s = np.sin(2 * math.pi * y / ny)
    return 2.0 / ny * float(np.mean(u[0], axis=(0, 2)) @ s)


@pytest.mark.parametrize("variant,mode", [(oracle.S_DTQ, oracle.GAMMA_ESTIMATE),
                                          (oracle.S_D, oracle.GAMMA_ESTIMATE),
                                          (oracle.S_DT, oracle.GAMMA_ESTIMATE),
                                          (oracle.S_DQ, oracle.GAMMA_ESTIMATE),
                                          (oracle.S_DTQ, oracle.GAMMA_LBGK),
                                          (oracle.S_CD, oracle.GAMMA_ESTIMATE),
                                          (oracle.S_CDTQ, oracle.GAMMA_ESTIMATE)])
def test_shear_wave_decays_at_lattice_viscosity(variant, mode):
    """u_x = U sin(k y) decays as exp(-nu k^2 t), nu = c_s^2 (1/(2 beta) - 1/2), for any gamma."""
    nx, ny, nz = 3, 32, 3
    nu = 0.02
    b = oracle.beta(nu)
    rho, u = wl.shear_wave(nx, ny, nz, 1e-4)
    f = oracle.init_equilibrium(rho, u)
    f, _, _ = oracle.run(f, 40, b, variant, mode)       # let the initial transient pass
    a0 = shear_amplitude(f, ny)
    steps = 400
    f, _, _ = oracle.run(f, steps, b, variant, mode)
    a1 = shear_amplitude(f, ny)
    k = 2 * math.pi / ny
    nu_fit = -math.log(a1 / a0) / (k * k * steps)
    assert nu_fit == pytest.approx(nu, rel=0.02)


def test_taylor_green_2d_energy_decay():
    """z-invariant Taylor-Green: E ~ exp(-2 nu |k|^2 t) with |k|^2 = 2 (2 pi / n)^2."""
    n, nz = 24, 3
    nu = 0.02
    b = oracle.beta(nu)
    rho, u = wl.taylor_green_2d(n, nz, 1e-4)
    f = oracle.init_equilibrium(rho, u)
    f, _, _ = oracle.run(f, 20, b)

    def energy(f):
        _, uu = oracle.macroscopic(f)
        return 0.5 * float(np.mean(np.sum(uu * uu, axis=0)))

    e0 = energy(f)
    steps = 200
    f, _, _ = oracle.run(f, steps, b)
    e1 = energy(f)
    k2 = 2 * (2 * math.pi / n) ** 2
    nu_fit = -math.log(e1 / e0) / (2 * k2 * steps)
    assert nu_fit == pytest.approx(nu, rel=0.02)


def test_kida_initial_kinetic_energy_closed_form():
    """k(0) of eq:kida on the grid is exactly 3 U0^2 / 8 (trigonometric orthogonality)."""
    U0 = 0.05
    rho, u = wl.kida(16, U0)
    d = oracle.diagnostics(rho, u, 1e-3)
    assert d["kinetic_energy"] == pytest.approx(3 * U0 * U0 / 8, rel=1e-13)
    assert d["mass"] == pytest.approx(16 ** 3, rel=1e-15)
    assert np.allclose(d["momentum"], 0.0, atol=1e-13)


def test_shear_wave_diagnostics_closed_form():
    """2nd-order central differences of U sin(k y): Omega = U^2 sin^2 k / 4, eps = nu U^2 sin^2 k / 2."""
    U, nu = 0.03, 2e-3
    for ny, mode in ((16, 1), (16, 3), (20, 2)):
        rho, u = wl.shear_wave(4, ny, 5, U, mode)
        d = oracle.diagnostics(rho, u, nu)
        kk = 2 * math.pi * mode / ny
        assert d["kinetic_energy"] == pytest.approx(U * U / 4, rel=1e-13)
        assert d["enstrophy"] == pytest.approx(U * U * math.sin(kk) ** 2 / 4, rel=1e-12)
        assert d["dissipation"] == pytest.approx(nu * U * U * math.sin(kk) ** 2 / 2, rel=1e-12)


def test_mean_flow_is_removed_from_statistics():
    """u' = u - <u> (Sec. "Numerical Simulations"): a uniform offset changes neither k nor Omega."""
    rho, u = wl.shear_wave(4, 16, 4, 0.02, 2)
    d0 = oracle.diagnostics(rho, u, 1e-3)
    u2 = u.copy()
    u2[1] += 0.01
    d1 = oracle.diagnostics(rho, u2, 1e-3)
    for key in ("kinetic_energy", "enstrophy", "dissipation"):
        assert d1[key] == pytest.approx(d0[key], rel=1e-12)


def test_eighth_order_gradients_converge_at_eighth_order():
    """Omega of a shear wave with 8th-order differences approaches the continuum U^2 kappa^2 / 4
    with an error that falls by 2^8 when the grid is refined by 2 (Table 2's stencils)."""
    U = 0.03
    errs = []
    for ny in (16, 32):
        rho, u = wl.shear_wave(3, ny, 3, U)
        d = oracle.diagnostics(rho, u, 1e-3, order=8)
        kk = 2 * math.pi / ny
        errs.append(abs(d["enstrophy"] / (U * U * kk * kk / 4) - 1))
    assert errs[0] < 5e-6
    assert errs[0] / errs[1] == pytest.approx(256.0, rel=0.05), errs
    # second order: the same wave gives sin^2(kappa) instead of kappa^2 (closed form above)
    d2 = oracle.diagnostics(*wl.shear_wave(3, 16, 3, U), 1e-3, order=2)
    assert d2["enstrophy"] == pytest.approx(U * U * math.sin(2 * math.pi / 16) ** 2 / 4,
                                            rel=1e-12)


@pytest.mark.parametrize("order", [2, 8])
def test_skewness_factors_of_a_longitudinal_wave(order):
    """u_x = U sin(kappa x): du_x/dx = U K cos(kappa x) for any difference order, so
    S3 = S5 = 0, S4 = <cos^4>/<cos^2>^2 = 3/2, S6 = <cos^6>/<cos^2>^3 = 5/2."""
    n = 24
    u = np.zeros((3, 4, 3, n))
    u[0] = 0.02 * np.sin(2 * math.pi * np.arange(n) / n)
    d = oracle.diagnostics(np.ones((4, 3, n)), u, 1e-3, order=order)
    s3, s4, s5, s6 = d["skewness"]
    assert abs(s3) < 1e-12 and abs(s5) < 1e-12
    assert s4 == pytest.approx(1.5, rel=1e-12)
    assert s6 == pytest.approx(2.5, rel=1e-12)


def test_skewness_factors_of_a_two_mode_wave_match_the_continuum():
    """u_x = U (sin th + sin(2 th)/2), th = kappa x: du_x/dx = U kappa (cos th + cos 2 th) in the
    continuum. Its S_n by quadrature on a fine grid; the 8th-order stencil on 32 points
    reproduces them to the stencil's error."""
    n = 32
    th = 2 * math.pi * np.arange(n) / n
    u = np.zeros((3, 3, 3, n))
    u[0] = 0.01 * (np.sin(th) + 0.5 * np.sin(2 * th))
    d = oracle.diagnostics(np.ones((3, 3, n)), u, 1e-3, order=8)
    fine = 2 * math.pi * np.arange(4096) / 4096
    g = np.cos(fine) + np.cos(2 * fine)
    m2 = np.mean(g ** 2)
    for i, m in enumerate((3, 4, 5, 6)):
        expect = (-1) ** m * np.mean(g ** m) / m2 ** (m / 2)
        assert d["skewness"][i] == pytest.approx(expect, rel=1e-5, abs=1e-9), (m, expect)
    # by hand: <g^2> = 1, <g^3> = 3 <cos^2 th cos 2th> = 3/4, so S3 = -3/4
    assert d["skewness"][0] == pytest.approx(-0.75, rel=1e-5)


def test_shear_wave_viscosity_converges_at_second_order():
    """The lattice's effective viscosity approaches nu as (grid spacing)^2 (the paper's
    second-order convergence): the relative error of the fitted decay rate falls by ~4 per
    doubling of the wave's resolution, over the same fraction of its decay time."""
    nu = 0.01
    b = oracle.beta(nu)
    errs = []
    for ny in (16, 32, 64):
        rho, u = wl.shear_wave(3, ny, 3, 1e-5)
        f = oracle.init_equilibrium(rho, u)
        T = int(0.2 * ny * ny / nu / (4 * math.pi ** 2))
        f, _, _ = oracle.run(f, T // 4, b)
        a0 = shear_amplitude(f, ny)
        f, _, _ = oracle.run(f, T, b)
        a1 = shear_amplitude(f, ny)
        k = 2 * math.pi / ny
        errs.append(abs(-math.log(a1 / a0) / (k * k * T) / nu - 1))
    assert errs[2] < 2e-3
    for r in (errs[0] / errs[1], errs[1] / errs[2]):
        assert 3.3 < r < 4.7, errs
