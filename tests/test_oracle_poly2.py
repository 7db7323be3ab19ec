"""Pins of the oracle's polynomial-equilibrium variant (eq:polynomial2)."""
import math

import numpy as np
import pytest

import oracle
from paper_1507_02518_gb300 import workloads as wl

V, W = oracle.lattice()


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_moments_of_the_polynomial_equilibrium(seed):
    """The standard LB equilibrium's moments on D3Q27, exactly: rho, rho u,
    rho (delta/3 + u u), third moments rho u_a / 3 for (a, b, b), b != a, zero for (x, y, z)."""
    rng = np.random.default_rng(seed)
    rho, u = 1 + rng.uniform(-0.1, 0.1), rng.uniform(-0.2, 0.2, 3)
    f = oracle.equilibrium_poly2(rho, u)
    Vf = V.astype(float)
    assert f.sum() == pytest.approx(rho, rel=1e-15)
    assert np.allclose(Vf.T @ f, rho * u, atol=1e-15)
    second = np.einsum("ia,ib,i->ab", Vf, Vf, f)
    assert np.allclose(second, rho * (np.eye(3) / 3 + np.outer(u, u)), atol=1e-15)
    for a in range(3):
        for b in range(3):
            if a != b:
                m = np.sum(Vf[:, a] * Vf[:, b] ** 2 * f)
                assert m == pytest.approx(rho * u[a] / 3, abs=1e-15)
    assert abs(np.sum(Vf[:, 0] * Vf[:, 1] * Vf[:, 2] * f)) < 1e-16


def test_agrees_with_the_product_form_to_second_order():
    """eq:polynomial2 is the second-order truncation of eq:entropic_eq: the gap is O(u^3)."""
    u0 = np.array([0.3, -0.2, 0.1])
    gaps = [np.max(np.abs(oracle.equilibrium_poly2(1.0, s * u0) - oracle.equilibrium(1.0, s * u0)))
            for s in (0.1, 0.05)]
    assert gaps[0] / gaps[1] == pytest.approx(8.0, rel=0.1)


def test_lbgk_with_the_polynomial_equilibrium():
    """gamma = 2: f' = f - 2 beta (f - f_eq^poly), whatever the shear part."""
    rng = np.random.default_rng(7)
    f = oracle.equilibrium(1.0, [0.04, -0.02, 0.03]) * (1 + 1e-3 * rng.uniform(-1, 1, 27))
    b = oracle.beta(1e-3)
    rho = f.sum()
    u = (V.T.astype(float) @ f) / rho
    expect = f - 2 * b * (f - oracle.equilibrium_poly2(rho, u))
    for variant in (oracle.S_D, oracle.S_DTQ, oracle.S_CDTQ):
        fo, g, _ = oracle.collide(f, b, variant | oracle.EQ_POLY2, oracle.GAMMA_LBGK)
        assert np.allclose(fo, expect, atol=2e-16, rtol=0), variant


@pytest.mark.parametrize("variant", [oracle.S_DTQ, oracle.S_D, oracle.S_CDTQ])
def test_collision_conserves_mass_and_momentum(variant):
    rng = np.random.default_rng(9)
    f = oracle.equilibrium(1.01, [0.05, 0.02, -0.04]) * (1 + 1e-3 * rng.uniform(-1, 1, 27))
    fo, _, _ = oracle.collide(f, oracle.beta(1e-4), variant | oracle.EQ_POLY2)
    assert fo.sum() == pytest.approx(f.sum(), rel=1e-15)
    assert np.allclose(V.T @ fo, V.T @ f, atol=1e-16)


def test_shear_wave_viscosity_with_the_polynomial_equilibrium():
    nx, ny, nz, nu = 3, 32, 3, 0.02
    b = oracle.beta(nu)
    rho, u = wl.shear_wave(nx, ny, nz, 1e-4)
    f = oracle.init_equilibrium(rho, u)
    var = oracle.S_DTQ | oracle.EQ_POLY2
    f, _, _ = oracle.run(f, 40, b, var)

    def amp(f):
        _, uu = oracle.macroscopic(f)
        return 2.0 / ny * float(np.mean(uu[0], axis=(0, 2)) @ np.sin(2 * math.pi * np.arange(ny) / ny))

    a0 = amp(f)
    f, _, _ = oracle.run(f, 400, b, var)
    k = 2 * math.pi / ny
    assert -math.log(amp(f) / a0) / (k * k * 400) == pytest.approx(nu, rel=0.02)
