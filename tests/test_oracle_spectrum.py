"""Pins of the oracle's kinetic-energy spectrum E(kappa) (Sec. "Numerical Simulations")."""
import math

import numpy as np
import pytest

import oracle
from paper_1507_02518_gb300 import workloads as wl


def test_parseval_sum_is_the_kinetic_energy():
    rho, u = wl.random_spectrum(24, 4.0, 0.04, seed=3)
    u[0] += 0.01                                      # a mean flow is removed
    E = oracle.spectrum(u, 40)
    k = oracle.diagnostics(rho, u, 1e-3)["kinetic_energy"]
    assert float(E.sum()) == pytest.approx(k, rel=1e-12)
    assert E[0] == 0.0


@pytest.mark.parametrize("m1,m2,shell", [(3, 0, 3), (3, 4, 5), (1, 1, 1), (2, 3, 4)])
def test_single_modes_land_in_their_shell(m1, m2, shell):
    """u_z = U sin(2 pi (m1 x + m2 y) / N): energy U^2/4 at |n| = sqrt(m1^2 + m2^2)."""
    n, U = 16, 0.03
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    u = np.zeros((3, n, n, n))
    u[2] = U * np.sin(2 * math.pi * (m1 * x + m2 * y) / n)
    E = oracle.spectrum(u, 20)
    assert E[shell] == pytest.approx(U * U / 4, rel=1e-12)
    assert float(E.sum() - E[shell]) == pytest.approx(0.0, abs=1e-18)


def test_truncated_bins_drop_the_high_shells():
    rho, u = wl.random_spectrum(16, 6.0, 0.04, seed=5)
    full = oracle.spectrum(u, 20)
    part = oracle.spectrum(u, 5)
    assert np.array_equal(part, full[:5])
