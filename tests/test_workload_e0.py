"""The second example's initial field (eq:E0): shell spectrum, energy and Taylor Reynolds
number. The closed forms follow from eq:E0: k = 3 u0'^2 / 2 (so u' = u0'), the spectral
dissipation 2 nu int kappa^2 E = 5 nu k / b, hence Re_lambda = (2 b)^(1/2) u0' / nu, which is
the "initial spectrum at Re_lambda = 2000" of the paper's parameters."""
import math

import numpy as np
import pytest

import oracle
from paper_1507_02518_gb300 import workloads as wl


def e0(kap, u0p, nu):
    b = 20000 * math.sqrt(2 / 3) * nu / u0p
    return 400 * (2 / 3) ** 0.25 * math.sqrt(2 * nu * u0p ** 3 / math.pi) * b * b * kap ** 4 * \
        np.exp(-b * kap * kap)


@pytest.mark.parametrize("n,seed", [(32, 3), (33, 4)])
def test_shells_carry_eq_e0(n, seed):
    u0p, nu = 0.01, 1.98e-6               # peak at shell ~4 of a 32^3 box
    _, u = wl.spectrum_e0(n, u0p, nu, seed=seed)
    u = u.numpy()
    nb = int(math.sqrt(3) * n / 2) + 2
    E = oracle.spectrum(u, nb)
    kap = 2 * math.pi * np.arange(nb) / n
    expect = e0(kap, u0p, nu) * 2 * math.pi / n
    expect[0] = 0.0
    # shells cut by the Nyquist planes keep their interior modes only; compare below n/2
    m = np.arange(nb) < n // 2
    assert np.allclose(E[m], expect[m], rtol=1e-12, atol=1e-20)
    assert float(E.sum()) == pytest.approx(1.5 * u0p ** 2, rel=2e-3)
    # solenoidal: the spectral divergence vanishes
    k = np.fft.fftfreq(n)
    div = (np.fft.fftn(u[0]) * k[None, None, :] + np.fft.fftn(u[1]) * k[None, :, None]
           + np.fft.fftn(u[2]) * k[:, None, None])
    assert np.abs(div).max() < 1e-12


def test_paper_parameters_give_re_lambda_2000():
    """With nu = 8.16497e-5, u0' = 0.01 the closed forms give Re_lambda = 2000 (caption of the
    energy-spectrum figure); the discrete shell sums on a 400^3 grid reproduce them."""
    n, u0p, nu = 400, wl.E0_U0P, wl.E0_NU
    b = 20000 * math.sqrt(2 / 3) * nu / u0p
    assert math.sqrt(2 * b) * u0p / nu == pytest.approx(2000.0, rel=1e-6)
    nb = int(math.sqrt(3) * n / 2) + 2
    kap = 2 * math.pi * np.arange(nb) / n
    E = e0(kap, u0p, nu) * 2 * math.pi / n
    k = E.sum()
    eps = 2 * nu * float(np.sum(kap ** 2 * E))
    lam = math.sqrt(15 * nu * (2 * k / 3) / eps)
    assert k == pytest.approx(1.5 * u0p ** 2, rel=1e-9)
    assert lam * math.sqrt(2 * k / 3) / nu == pytest.approx(2000.0, rel=1e-6)
