"""Seeded synthetic inputs (initial density and velocity fields) for the KBC step.

This module holds input generation only: no lattice-Boltzmann arithmetic (no equilibrium,
moments or collision). Both the CUDA path and the CPU oracle take their inputs from here.

Arrays are float64, indexed ``[z, y, x]`` (x fastest); velocities are ``u[3, z, y, x]``.
Node ``j`` on an axis of ``n`` nodes sits at ``x_j = 2*pi*j/n`` when a flow is written on
``[0, 2*pi]`` (Sec. "Numerical Simulations", eq:kida).
"""
from __future__ import annotations

import math

import numpy as np

BATCH_EDGES = (32, 48, 64, 96, 128)
BATCH_BASE_SEED = 20150702


def _grid(nx: int, ny: int, nz: int):
    z, y, x = np.meshgrid(np.arange(nz, dtype=np.float64), np.arange(ny, dtype=np.float64),
                          np.arange(nx, dtype=np.float64), indexing="ij")
    return x, y, z


def taylor_green(n: int, u0: float = 0.05, k: float | None = None):
    """3D Taylor-Green vortex: u = u0 sin kx cos ky cos kz, v = -u0 cos kx sin ky cos kz, w = 0.

    ``k`` defaults to 2*pi/n (one period per box). Density is 1.
    """
    k = 2.0 * math.pi / n if k is None else k
    x, y, z = _grid(n, n, n)
    u = np.zeros((3, n, n, n))
    u[0] = u0 * np.sin(k * x) * np.cos(k * y) * np.cos(k * z)
    u[1] = -u0 * np.cos(k * x) * np.sin(k * y) * np.cos(k * z)
    return np.ones((n, n, n)), u


def taylor_green_2d(n: int, nz: int, u0: float):
    """z-invariant 2D Taylor-Green vortex on an n x n x nz box (density 1)."""
    k = 2.0 * math.pi / n
    x, y, _ = _grid(n, n, nz)
    u = np.zeros((3, nz, n, n))
    u[0] = u0 * np.sin(k * x) * np.cos(k * y)
    u[1] = -u0 * np.cos(k * x) * np.sin(k * y)
    return np.ones((nz, n, n)), u


def shear_wave(nx: int, ny: int, nz: int, u0: float, mode: int = 1):
    """Transverse shear wave u_x = u0 sin(2 pi mode y / ny) (density 1)."""
    x, y, _ = _grid(nx, ny, nz)
    u = np.zeros((3, nz, ny, nx))
    u[0] = u0 * np.sin(2.0 * math.pi * mode * y / ny)
    return np.ones((nz, ny, nx)), u


def kida(n: int, U0: float = 0.05):
    """Kida vortex (eq:kida) on x, y, z in [0, 2 pi) sampled at 2 pi j / n; density 1."""
    h = 2.0 * math.pi / n
    x, y, z = (a * h for a in _grid(n, n, n))
    u = np.zeros((3, n, n, n))
    u[0] = U0 * np.sin(x) * (np.cos(3 * y) * np.cos(z) - np.cos(y) * np.cos(3 * z))
    u[1] = U0 * np.sin(y) * (np.cos(3 * z) * np.cos(x) - np.cos(z) * np.cos(3 * x))
    u[2] = U0 * np.sin(z) * (np.cos(3 * x) * np.cos(y) - np.cos(x) * np.cos(3 * y))
    return np.ones((n, n, n)), u


def random_spectrum(n: int, k0: float, urms: float, seed: int, dtype=np.float64):
    """Random-phase solenoidal field with shell spectrum E(k) ~ k^4 exp(-2 (k/k0)^2).

    ``k0`` is the peak wavenumber in units of 2 pi / n. White Gaussian noise per component
    is transformed, shaped so that each spherical shell carries energy proportional to
    E(k), projected onto divergence-free modes, stripped of the mean and Nyquist modes, and
    transformed back; the result is scaled so that the r.m.s. of one component,
    ``sqrt(<u.u>/3)``, equals ``urms`` (the u' of Table 2's caption). Density is 1.
    """
    rng = np.random.default_rng(seed)
    kf = np.fft.fftfreq(n) * n
    kr = np.fft.rfftfreq(n) * n
    KZ, KY, KX = np.meshgrid(kf, kf, kr, indexing="ij")
    K2 = KX * KX + KY * KY + KZ * KZ
    K = np.sqrt(K2)
    # |a|^2 per mode ~ E(K) / K^2 so that a shell (4 pi K^2 modes) carries E(K)
    amp = K * np.exp(-((K / k0) ** 2))
    nyq = n // 2
    mask = (np.abs(KX) == nyq) | (np.abs(KY) == nyq) | (np.abs(KZ) == nyq) | (K == 0)
    amp[mask] = 0.0
    a = np.empty((3,) + K.shape, dtype=np.complex128)
    for c in range(3):
        a[c] = np.fft.rfftn(rng.standard_normal((n, n, n))) * amp
    with np.errstate(divide="ignore", invalid="ignore"):
        kdota = (KX * a[0] + KY * a[1] + KZ * a[2]) / np.where(K2 > 0, K2, 1.0)
    a[0] -= KX * kdota
    a[1] -= KY * kdota
    a[2] -= KZ * kdota
    u = np.stack([np.fft.irfftn(a[c], s=(n, n, n), axes=(0, 1, 2)) for c in range(3)])
    rms = math.sqrt(float(np.mean(np.sum(u * u, axis=0))) / 3.0)
    u *= urms / rms
    return np.ones((n, n, n)), u.astype(dtype, copy=False)


def random_spectrum_device(n: int, k0: float, urms: float, seed: int, device="cuda"):
    """The recipe of random_spectrum generated on a GPU with torch (float64), for boxes whose
    host generation would be slow (768^3). Same spectrum, projection and scaling; the white
    noise comes from torch's generator seeded with ``seed``, so the field differs from the
    numpy version of the same seed. Returns (None, u[3, n, n, n]) on ``device`` (density 1).
    """
    import torch
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    kf = torch.fft.fftfreq(n, d=1.0 / n, dtype=torch.float64, device=device)
    kr = torch.fft.rfftfreq(n, d=1.0 / n, dtype=torch.float64, device=device)
    KZ = kf.view(n, 1, 1)
    KY = kf.view(1, n, 1)
    KX = kr.view(1, 1, -1)
    K2 = KX * KX + KY * KY + KZ * KZ
    K = torch.sqrt(K2)
    amp = K * torch.exp(-((K / k0) ** 2))
    nyq = n // 2
    mask = (KX.abs() == nyq) | (KY.abs() == nyq) | (KZ.abs() == nyq) | (K == 0)
    amp = torch.where(mask, torch.zeros_like(amp), amp)
    a = []
    for _ in range(3):
        noise = torch.randn((n, n, n), generator=gen, dtype=torch.float64, device=device)
        a.append(torch.fft.rfftn(noise) * amp)
        del noise
    safe = torch.where(K2 > 0, K2, torch.ones_like(K2))
    kdota = (KX * a[0] + KY * a[1] + KZ * a[2]) / safe
    a[0] = a[0] - KX * kdota
    a[1] = a[1] - KY * kdota
    a[2] = a[2] - KZ * kdota
    del kdota, K, K2, amp, mask, safe
    u = torch.empty((3, n, n, n), dtype=torch.float64, device=device)
    for c in range(3):
        u[c] = torch.fft.irfftn(a[c], s=(n, n, n))
        a[c] = None
    rms = math.sqrt(float((u * u).sum()) / (3.0 * n ** 3))
    u *= urms / rms
    return None, u


E0_U0P = 0.01           # u0' of eq:E0 (Sec. "Numerical Simulations", second example)
E0_NU = 8.164970e-5     # nu of eq:E0


def spectrum_e0(n: int, u0p: float = E0_U0P, nu: float = E0_NU, seed: int = 1, device="cpu"):
    """Random solenoidal field whose shell spectrum is eq:E0:
        E0(kappa) = 400 (2/3)^(1/4) (2 nu u0'^3 / pi)^(1/2) b^2 kappa^4 exp(-b kappa^2),
        b = 20000 (2/3)^(1/2) nu / u0',
    kappa in lattice units (2 pi m / n for shell m). White Gaussian noise per component is
    transformed, projected onto divergence-free modes (mean and Nyquist modes removed), and
    each shell m = rint(|n|) is rescaled so that it carries exactly E0(kappa_m) d kappa,
    d kappa = 2 pi / n (so k = sum of the shells, which is 3 u0'^2 / 2 when the peak is
    resolved). torch (float64) on ``device``; returns (None, u[3, n, n, n]) there."""
    import torch
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    f64 = dict(dtype=torch.float64, device=device)
    kf = torch.fft.fftfreq(n, d=1.0 / n, **f64)
    kr = torch.fft.rfftfreq(n, d=1.0 / n, **f64)
    KZ, KY, KX = kf.view(n, 1, 1), kf.view(1, n, 1), kr.view(1, 1, -1)
    K2 = KX * KX + KY * KY + KZ * KZ
    shell = torch.round(torch.sqrt(K2)).to(torch.int64)
    nyq = n // 2
    keep = ~((KX.abs() == nyq) | (KY.abs() == nyq) | (KZ.abs() == nyq) | (K2 == 0))
    a = []
    for _ in range(3):
        noise = torch.randn((n, n, n), generator=gen, **f64)
        a.append(torch.fft.rfftn(noise) * keep)
        del noise
    safe = torch.where(K2 > 0, K2, torch.ones_like(K2))
    kdota = (KX * a[0] + KY * a[1] + KZ * a[2]) / safe
    a = [a[0] - KX * kdota, a[1] - KY * kdota, a[2] - KZ * kdota]
    del kdota, safe
    # shell energies of the half spectrum: 1/2 |u_hat|^2, u_hat = rfft / P, doubled off the
    # kx = 0 and kx = n/2 planes (they stand for the conjugate modes too)
    P = float(n) ** 3
    w = torch.full((1, 1, kr.numel()), 2.0, **f64)
    w[..., 0] = 1.0
    if n % 2 == 0:
        w[..., -1] = 1.0
    e = 0.5 * w * sum((c.abs() ** 2) for c in a) / (P * P)
    nb = int(shell.max()) + 1
    E = torch.zeros(nb, **f64).index_add_(0, shell.flatten(), e.expand_as(shell).flatten())
    b = 20000.0 * math.sqrt(2.0 / 3.0) * nu / u0p
    kap = 2.0 * math.pi * torch.arange(nb, **f64) / n
    target = (400.0 * (2.0 / 3.0) ** 0.25 * math.sqrt(2.0 * nu * u0p ** 3 / math.pi) * b * b
              * kap ** 4 * torch.exp(-b * kap * kap)) * (2.0 * math.pi / n)
    scale = torch.where(E > 0, torch.sqrt(target / torch.where(E > 0, E, torch.ones_like(E))),
                        torch.zeros_like(E))
    sc = scale[shell]
    u = torch.empty((3, n, n, n), **f64)
    for c in range(3):
        u[c] = torch.fft.irfftn(a[c] * sc, s=(n, n, n))
        a[c] = None
    return None, u


def kida_device(n: int, U0: float = 0.05, device="cuda"):
    """eq:kida on a GPU with torch (float64); returns (None, u[3, n, n, n]) on ``device``."""
    import torch
    x = torch.arange(n, dtype=torch.float64, device=device) * (2.0 * math.pi / n)
    X, Y, Z = x.view(1, 1, n), x.view(1, n, 1), x.view(n, 1, 1)
    u = torch.empty((3, n, n, n), dtype=torch.float64, device=device)
    u[0] = U0 * torch.sin(X) * (torch.cos(3 * Y) * torch.cos(Z) - torch.cos(Y) * torch.cos(3 * Z))
    u[1] = U0 * torch.sin(Y) * (torch.cos(3 * Z) * torch.cos(X) - torch.cos(Z) * torch.cos(3 * X))
    u[2] = U0 * torch.sin(Z) * (torch.cos(3 * X) * torch.cos(Y) - torch.cos(X) * torch.cos(3 * Y))
    return None, u


def population_noise(nx: int, ny: int, nz: int, seed: int):
    """Uniform noise in [-1, 1] shaped like a population field, [27, z, y, x]."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-1.0, 1.0, size=(27, nz, ny, nx))


def batch_boxes(nbox: int = 96, seed: int = BATCH_BASE_SEED):
    """Parameters of the batched decaying-turbulence ensemble.

    Edge uniform in {32, 48, 64, 96, 128}; k0 ~ U[2, 6]; u_rms ~ U[0.02, 0.06];
    nu log-uniform in [1e-5, 1e-3]; the field of box b is seeded with ``seed + b``.
    """
    rng = np.random.default_rng(seed)
    edges = rng.choice(np.array(BATCH_EDGES), size=nbox)
    k0 = rng.uniform(2.0, 6.0, size=nbox)
    urms = rng.uniform(0.02, 0.06, size=nbox)
    nu = np.exp(rng.uniform(math.log(1e-5), math.log(1e-3), size=nbox))
    return [{"n": int(edges[b]), "k0": float(k0[b]), "urms": float(urms[b]),
             "nu": float(nu[b]), "seed": int(seed + b)} for b in range(nbox)]
