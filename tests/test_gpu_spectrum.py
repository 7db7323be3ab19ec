"""Kinetic-energy spectrum E(kappa) on the GPU (lb_spectrum: cuFFT transforms, own shell
binning) against the oracle's numpy spectrum of the same velocity field."""
import math

import numpy as np
import pytest

import oracle
from paper_1507_02518_gb300 import lb, workloads

from test_gpu_parity import lattice

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("storage,rel", [("f64", 1e-11), ("f32", 2e-5), ("f16", 2e-5)])
@pytest.mark.parametrize("n", [24, 17])
def test_spectrum_matches_oracle(kbc, storage, rel, n):
    rho, u = workloads.random_spectrum(n, 3.0, 0.04, seed=2)
    lat = lattice((n, n, n), nu=1e-3, storage=storage, scheme="aa")
    lat.init_field(rho, u)
    lat.step(5)
    nb = int(math.sqrt(3) * n / 2) + 2
    E = lat.spectrum(nb)
    # the oracle bins the velocity of the same (decoded) state
    _, uu = oracle.macroscopic(lat.get_populations())
    ref = oracle.spectrum(uu, nb)
    assert E[0] == 0.0
    assert np.allclose(E, ref, rtol=rel, atol=rel * ref.max()), np.max(np.abs(E - ref))
    k = lat.diagnostics()["kinetic_energy"]
    assert float(E.sum()) == pytest.approx(k, rel=max(rel, 1e-12))


def test_single_mode_lands_in_its_shell(kbc):
    n, U = 16, 0.02
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    u = np.zeros((3, n, n, n))
    u[2] = U * np.sin(2 * math.pi * (3 * x + 4 * y) / n)
    lat = lattice((n, n, n), storage="f64", scheme="pull")
    lat.init_field(None, u)
    E = lat.spectrum(16)
    _, uu = oracle.macroscopic(lat.get_populations())
    assert E[5] == pytest.approx(oracle.spectrum(uu, 16)[5], rel=1e-12)
    assert E[5] == pytest.approx(U * U / 4, rel=1e-6)     # u of f_eq(1, u0) is u0 to O(1e-16)


def test_full_size_spectrum_sums_to_k(kbc):
    rho, u = workloads.random_spectrum(256, 4.0, 0.04, seed=1)
    lat = lattice((256, 256, 256), nu=2e-4, storage="f32", scheme="pull")
    lat.init_field(None, u)
    lat.step(10)
    E = lat.spectrum()
    k = lat.diagnostics()["kinetic_energy"]
    assert float(E.sum()) == pytest.approx(k, rel=1e-5)
    m = int(np.argmax(E))
    assert 2 <= m <= 8                                      # peak near k0 = 4


def test_spectrum_arguments(kbc):
    lat = lattice((12, 10, 12), storage="f32", scheme="aa")
    with pytest.raises(lb.LBError) as e:
        lat.spectrum(8)
    assert e.value.status == lb.LB_ERR_UNSUPPORTED
    cube = lattice((12, 12, 12), storage="f32", scheme="aa")
    for bad in (0, 7000):
        assert lb.lb_spectrum_work_bytes(cube.ctx, bad) == 0
    need = lb.lb_spectrum_work_bytes(cube.ctx, 8)
    import torch
    buf = torch.empty(need + 512, dtype=torch.uint8, device="cuda")
    ptr = (buf.data_ptr() + 255) // 256 * 256
    with pytest.raises(lb.LBError) as e:
        lb.lb_spectrum(cube.ctx, ptr, need - 256, 8)
    assert e.value.status == lb.LB_ERR_INVALID_ARG
    assert lb.lb_spectrum(cube.ctx, ptr, need, 8)[0] == 0.0
