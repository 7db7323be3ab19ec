"""Each workload configuration of the benchmark suite, at its stated size, on the GPU:
the 32^3 Taylor-Green case against the oracle over its full 200 steps, and one-step sampled
parity (the oracle collides the 27 upstream neighbours of each sampled node) for the 256^3
FP64 case, the 512^3 Kida case in FP32 and FP16 AA storage, and the 96-box ensemble."""
import math

import numpy as np
import pytest

import oracle
from paper_1507_02518_gb300 import lb, workloads

from test_gpu_parity import FP32_STEP_TOL, FP64_TOL, _sampled_step_check

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("scheme", ["pull", "aa"])
def test_taylor_green_32cubed_fp64_200_steps(kbc, scheme):
    """32^3, u0 = 0.05, k = 2 pi / 32, nu = 1e-3, rho0 = 1, 200 steps: max |df| <= 1e-12 and the
    kinetic energy of every 50th step equal to the oracle's."""
    n, nu = 32, 1e-3
    rho, u = workloads.taylor_green(n, 0.05)
    f = oracle.init_equilibrium(rho, u)
    lat = lb.Lattice(n, nu=nu, storage="f64", scheme=scheme)
    lat.init_field(rho, u)
    b = oracle.beta(nu)
    for _ in range(4):
        lat.step(50)
        f, _, _ = oracle.run(f, 50, b)
        r, uu = oracle.macroscopic(f)
        k_ref = oracle.diagnostics(r, uu, nu)["kinetic_energy"]
        assert lat.diagnostics()["kinetic_energy"] == pytest.approx(k_ref, rel=1e-12)
    assert np.max(np.abs(lat.get_populations() - f)) <= FP64_TOL


def test_taylor_green_small_amplitude_decays_at_the_viscous_rate(kbc):
    """At u0 = 1e-3 the vortex decays as exp(-2 nu |K|^2 t), |K|^2 = 3 (2 pi / 32)^2; measured
    between steps 100 and 200 the rate is within 5 % of it (4 % above on this grid: KBC's
    stabilizer and the lattice's O(k^2) terms; the oracle gives the same)."""
    n, nu = 32, 1e-3
    rho, u = workloads.taylor_green(n, 1e-3)
    lat = lb.Lattice(n, nu=nu, storage="f64", scheme="aa")
    lat.init_field(rho, u)
    lat.step(100)
    k1 = lat.diagnostics()["kinetic_energy"]
    lat.step(100)
    k2 = lat.diagnostics()["kinetic_energy"]
    rate = -math.log(k2 / k1) / 100
    assert rate == pytest.approx(2 * nu * 3 * (2 * math.pi / n) ** 2, rel=0.05)


def test_hit_256cubed_fp64_sampled_parity(kbc):
    n, nu = 256, 2e-4
    rho, u = workloads.random_spectrum(n, 4, 0.04, seed=1)
    lat = lb.Lattice(n, nu=nu, storage="f64", scheme="pull")
    lat.init_field(rho, u)
    lat.step(4)
    _sampled_step_check(lat, 24, FP64_TOL, np.random.default_rng(2))


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_kida_512cubed_aa_sampled_parity(kbc, storage):
    import torch
    n, nu = 512, 5e-5
    _, u = workloads.kida_device(n, 0.05)
    lat = lb.Lattice(n, nu=nu, storage=storage, scheme="aa")
    lat.init_field(None, u)
    del u
    torch.cuda.empty_cache()
    lat.step(5)
    rng = np.random.default_rng(3)
    _sampled_step_check(lat, 16, FP32_STEP_TOL, rng, half=storage == "f16")   # odd step
    _sampled_step_check(lat, 16, FP32_STEP_TOL, rng, half=storage == "f16")   # even step


class _BoxView:
    """The pieces of a Lattice that the sampled check uses, for box k of a batch."""

    def __init__(self, batch, k):
        c = batch.cfgs[k]
        self.shape = (c.nz, c.ny, c.nx)
        self.P = c.nx * c.ny * c.nz
        self.ctx = batch.box(k)
        self.beta = lb.lb_beta(self.ctx)
        self.step = batch.step


def test_batch96_sampled_parity(kbc):
    """The 96-box ensemble (73.5 M nodes, FP32 pull, autotuned, graph-replayed): one-step
    sampled parity in three boxes of different sizes."""
    import torch
    boxes = workloads.batch_boxes(96)
    batch = lb.Batch(boxes, storage="f32", scheme="pull")
    fields = [np.ascontiguousarray(workloads.random_spectrum(b["n"], b["k0"], b["urms"],
                                                             b["seed"])[1]) for b in boxes]
    for _ in range(2):          # tuned on the initial fields, which are then set again
        for k in range(len(boxes)):
            lb.lb_init_field(batch.box(k), 0, fields[k].ctypes.data, False)
        if _ == 0:
            batch.autotune(2)
    torch.cuda.synchronize()
    batch.step(3)
    sizes = [b["n"] for b in boxes]
    picks = [sizes.index(e) for e in (32, 48, 128) if e in sizes]
    rng = np.random.default_rng(4)
    for k in picks:
        _sampled_step_check(_BoxView(batch, k), 12, FP32_STEP_TOL, rng)
    assert all(d["nonfinite_count"] == 0 for d in batch.diagnostics())
