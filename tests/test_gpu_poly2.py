"""Polynomial-equilibrium variant (eq:polynomial2) of the CUDA collision against the oracle."""
import numpy as np
import pytest

import oracle
from paper_1507_02518_gb300 import lb, workloads

from test_gpu_parity import FP32_STEP_TOL, FP64_TOL, lattice, seeded_state

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("variant", ["d", "d+t+q", "cd+ct+cq", "d+q"])
@pytest.mark.parametrize("gamma", ["estimate", "lbgk", "rlb"])
@pytest.mark.parametrize("scheme", ["pull", "aa"])
def test_fp64_poly2_matches_oracle(kbc, variant, gamma, scheme):
    f0 = seeded_state(10, 9, 8, noise=1e-3)
    steps, nu = 6, 5e-4
    lat = lattice((10, 9, 8), nu=nu, storage="f64", scheme=scheme, variant=variant, gamma=gamma,
                  equilibrium="poly2")
    lat.set_populations(f0)
    lat.step(steps)
    ref, _, _ = oracle.run(f0, steps, oracle.beta(nu), lb.VARIANT[variant] | oracle.EQ_POLY2,
                           lb.GAMMA[gamma])
    err = np.max(np.abs(lat.get_populations() - ref))
    assert err <= FP64_TOL, err


def test_poly2_differs_from_the_product_form(kbc):
    f0 = seeded_state(10, 9, 8, noise=1e-3)
    out = {}
    for eq in ("product", "poly2"):
        lat = lattice((10, 9, 8), nu=5e-4, storage="f64", scheme="aa", equilibrium=eq)
        lat.set_populations(f0)
        lat.step(1)
        out[eq] = lat.get_populations()
    d = np.max(np.abs(out["poly2"] - out["product"]))
    assert 1e-9 < d < 1e-4, d          # O(u^3) with u ~ 0.05


@pytest.mark.parametrize("scheme", ["pull", "aa"])
@pytest.mark.parametrize("kind", ["direct", "packed"])
@pytest.mark.parametrize("variant", ["d+t+q", "cd+ct+cq"])
def test_fp32_poly2_one_step_parity(kbc, scheme, kind, variant):
    n = 20
    rho, u = workloads.random_spectrum(n, 4, 0.04, seed=1)
    f0 = oracle.init_equilibrium(rho, u) * (1 + 1e-4 * workloads.population_noise(n, n, n, 5))
    lat = lattice((n, n, n), nu=2e-4, storage="f32", scheme=scheme, variant=variant,
                  equilibrium="poly2")
    lat.set_kernel(kind)
    lat.set_populations(f0)
    lat.step(3)
    f_in = lat.get_populations()
    ref, _, _ = oracle.run(f_in, 1, lat.beta, lb.VARIANT[variant] | oracle.EQ_POLY2)
    lat.step(1)
    err = np.max(np.abs(lat.get_populations() - ref))
    assert err <= FP32_STEP_TOL, err


def test_poly2_is_refused_where_it_is_not_built(kbc):
    import torch
    lat = lattice((8, 8, 8), storage="f32", scheme="pull", equilibrium="poly2")
    with pytest.raises(lb.LBError) as e:
        lat.stabilizer_gap()
    assert e.value.status == lb.LB_ERR_UNSUPPORTED
    for kind in ("staged", "persistent"):
        with pytest.raises(lb.LBError) as e:
            lat.set_kernel(kind)
        assert e.value.status == lb.LB_ERR_UNSUPPORTED
    cfgs = [lb.make_config(8, storage="f32", equilibrium="poly2")]
    need = lb.lb_batch_required_bytes(cfgs)
    buf = torch.empty(need + 256, dtype=torch.uint8, device="cuda")
    with pytest.raises(lb.LBError) as e:
        lb.lb_batch_create(cfgs, (buf.data_ptr() + 255) // 256 * 256, need)
    assert e.value.status == lb.LB_ERR_UNSUPPORTED
