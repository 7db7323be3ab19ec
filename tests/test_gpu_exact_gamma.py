"""Exact stabilizer (root of eq:result1) and the stabilizer gap on the GPU against the oracle.

The oracle's root is pinned independently in test_oracle_pins.py (bracketing root of the
entropy derivative). Tolerances: FP64 populations 1e-12 (the FP64 bar); FP32 one step from
identical stored inputs within the FP32 collision bound; gap statistics to the precision
their arithmetic allows (FP64: 1e-10 relative; FP32: the Newton tolerance 1e-6 per node).
"""
import numpy as np
import pytest

import oracle
from paper_1507_02518_gb300 import lb, workloads

from test_gpu_parity import FP32_STEP_TOL, FP64_TOL, lattice, seeded_state

pytestmark = pytest.mark.gpu


def oracle_gammas(f, beta, variant):
    _, g_est, _ = oracle.collide_field(f, beta, variant, oracle.GAMMA_ESTIMATE, want_gamma=True)
    _, g_ex, _ = oracle.collide_field(f, beta, variant, oracle.GAMMA_EXACT, want_gamma=True)
    return g_est, g_ex


@pytest.mark.parametrize("variant", ["d+t+q", "d", "cd+ct+cq"])
@pytest.mark.parametrize("scheme", ["pull", "aa"])
def test_exact_fp64_matches_oracle(kbc, variant, scheme):
    f0 = seeded_state(10, 9, 8, noise=1e-3)
    steps, nu = 7, 5e-4
    lat = lattice((10, 9, 8), nu=nu, storage="f64", scheme=scheme, variant=variant, gamma="exact")
    lat.set_populations(f0)
    lat.step(steps)
    ref, g_ref, guarded = oracle.run(f0, steps, oracle.beta(nu), lb.VARIANT[variant],
                                     oracle.GAMMA_EXACT, want_gamma=True)
    err = np.max(np.abs(lat.get_populations() - ref))
    assert err <= FP64_TOL, err
    d = lat.diagnostics()
    # the recorded gamma field is FP32 (one rounding per node)
    assert d["gamma_mean"] == pytest.approx(float(np.mean(g_ref)), abs=2e-7)
    assert d["gamma_std"] == pytest.approx(float(np.std(g_ref)), rel=1e-4, abs=2e-7)
    assert d["den_guard_count"] == guarded


def test_exact_differs_from_estimate_by_the_gap(kbc):
    """The two modes give different trajectories; the difference is the gamma gap times dh."""
    f0 = seeded_state(10, 9, 8, noise=1e-3)
    nu = 5e-4
    out = {}
    for gamma in ("estimate", "exact"):
        lat = lattice((10, 9, 8), nu=nu, storage="f64", scheme="aa", gamma=gamma)
        lat.set_populations(f0)
        lat.step(1)
        out[gamma] = lat.get_populations()
    diff = np.max(np.abs(out["exact"] - out["estimate"]))
    assert 1e-12 < diff < 1e-4, diff


@pytest.mark.parametrize("scheme", ["pull", "aa"])
def test_exact_fp32_one_step_parity(kbc, scheme):
    n = 20
    rho, u = workloads.random_spectrum(n, 4, 0.04, seed=1)
    f0 = oracle.init_equilibrium(rho, u) * (1 + 1e-3 * workloads.population_noise(n, n, n, 5))
    nu = 2e-4
    lat = lattice((n, n, n), nu=nu, storage="f32", scheme=scheme, gamma="exact")
    lat.set_populations(f0)
    lat.step(3)
    f_in = lat.get_populations()
    ref, _, _ = oracle.run(f_in, 1, lat.beta, oracle.S_DTQ, oracle.GAMMA_EXACT)
    lat.step(1)
    err = np.max(np.abs(lat.get_populations() - ref))
    assert err <= FP32_STEP_TOL, err


@pytest.mark.parametrize("storage,scheme,t", [("f64", "pull", 0), ("f64", "aa", 3),
                                              ("f64", "pull", 4), ("f32", "aa", 2),
                                              ("f32", "pull", 1), ("f16", "aa", 1)])
@pytest.mark.parametrize("variant", ["d+t+q", "cd+ct+cq"])
def test_stabilizer_gap_matches_oracle(kbc, storage, scheme, t, variant):
    shape = (14, 11, 9)
    f0 = seeded_state(*shape, noise=2e-3)
    nu = 5e-4
    lat = lattice(shape, nu=nu, storage=storage, scheme=scheme, variant=variant)
    lat.set_populations(f0)
    lat.step(t)
    f = lat.get_populations()                       # the state the gap is evaluated on
    g_est, g_ex = oracle_gammas(f, lat.beta, lb.VARIANT[variant])
    gap = lat.stabilizer_gap()
    P = f0[0].size
    assert gap["step"] == t
    assert gap["nodes"] + gap["skipped"] == P
    assert gap["skipped"] == 0
    assert gap["unconverged"] == 0
    diff = np.abs(g_ex - g_est)
    print("gap %s %s t=%d %s: <|d|> = %.4e (oracle %.4e), max %.4e (oracle %.4e)"
          % (storage, scheme, t, variant, gap["mean_abs"], diff.mean(), gap["max_abs"],
             diff.max()))
    if storage == "f64":
        assert gap["mean_abs"] == pytest.approx(diff.mean(), rel=1e-10)
        assert gap["max_abs"] == pytest.approx(diff.max(), rel=1e-10)
        assert gap["mean_estimate"] == pytest.approx(g_est.mean(), rel=1e-13)
        assert gap["mean_exact"] == pytest.approx(g_ex.mean(), rel=1e-13)
    else:
        # FP32 collision: each gamma to ~1e-6, so the averages to a few 1e-6
        assert gap["mean_abs"] == pytest.approx(diff.mean(), abs=4e-6, rel=1e-3)
        assert gap["max_abs"] == pytest.approx(diff.max(), abs=4e-6, rel=1e-3)
        assert gap["mean_estimate"] == pytest.approx(g_est.mean(), abs=4e-6)
        assert gap["mean_exact"] == pytest.approx(g_ex.mean(), abs=4e-6)


def test_gap_does_not_change_the_state(kbc):
    f0 = seeded_state(9, 8, 7, noise=1e-3)
    lat = lattice((9, 8, 7), storage="f64", scheme="aa")
    lat.set_populations(f0)
    lat.step(3)
    before = lat.get_populations()
    lat.stabilizer_gap()
    assert lat.t == 3
    assert np.array_equal(lat.get_populations(), before)


def test_gap_on_the_rest_state_skips_every_node(kbc):
    lat = lattice((6, 5, 4), storage="f64", scheme="pull")
    gap = lat.stabilizer_gap()
    assert gap["nodes"] == 0 and gap["skipped"] == 6 * 5 * 4
    assert np.isnan(gap["mean_abs"]) and np.isnan(gap["mean_exact"])


def test_exact_mode_is_rejected_where_it_is_not_built(kbc):
    import torch
    lat = lattice((8, 8, 8), storage="f32", scheme="pull", gamma="exact")
    for kind in ("packed", "staged", "persistent"):
        with pytest.raises(lb.LBError) as e:
            lat.set_kernel(kind)
        assert e.value.status == lb.LB_ERR_UNSUPPORTED
    lat.set_kernel("direct")
    cfgs = [lb.make_config(8, gamma="exact", storage="f32")]
    need = lb.lb_batch_required_bytes(cfgs)
    assert need > 0
    buf = torch.empty(need + 256, dtype=torch.uint8, device="cuda")
    with pytest.raises(lb.LBError) as e:
        lb.lb_batch_create(cfgs, (buf.data_ptr() + 255) // 256 * 256, need)
    assert e.value.status == lb.LB_ERR_UNSUPPORTED
