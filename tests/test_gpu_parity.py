"""GPU (CUDA, through the C ABI) against the FP64 CPU oracle on the same seeded inputs.

Tolerances:
  * FP64 storage: max |df| <= 1e-12 after 100 steps (the stated FP64 bar).
  * FP32 storage, one step from identical stored inputs: every population within
    FP32_STEP_TOL of the oracle: the collision works on shifts |f - W| <~ 0.05 with ~50
    rounded operations per output at a unit round-off of 6e-8 relative to operands <~ W ~ 0.3,
    a few 1e-8 typically and 2e-7 as a bound, plus the storage rounding.
  * FP16 storage, one step: the stored half of (f - W)/W equals the oracle's result rounded
    to half, or is one half-ulp away (the two sides round values that differ by FP32 error).
  * Index/layout work (set/get round trips, pull vs AA, batch vs single box, checkpoints):
    bit-exact.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1507_02518_gb300 import lb, workloads

pytestmark = pytest.mark.gpu

V, W = oracle.lattice()
W4 = W.reshape(27, 1, 1, 1)
FP64_TOL = 1e-12
FP32_STEP_TOL = 2e-7


def seeded_state(nx, ny, nz, seed=3, u0=0.05, noise=1e-4):
    """Taylor-Green-like velocity on any box, plus multiplicative noise 1e-4 on populations."""
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    kx, ky, kz = 2 * math.pi / nx, 2 * math.pi / ny, 2 * math.pi / nz
    u = np.zeros((3, nz, ny, nx))
    u[0] = u0 * np.sin(kx * x) * np.cos(ky * y) * np.cos(kz * z)
    u[1] = -u0 * np.cos(kx * x) * np.sin(ky * y) * np.cos(kz * z)
    u[2] = 0.3 * u0 * np.sin(kz * z) * np.cos(kx * x)
    rho = 1.0 + 0.01 * np.cos(kx * x + ky * y)
    f = oracle.init_equilibrium(rho, u)
    return f * (1.0 + noise * workloads.population_noise(nx, ny, nz, seed))


def lattice(shape, **kw):
    nx, ny, nz = shape
    return lb.Lattice(nx, ny, nz, **kw)


# ------------------------------------------------------------------ layout and transfer

@pytest.mark.parametrize("scheme", ["pull", "aa"])
@pytest.mark.parametrize("t", [0, 1, 4, 7])
def test_set_get_roundtrip_is_exact_fp64(kbc, scheme, t):
    f = seeded_state(5, 7, 9)
    lat = lattice((5, 7, 9), storage="f64", scheme=scheme)
    lb.lb_set_time(lat.ctx, t)
    lat.set_populations(f)
    g = lat.get_populations()
    # stored as f - W in FP64: the round trip may move the last bit of f only
    assert np.max(np.abs(g - f)) <= 1.2e-16


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_set_get_rounds_to_storage(kbc, storage):
    f = seeded_state(6, 5, 4)
    lat = lattice((6, 5, 4), storage=storage, scheme="aa")
    lat.set_populations(f)
    g = lat.get_populations()
    if storage == "f32":
        expect = W4 + (f - W4).astype(np.float32).astype(np.float64)
    else:
        expect = W4 + W4 * ((f - W4) / W4).astype(np.float16).astype(np.float64)
    assert np.max(np.abs(g - expect)) <= 1e-16


@pytest.mark.parametrize("scheme", ["pull", "aa"])
def test_init_field_matches_oracle_equilibrium(kbc, scheme):
    import torch
    rho, u = workloads.kida(12, 0.05)
    rho = rho * (1.0 + 0.02 * np.sin(np.arange(12))[None, None, :])
    ref = oracle.init_equilibrium(rho, u)
    lat = lattice((12, 12, 12), storage="f64", scheme=scheme)
    lat.init_field(rho, u)                                     # host path
    assert lat.t == 0
    assert np.max(np.abs(lat.get_populations() - ref)) <= 2e-16
    lat.init_field(torch.from_numpy(rho).cuda(), torch.from_numpy(u).cuda())   # device path
    assert np.max(np.abs(lat.get_populations() - ref)) <= 2e-16


def test_zero_steps_is_identity(kbc):
    f = seeded_state(8, 8, 8)
    lat = lattice((8, 8, 8), storage="f64", scheme="aa")
    lat.set_populations(f)
    lat.step(0)
    assert lat.t == 0
    assert np.array_equal(lat.get_populations(), lat.get_populations())
    with pytest.raises(lb.LBError):
        lat.step(-1)


# ------------------------------------------------------------------ FP64 parity

@pytest.mark.parametrize("scheme", ["pull", "aa"])
def test_fp64_matches_oracle_100_steps_32cubed(kbc, scheme):
    """32^3 Taylor-Green + seeded noise, nu = 1e-3: max |df| <= 1e-12 after 100 steps."""
    n, nu, steps = 32, 1e-3, 100
    rho, u = workloads.taylor_green(n, 0.05)
    f0 = oracle.init_equilibrium(rho, u) * (1 + 1e-4 * workloads.population_noise(n, n, n, 11))
    lat = lattice((n, n, n), nu=nu, storage="f64", scheme=scheme)
    lat.set_populations(f0)
    lat.step(steps)
    ref, _, _ = oracle.run(f0, steps, oracle.beta(nu))
    err = np.max(np.abs(lat.get_populations() - ref))
    assert err <= FP64_TOL, err


@pytest.mark.parametrize("shape", [(3, 3, 3), (5, 7, 9), (40, 6, 3), (33, 17, 5)])
@pytest.mark.parametrize("scheme", ["pull", "aa"])
def test_fp64_matches_oracle_ragged_boxes(kbc, shape, scheme):
    f0 = seeded_state(*shape)
    steps = 9
    lat = lattice(shape, nu=2e-3, storage="f64", scheme=scheme)
    lat.set_populations(f0)
    lat.step(steps)
    ref, _, _ = oracle.run(f0, steps, oracle.beta(2e-3))
    assert np.max(np.abs(lat.get_populations() - ref)) <= FP64_TOL


@pytest.mark.parametrize("variant", ["d", "d+t", "d+q", "d+t+q", "cd", "cd+ct", "cd+cq", "cd+ct+cq"])
@pytest.mark.parametrize("gamma", ["estimate", "lbgk", "rlb"])
def test_fp64_matches_oracle_variants(kbc, variant, gamma):
    f0 = seeded_state(10, 9, 8, noise=1e-3)
    steps = 6
    nu = 5e-4
    lat = lattice((10, 9, 8), nu=nu, storage="f64", scheme="aa", variant=variant, gamma=gamma)
    lat.set_populations(f0)
    lat.step(steps)
    ref, _, _ = oracle.run(f0, steps, oracle.beta(nu), lb.VARIANT[variant], lb.GAMMA[gamma])
    assert np.max(np.abs(lat.get_populations() - ref)) <= FP64_TOL


@pytest.mark.parametrize("bx,by", [(32, 2), (64, 1), (32, 8), (128, 2)])
def test_fp64_launch_shapes_agree(kbc, bx, by):
    f0 = seeded_state(37, 11, 5)
    lat = lattice((37, 11, 5), storage="f64", scheme="pull")
    lat.set_kernel("direct")
    lat.set_block(bx, by)
    lat.set_populations(f0)
    lat.step(3)
    ref, _, _ = oracle.run(f0, 3, oracle.beta(1e-3))
    assert np.max(np.abs(lat.get_populations() - ref)) <= FP64_TOL


# ------------------------------------------------------------------ cross-scheme, determinism

@pytest.mark.parametrize("storage", ["f64", "f32", "f16"])
@pytest.mark.parametrize("steps", [7, 8])
@pytest.mark.parametrize("kind", ["direct", "packed"])
def test_pull_and_aa_are_bitwise_identical(kbc, storage, steps, kind):
    if kind == "packed" and storage == "f64":
        pytest.skip("no packed FP64")
    f0 = seeded_state(20, 12, 9)
    out = []
    for scheme in ("pull", "aa"):
        lat = lattice((20, 12, 9), storage=storage, scheme=scheme)
        lat.set_kernel(kind)
        lat.set_populations(f0)
        lat.step(steps)
        out.append(lat.get_populations())
    assert np.array_equal(out[0], out[1])


@pytest.mark.parametrize("storage", ["f64", "f32", "f16"])
@pytest.mark.parametrize("scheme", ["pull", "aa"])
@pytest.mark.parametrize("shape", [(200, 3, 4), (256, 5, 3), (8, 6, 5), (40, 3, 3)])
def test_all_step_kernels_are_bitwise_identical(kbc, storage, scheme, shape):
    """Every step kernel -- direct, shared-memory staged (bulk copies, several x-segments,
    ragged last segment, periodic wrap inside the staged rows), persistent (with and without L2
    prefetch), packed (x, x + 32) pairs and adjacent pairs -- gives identical bits: the FP32
    kernels of one node per thread run the FP32x2 collision with the node in both lanes."""
    f0 = seeded_state(*shape, seed=9)
    out = []
    for kind, pf in (("direct", 2), ("staged", 2), ("persistent", 0), ("persistent", 3)):
        lat = lattice(shape, storage=storage, scheme=scheme)
        lat.set_kernel(kind)
        lb.lb_set_prefetch(lat.ctx, pf)
        lat.set_populations(f0)
        lat.step(5)
        out.append(lat.get_populations())
    for o in out[1:]:
        assert np.array_equal(out[0], o)
    ref, _, _ = oracle.run(f0, 5, oracle.beta(1e-3))
    tol = {"f64": FP64_TOL, "f32": 1e-6, "f16": 2e-3}[storage]
    assert np.max(np.abs(out[0] - ref)) <= tol
    if storage != "f64":
        for kind in ("packed", "adj"):
            lat = lattice(shape, storage=storage, scheme=scheme)
            if kind == "adj" and shape[0] % 2:
                continue
            lat.set_kernel(kind)
            lat.set_populations(f0)
            lat.step(5)
            assert np.array_equal(lat.get_populations(), out[0]), kind


@pytest.mark.parametrize("storage", ["f32", "f16"])
@pytest.mark.parametrize("scheme", ["pull", "aa"])
@pytest.mark.parametrize("shape", [(256, 5, 3), (64, 8, 5), (32, 16, 3), (128, 6, 4),
                                   (96, 4, 3), (24, 8, 3), (512, 3, 3), (768, 3, 3)])
@pytest.mark.parametrize("steps", [4, 5])
def test_two_node_kernels_match_bitwise(kbc, storage, scheme, shape, steps):
    """The row-staged kernel (whole rows of R x nx nodes, or 256-node segments with halos;
    tiles that wrap in y; odd and even AA steps) and the adjacent-pair kernel compute the same
    FP32x2 collision as the packed kernel, only on other node pairs, so the three agree bit for
    bit; all stay within the oracle tolerance."""
    f0 = seeded_state(*shape, seed=21)
    out = []
    for kind in ("packed", "rows", "adj"):
        lat = lattice(shape, storage=storage, scheme=scheme)
        lat.set_kernel(kind)
        lat.set_populations(f0)
        lat.step(steps)
        out.append(lat.get_populations())
    assert np.array_equal(out[0], out[1])
    assert np.array_equal(out[0], out[2])
    ref, _, _ = oracle.run(f0, steps, oracle.beta(1e-3))
    tol = {"f32": 1e-6, "f16": 2e-3}[storage]
    assert np.max(np.abs(out[1] - ref)) <= tol


def test_rows_kernel_rejects_shapes_it_does_not_take(kbc):
    for shape in [(100, 8, 8), (200, 4, 4), (64, 7, 3), (40, 3, 3), (300, 3, 3)]:
        lat = lattice(shape, storage="f32", scheme="aa")
        with pytest.raises(lb.LBError) as e:
            lat.set_kernel("rows")
        assert e.value.status == lb.LB_ERR_UNSUPPORTED
    lat64 = lattice((256, 3, 3), storage="f64", scheme="aa")
    with pytest.raises(lb.LBError):
        lat64.set_kernel("rows")
    latc = lattice((256, 3, 3), storage="f32", scheme="aa", variant="cd+ct+cq")
    with pytest.raises(lb.LBError):
        latc.set_kernel("rows")


@pytest.mark.parametrize("storage", ["f32", "f16"])
@pytest.mark.parametrize("kind", ["direct", "packed", "rows", "adj"])
def test_fp64_denominator_fallback_near_equilibrium(kbc, storage, kind):
    """Populations 1e-7 (relative) away from equilibrium. In FP32 storage <dh|dh> ~ 1e-14 is
    under the 1e-13 threshold at every node, so each node is collided in FP64 from its stored
    inputs: its gamma equals the oracle's gamma of the same stored state to the FP32 rounding
    of gamma (in FP32 arithmetic dh would carry a relative error of order 0.1 at this size),
    and its populations are the FP64 collision rounded to FP32. FP16 storage rounds the 1e-7
    away (its half quantum is ~2e-5 relative), leaving <dh|dh> of 1e-11 .. 1e-9 from the
    rounding: FP32 collisions whose gamma is within a few per cent of the oracle's. A state 1e-3
    away stays on the FP32 collision; there gamma agrees to 1e-3."""
    n, nu = 24, 2e-4
    rho, u = workloads.random_spectrum(n, 4, 0.04, seed=4)
    feq = oracle.init_equilibrium(rho, u)
    near_tol = 1e-6 if storage == "f32" else 5e-2
    for noise, tol in ((1e-7, near_tol), (1e-3, 1e-3)):
        f0 = feq * (1 + noise * workloads.population_noise(n, n, n, 8))
        lat = lattice((n, n, n), nu=nu, storage=storage, scheme="aa")
        lat.set_kernel(kind)
        lat.set_populations(f0)
        f_in = lat.get_populations()             # the stored (rounded) inputs
        lat.step(1)
        g_gpu = lat.gamma().astype(np.float64)
        fo, g_ref, guarded = oracle.collide_field(f_in, lat.beta, want_gamma=True)
        err = np.abs(g_gpu - g_ref) / np.maximum(np.abs(g_ref), 1.0)
        assert np.max(err) <= tol, (noise, float(np.max(err)))
        assert lat.diagnostics()["den_guard_count"] == guarded == 0
        if noise == 1e-7 and storage == "f32":
            expect = oracle.stream(fo)
            expect = W4 + (expect - W4).astype(np.float32).astype(np.float64)
            got = lat.get_populations()
            # equal, or one FP32 ulp of the shift apart where the two FP64 collisions (same
            # inputs, different operation order) straddle a rounding boundary
            assert np.max(np.abs(got - expect)) <= 4e-9
            assert np.mean(got == expect) > 0.99


@pytest.mark.parametrize("variant", ["cd", "cd+ct+cq"])
@pytest.mark.parametrize("scheme", ["pull", "aa"])
@pytest.mark.parametrize("kind", ["direct", "packed"])
def test_central_variants_fp32_one_step_parity(kbc, variant, scheme, kind):
    n = 24
    rho, u = workloads.random_spectrum(n, 4, 0.04, seed=8)
    f0 = oracle.init_equilibrium(rho, u) * (1 + 1e-4 * workloads.population_noise(n, n, n, 9))
    lat = lattice((n, n, n), nu=2e-4, storage="f32", scheme=scheme, variant=variant)
    lat.set_kernel(kind)
    lat.set_populations(f0)
    lat.step(3)
    f_in = lat.get_populations()
    ref, _, _ = oracle.run(f_in, 1, lat.beta, lb.VARIANT[variant])
    lat.step(1)
    assert np.max(np.abs(lat.get_populations() - ref)) <= FP32_STEP_TOL


def test_central_batch_matches_single_box(kbc):
    boxes = [{"n": 12, "nu": 1e-3}, {"n": 9, "ny": 14, "nz": 5, "nu": 3e-4}]
    batch = lb.Batch(boxes, storage="f32", scheme="aa", variant="cd+ct+cq")
    states = []
    for k, b in enumerate(boxes):
        nx, ny, nz = b["n"], b.get("ny", b["n"]), b.get("nz", b["n"])
        f0 = np.ascontiguousarray(seeded_state(nx, ny, nz, seed=40 + k))
        states.append(f0)
        lb.lb_set_populations(batch.box(k), f0.ctypes.data, False)
    batch.step(5)
    for k, b in enumerate(boxes):
        nx, ny, nz = b["n"], b.get("ny", b["n"]), b.get("nz", b["n"])
        single = lb.Lattice(nx, ny, nz, nu=b["nu"], storage="f32", scheme="aa",
                            variant="cd+ct+cq")
        single.set_kernel("packed")
        single.set_populations(states[k])
        single.step(5)
        got = np.empty((27, nz, ny, nx))
        lb.lb_get_populations(batch.box(k), got.ctypes.data, False)
        assert np.array_equal(got, single.get_populations())


def test_kernel_choice_is_validated(kbc):
    lat = lattice((6, 4, 4), storage="f32")   # 24-byte rows
    with pytest.raises(lb.LBError) as e:
        lat.set_kernel("staged")
    assert e.value.status == lb.LB_ERR_UNSUPPORTED
    lat64 = lattice((8, 4, 4), storage="f64")
    with pytest.raises(lb.LBError) as e:
        lat64.set_kernel("packed")
    assert e.value.status == lb.LB_ERR_UNSUPPORTED
    latc = lattice((8, 4, 4), storage="f32", variant="cd")
    with pytest.raises(lb.LBError) as e:
        latc.set_kernel("staged")
    assert e.value.status == lb.LB_ERR_UNSUPPORTED


@pytest.mark.parametrize("storage", ["f32", "f16"])
@pytest.mark.parametrize("scheme", ["pull", "aa"])
@pytest.mark.parametrize("shape", [(37, 5, 4), (3, 3, 3), (65, 4, 3)])
def test_packed_kernel_on_ragged_rows(kbc, storage, scheme, shape):
    """Packed pairs with an odd tail (x + 32 outside the row): every node written, each within
    FP32 round-off of the oracle step taken from the same stored state."""
    f0 = seeded_state(*shape, seed=4)
    lat = lattice(shape, storage=storage, scheme=scheme)
    lat.set_kernel("packed")
    lat.set_populations(f0)
    lat.step(3)
    got, ref, _ = one_step_reference(lat)
    if storage == "f32":
        assert np.max(np.abs(got - ref)) <= FP32_STEP_TOL
    else:
        h_got = ((got - W4) / W4).astype(np.float16).astype(np.float64)
        h_ref = ((ref - W4) / W4).astype(np.float16)
        ulp = np.spacing(np.abs(h_ref)).astype(np.float64)
        diff = np.abs(h_got - h_ref.astype(np.float64)) * W4
        assert np.all(diff <= ulp * W4 * 1.0001 + FP32_STEP_TOL)
    d = lat.diagnostics()
    assert d["nonfinite_count"] == 0


@pytest.mark.parametrize("kind", ["staged", "rows"])
def test_bounded_wait_reports_timeout_and_context_recovers(kbc, kind):
    """Test hook: the staged kernels issue no copies, so their first bounded wait runs out. The
    kernel returns, the next synchronising call reports LB_ERR_TIMEOUT, and the context keeps
    working once the hook is off."""
    shape = (64, 8, 8)
    f0 = seeded_state(*shape)
    lat = lattice(shape, storage="f32", scheme="pull")
    lat.set_kernel(kind)
    lat.set_populations(f0)
    lb.lb_set_wait_budget(lat.ctx, 200000, True)     # ~0.1 ms at 2 GHz
    lat.step(1)
    with pytest.raises(lb.LBError) as e:
        lat.diagnostics()
    assert e.value.status == lb.LB_ERR_TIMEOUT
    with pytest.raises(lb.LBError) as e:        # the state must be rewritten first
        lat.step(1)
    assert e.value.status == lb.LB_ERR_TIMEOUT
    lb.lb_set_wait_budget(lat.ctx, 2000000000, False)
    lb.lb_set_time(lat.ctx, 0)
    lat.set_populations(f0)
    lat.step(3)
    ref, _, _ = oracle.run(f0, 3, lat.beta)
    assert np.max(np.abs(lat.get_populations() - ref)) <= 1e-6
    lat.diagnostics()


@pytest.mark.parametrize("scheme", ["pull", "aa"])
def test_checkpoint_resume_is_bitwise(kbc, scheme, tmp_path):
    f0 = seeded_state(16, 8, 6)
    a = lattice((16, 8, 6), storage="f32", scheme=scheme)
    a.set_populations(f0)
    a.step(11)
    ref = a.get_populations()
    b = lattice((16, 8, 6), storage="f32", scheme=scheme)
    b.set_populations(f0)
    b.step(5)
    path = str(tmp_path / "ck.bin")
    b.save_checkpoint(path)
    c = lattice((16, 8, 6), storage="f32", scheme=scheme)
    c.load_checkpoint(path)
    assert c.t == 5
    c.step(6)
    assert np.array_equal(c.get_populations(), ref)
    # a truncated checkpoint is rejected
    with open(path, "rb") as fh:
        data = fh.read()
    with open(path, "wb") as fh:
        fh.write(data[:-8])
    with pytest.raises(lb.LBError):
        c.load_checkpoint(path)


# ------------------------------------------------------------------ FP32 / FP16 parity

def one_step_reference(lat):
    """Oracle step from exactly the state the GPU holds (decoded from its storage)."""
    f_in = lat.get_populations()
    ref, _, _ = oracle.run(f_in, 1, lat.beta)
    lat.step(1)
    return lat.get_populations(), ref, f_in


@pytest.mark.parametrize("scheme", ["pull", "aa"])
@pytest.mark.parametrize("kind", ["direct", "packed", "rows", "adj"])
def test_fp32_one_step_parity(kbc, scheme, kind):
    n = 24
    rho, u = workloads.random_spectrum(n, 4, 0.04, seed=1)
    f0 = oracle.init_equilibrium(rho, u) * (1 + 1e-4 * workloads.population_noise(n, n, n, 5))
    lat = lattice((n, n, n), nu=2e-4, storage="f32", scheme=scheme)
    lat.set_kernel(kind)
    lat.set_populations(f0)
    lat.step(3)                      # odd number: AA is in its swapped layout
    got, ref, _ = one_step_reference(lat)
    err = np.max(np.abs(got - ref))
    assert err <= FP32_STEP_TOL, err


@pytest.mark.parametrize("scheme", ["pull", "aa"])
@pytest.mark.parametrize("kind", ["direct", "packed", "rows", "adj"])
def test_fp16_one_step_parity_within_one_half_ulp(kbc, scheme, kind):
    n = 24
    rho, u = workloads.random_spectrum(n, 4, 0.04, seed=2)
    f0 = oracle.init_equilibrium(rho, u) * (1 + 1e-4 * workloads.population_noise(n, n, n, 6))
    lat = lattice((n, n, n), nu=2e-4, storage="f16", scheme=scheme)
    lat.set_kernel(kind)
    lat.set_populations(f0)
    lat.step(2)
    got, ref, _ = one_step_reference(lat)
    h_got = ((got - W4) / W4).astype(np.float16)
    h_ref = ((ref - W4) / W4).astype(np.float16)
    # The two sides round to half values that differ by the FP32 error of the collision, so
    # allow one half-ulp plus that error (it dominates near zero, where halves are subnormal).
    ulp = np.spacing(np.abs(h_ref)).astype(np.float64)
    diff = np.abs(h_got.astype(np.float64) - h_ref.astype(np.float64)) * W4
    assert np.all(diff <= ulp * W4 * 1.0001 + FP32_STEP_TOL), float(np.max(diff))
    assert np.mean(h_got == h_ref) > 0.99


def test_fp32_and_fp16_trajectory_error_vs_fp64(kbc):
    """Stated error of the reduced-precision storage after 100 steps on a 24^3 random field."""
    n, nu, steps = 24, 2e-4, 100
    rho, u = workloads.random_spectrum(n, 4, 0.04, seed=3)
    f0 = oracle.init_equilibrium(rho, u)
    ref, _, _ = oracle.run(f0, steps, oracle.beta(nu))
    errs = {}
    for storage in ("f32", "f16"):
        lat = lattice((n, n, n), nu=nu, storage=storage, scheme="aa")
        lat.init_field(rho, u)
        lat.step(steps)
        errs[storage] = float(np.max(np.abs(lat.get_populations() - ref)))
    # measured on GB300: f32 4.8e-7, f16 5.0e-4 (max |df| over all populations); the bounds
    # leave a factor of about 2 for changes in rounding order
    assert errs["f32"] <= 1e-6, errs
    assert errs["f16"] <= 1e-3, errs


# ------------------------------------------------------------------ moments and diagnostics

@pytest.mark.parametrize("scheme", ["pull", "aa"])
def test_moments_and_diagnostics_match_oracle(kbc, scheme):
    n, nu = 16, 1e-3
    rho, u = workloads.kida(n, 0.05)
    f0 = oracle.init_equilibrium(rho, u)
    lat = lattice((n, n, n), nu=nu, storage="f64", scheme=scheme)
    lat.set_populations(f0)
    lat.step(4)
    f_prev = lat.get_populations()
    lat.step(1)
    f = lat.get_populations()
    r_ref, u_ref = oracle.macroscopic(f)
    r_gpu, u_gpu = lat.moments()
    assert np.max(np.abs(r_gpu - r_ref)) <= 1e-14
    assert np.max(np.abs(u_gpu - u_ref)) <= 1e-14
    d = lat.diagnostics()
    dref = oracle.diagnostics(r_ref, u_ref, nu)
    assert d["step"] == 5 and d["nodes"] == n ** 3
    assert d["mass"] == pytest.approx(dref["mass"], rel=1e-13)
    assert np.allclose(d["momentum"], dref["momentum"], atol=1e-12)
    for key in ("kinetic_energy", "enstrophy", "dissipation"):
        assert d[key] == pytest.approx(dref[key], rel=1e-10), key
    # gamma statistics of the collision that produced f (recorded in FP32 per node)
    _, g_ref, guarded = oracle.collide_field(f_prev, lat.beta, want_gamma=True)
    assert d["gamma_mean"] == pytest.approx(float(np.mean(g_ref)), rel=1e-6)
    assert d["gamma_std"] == pytest.approx(float(np.std(g_ref)), rel=1e-4, abs=1e-7)
    assert d["den_guard_count"] == guarded
    assert d["nonfinite_count"] == 0
    assert d["grad_order"] == 2
    assert np.allclose(d["skewness"], dref["skewness"], rtol=1e-9, atol=1e-12)


@pytest.mark.parametrize("storage,rel", [("f64", 1e-10), ("f32", 2e-4)])
@pytest.mark.parametrize("shape", [(16, 16, 16), (20, 9, 5), (3, 3, 3)])
def test_eighth_order_diagnostics_match_oracle(kbc, storage, rel, shape):
    """Table 2's gradient statistics (8th-order central differences) on ragged and tiny boxes
    (the 9-point stencil wraps more than once around a 3-node period)."""
    nx, ny, nz = shape
    f0 = seeded_state(nx, ny, nz, noise=1e-3)
    lat = lattice(shape, nu=1e-3, storage=storage, scheme="aa")
    lat.set_populations(f0)
    lat.step(3)
    lat.set_diag_order(8)
    d = lat.diagnostics()
    r, u = oracle.macroscopic(lat.get_populations())
    dref = oracle.diagnostics(r, u, 1e-3, order=8)
    assert d["grad_order"] == 8
    for key in ("kinetic_energy", "enstrophy", "dissipation", "dudx2"):
        assert d[key] == pytest.approx(dref[key], rel=rel), key
    assert np.allclose(d["skewness"], dref["skewness"], rtol=50 * rel, atol=50 * rel)
    with pytest.raises(lb.LBError):
        lat.set_diag_order(4)


def test_rest_state_is_exact_and_guarded(kbc):
    lat = lattice((8, 6, 4), storage="f32", scheme="pull")
    lat.step(3)
    f = lat.get_populations()
    assert np.array_equal(f, np.broadcast_to(W4, f.shape))
    d = lat.diagnostics()
    assert d["den_guard_count"] == 8 * 6 * 4 and d["gamma_mean"] == 2.0


def test_nonfinite_is_reported(kbc):
    f = seeded_state(6, 6, 6)
    f[3, 2, 2, 2] = np.nan
    lat = lattice((6, 6, 6), storage="f32", scheme="aa")
    lat.set_populations(f)
    lat.step(2)
    with pytest.raises(lb.LBError) as e:
        lat.diagnostics()
    assert e.value.status == lb.LB_ERR_NONFINITE
    d = lat.diagnostics(raise_nonfinite=False)
    assert d["nonfinite_count"] > 0


# ------------------------------------------------------------------ batched ensemble

@pytest.mark.parametrize("storage,scheme,kind", [("f32", "pull", "direct"), ("f32", "aa", "direct"),
                                                 ("f64", "pull", "direct"), ("f16", "aa", "direct"),
                                                 ("f32", "pull", "packed"), ("f32", "aa", "packed"),
                                                 ("f16", "aa", "packed"), ("f16", "pull", "packed"),
                                                 ("f32", "pull", "adj"), ("f32", "aa", "adj"),
                                                 ("f16", "aa", "adj"), ("f16", "pull", "adj")])
def test_batch_matches_single_boxes_bitwise(kbc, storage, scheme, kind):
    if kind == "adj":   # every nx even; rows of 4, 10, 12 and 34 nodes (items cross rows)
        boxes = [{"n": 12, "nu": 1e-3}, {"n": 10, "ny": 14, "nz": 5, "nu": 3e-4},
                 {"n": 34, "ny": 4, "nz": 6, "nu": 2e-5}, {"n": 4, "ny": 6, "nz": 3, "nu": 1e-3}]
    else:
        boxes = [{"n": 12, "nu": 1e-3}, {"n": 9, "ny": 14, "nz": 5, "nu": 3e-4},
                 {"n": 33, "ny": 4, "nz": 6, "nu": 2e-5}]
    batch = lb.Batch(boxes, storage=storage, scheme=scheme)
    batch.set_kernel(kind)
    states = []
    for k, b in enumerate(boxes):
        nx, ny, nz = b["n"], b.get("ny", b["n"]), b.get("nz", b["n"])
        f0 = seeded_state(nx, ny, nz, seed=20 + k)
        states.append(f0)
        view = batch.box(k)
        ff = np.ascontiguousarray(f0)
        lb.lb_set_populations(view, ff.ctypes.data, False)
    batch.set_tile(128, 64 if kind == "direct" else 256)
    batch.step(5)
    batch.step(2)
    for k, b in enumerate(boxes):
        nx, ny, nz = b["n"], b.get("ny", b["n"]), b.get("nz", b["n"])
        single = lb.Lattice(nx, ny, nz, nu=b["nu"], storage=storage, scheme=scheme)
        single.set_kernel(kind)              # same kernel family as the batch
        single.set_populations(states[k])
        single.step(7)
        got = np.empty((27, nz, ny, nx))
        lb.lb_get_populations(batch.box(k), got.ctypes.data, False)
        assert np.array_equal(got, single.get_populations()), k
    diags = batch.diagnostics()
    assert len(diags) == len(boxes) and all(d["step"] == 7 for d in diags)


@pytest.mark.parametrize("scheme", ["pull", "aa"])
@pytest.mark.parametrize("kind", ["direct", "packed", "adj"])
def test_batch_fp64_pass_matches_single_boxes(kbc, scheme, kind):
    """Boxes 0 and 2 start 1e-7 (relative) from equilibrium, so every node of theirs goes to
    the FP64 re-collision pass; box 1 starts 1e-3 away, so none of its nodes does. Each box of
    the batch ends with the single-box populations and gammas, bit for bit."""
    boxes = [{"n": 12, "nu": 1e-3}, {"n": 10, "nu": 3e-4}, {"n": 14, "nu": 2e-4}]
    noises = [1e-7, 1e-3, 1e-7]
    batch = lb.Batch(boxes, storage="f32", scheme=scheme)
    batch.set_kernel(kind)
    states = []
    for k, (b, noise) in enumerate(zip(boxes, noises)):
        n = b["n"]
        rho, u = workloads.random_spectrum(n, 3, 0.04, seed=60 + k)
        f0 = oracle.init_equilibrium(rho, u) * (
            1 + noise * workloads.population_noise(n, n, n, 61 + k))
        states.append(np.ascontiguousarray(f0))
        lb.lb_set_populations(batch.box(k), states[-1].ctypes.data, False)
    batch.step(3)
    for k, b in enumerate(boxes):
        n = b["n"]
        single = lb.Lattice(n, nu=b["nu"], storage="f32", scheme=scheme)
        single.set_kernel(kind)
        single.set_populations(states[k])
        single.step(3)
        got = np.empty((27, n, n, n))
        lb.lb_get_populations(batch.box(k), got.ctypes.data, False)
        assert np.array_equal(got, single.get_populations()), k
        g = np.empty((n, n, n), dtype=np.float32)
        lb.lb_get_gamma(batch.box(k), g.ctypes.data, False)
        assert np.array_equal(g, single.gamma()), k
        single.close()


def test_rest_state_steps_through_the_fp64_pass(kbc):
    """At rest every FP32 node has <dh|dh> = 0 and is re-collided in FP64 each step; the
    populations stay at rest to FP32 rounding, and the pass leaves nothing flagged behind
    (the next steps from a disturbed state equal a fresh box's)."""
    n = 16
    lat = lattice((n, n, n), storage="f32", scheme="aa")
    lat.step(4)
    f = lat.get_populations()
    assert np.max(np.abs(f - W4)) <= 1e-8
    f0 = seeded_state(n, n, n, seed=70)
    lat.set_populations(f0)
    lat.step(3)
    fresh = lattice((n, n, n), storage="f32", scheme="aa")
    fresh.set_populations(f0)
    fresh.step(3)
    assert np.array_equal(lat.get_populations(), fresh.get_populations())
    assert np.array_equal(lat.gamma(), fresh.gamma())


def test_batch_adj_kernel_needs_even_rows(kbc):
    batch = lb.Batch([{"n": 12, "nu": 1e-3}, {"n": 9, "nu": 1e-3}], storage="f32", scheme="aa")
    with pytest.raises(lb.LBError) as e:
        batch.set_kernel("adj")
    assert e.value.status == lb.LB_ERR_UNSUPPORTED
    batch.set_kernel("auto")            # falls back to the (n, n + 32) pairs
    batch.step(2)
    f64 = lb.Batch([{"n": 12, "nu": 1e-3}], storage="f64", scheme="aa")
    with pytest.raises(lb.LBError) as e:
        f64.set_kernel("adj")
    assert e.value.status == lb.LB_ERR_UNSUPPORTED


def test_batch_autotune_and_graph_replay(kbc):
    boxes = [{"n": 16, "nu": 1e-3}, {"n": 24, "nu": 1e-4}]
    batch = lb.Batch(boxes, storage="f32", scheme="pull")
    th, tile, ms = batch.autotune(2)
    assert th in (128, 256, 512) and tile >= 256 and ms > 0
    rho, u = workloads.taylor_green(16, 0.03)
    lb.lb_init_field(batch.box(0), rho.ctypes.data, np.ascontiguousarray(u).ctypes.data, False)
    rho2, u2 = workloads.taylor_green(24, 0.03)
    lb.lb_init_field(batch.box(1), rho2.ctypes.data, np.ascontiguousarray(u2).ctypes.data, False)
    for _ in range(3):
        batch.step(4)            # the same graph replays
    ref = lb.Lattice(16, nu=1e-3, storage="f32", scheme="pull")
    ref.set_kernel("packed")
    ref.init_field(rho, u)
    ref.step(12)
    got = np.empty((27, 16, 16, 16))
    lb.lb_get_populations(batch.box(0), got.ctypes.data, False)
    assert np.array_equal(got, ref.get_populations())



def test_batch_step_longer_than_one_graph(kbc):
    """lb_batch_step splits n into graphs of at most 64 steps; 131 + 1 steps (chunks 64, 64, 3,
    then one step from odd parity) of an AA batch equal 132 single-box steps bitwise, and
    gamma is recorded on the last step only."""
    boxes = [{"n": 12, "nu": 2e-3}, {"n": 16, "nu": 5e-4}]
    batch = lb.Batch(boxes, storage="f32", scheme="aa")
    fields = []
    for k, b in enumerate(boxes):
        rho, u = workloads.taylor_green(b["n"], 0.04)
        fields.append((rho, u))
        lb.lb_init_field(batch.box(k), rho.ctypes.data, np.ascontiguousarray(u).ctypes.data,
                         False)
    batch.step(131)
    batch.step(1)
    diags = batch.diagnostics()
    for k, b in enumerate(boxes):
        ref = lb.Lattice(b["n"], nu=b["nu"], storage="f32", scheme="aa")
        ref.set_kernel("packed")
        ref.init_field(*fields[k])
        ref.step(132)
        got = np.empty((27, b["n"] ** 3))
        lb.lb_get_populations(batch.box(k), got.ctypes.data, False)
        assert np.array_equal(got, ref.get_populations().reshape(27, -1))
        d = ref.diagnostics()
        assert diags[k]["step"] == 132
        assert diags[k]["gamma_mean"] == d["gamma_mean"]
        assert diags[k]["den_guard_count"] == d["den_guard_count"]
        ref.close()



def test_side_stream_matches_default_stream(kbc):
    """A context on a caller-made stream (its buffer recorded on that stream) steps exactly as
    one on torch's current stream."""
    import torch
    f0 = seeded_state(12, 10, 9, seed=4)
    side = torch.cuda.Stream()
    out = []
    for st in (None, side):
        lat = lb.Lattice(12, 10, 9, storage="f32", scheme="aa", stream=st)
        lat.set_populations(f0)
        lat.step(5)
        out.append(lat.get_populations())
        lat.close()
    assert np.array_equal(out[0], out[1])


# ------------------------------------------------------------------ full-size sampled parity

def _sampled_step_check(lat, nsample, tol, rng, half=False):
    """Compare f(t+1) at sampled nodes with the oracle applied to the GPU's f(t) (FP64 copy).
    half: the result is stored in FP16, so allow one half-ulp of (f - W)/W on top of tol."""
    import torch
    nz, ny, nx = lat.shape
    P = lat.P
    dev = torch.empty((27, P), dtype=torch.float64, device="cuda")
    lb.lb_get_populations(lat.ctx, dev.data_ptr(), True)
    idx = rng.integers(0, P, nsample)
    zs, ys, xs = idx // (nx * ny), (idx // nx) % ny, idx % nx
    # the 27 neighbours x - v_i whose post-collision values stream into each sample
    nbr_nodes = []
    for i in range(27):
        vx, vy, vz = V[i]
        nbr_nodes.append(((zs - vz) % nz) * nx * ny + ((ys - vy) % ny) * nx + (xs - vx) % nx)
    nbr = np.stack(nbr_nodes)                             # [27 (direction), nsample]
    cols = torch.from_numpy(nbr.reshape(-1)).cuda()
    fin = dev[:, cols].cpu().numpy().reshape(27, 27, nsample)   # [pop, dir, sample]
    lat.step(1)
    lb.lb_get_populations(lat.ctx, dev.data_ptr(), True)
    fout = dev[:, torch.from_numpy(idx).cuda()].cpu().numpy()   # [pop, sample]
    del dev
    torch.cuda.empty_cache()
    beta = lat.beta
    worst = 0.0
    for s in range(nsample):
        for i in range(27):
            post, _, _ = oracle.collide(fin[:, i, s], beta)
            err = abs(post[i] - fout[i, s])
            if half:
                h = np.float16((post[i] - W[i]) / W[i])
                err = max(0.0, err - W[i] * float(np.spacing(np.abs(h))))
            worst = max(worst, err)
    assert worst <= tol, worst
    return worst


def test_full_size_256cubed_fp32_sampled_parity(kbc):
    """The benchmark configuration (256^3 random spectrum, FP32, pull): sampled one-step parity
    and mass conservation over 10 steps."""
    n, nu = 256, 2e-4
    rho, u = workloads.random_spectrum(n, 4, 0.04, seed=1)
    lat = lb.Lattice(n, nu=nu, storage="f32", scheme="pull")
    lat.init_field(rho, u)
    d0 = lat.diagnostics()
    lat.step(10)
    d1 = lat.diagnostics()
    assert abs(d1["mass"] - d0["mass"]) / d0["mass"] < 1e-7
    rng = np.random.default_rng(0)
    _sampled_step_check(lat, 48, FP32_STEP_TOL, rng)


def test_max_size_768cubed_fp16_aa_sampled_parity(kbc):
    """The largest configuration (768^3 = 453 M nodes, FP16 AA in place, 24.5 GB): 64-bit plane
    offsets and the in-place odd/even steps at full size. Kida field generated on the GPU."""
    import torch
    n, nu = 768, 2e-5
    _, u = workloads.kida_device(n, 0.05)
    lat = lb.Lattice(n, nu=nu, storage="f16", scheme="aa")
    lat.init_field(None, u)
    del u
    torch.cuda.empty_cache()
    d0 = lat.diagnostics()
    assert d0["kinetic_energy"] == pytest.approx(3 * 0.05 ** 2 / 8, rel=2e-3)
    lat.step(3)
    d1 = lat.diagnostics()
    assert d1["nonfinite_count"] == 0
    assert abs(d1["mass"] - d0["mass"]) / d0["mass"] < 1e-6
    rng = np.random.default_rng(1)
    _sampled_step_check(lat, 24, FP32_STEP_TOL, rng, half=True)     # the odd step t = 3 -> 4
    _sampled_step_check(lat, 24, FP32_STEP_TOL, rng, half=True)     # the even step t = 4 -> 5


def test_max_size_768cubed_fp32_aa_sampled_parity(kbc):
    """The 768^3 decaying-turbulence configuration in FP32 AA (453 M nodes, 49 GB in place):
    the first step from f_eq sends every node through the FP64 re-collision pass at full size,
    then one-step parity of the odd and the even step at sampled nodes."""
    import torch
    n, nu = 768, 2e-5
    _, u = workloads.random_spectrum_device(n, 4.0, 0.05, 1, "cuda")
    lat = lb.Lattice(n, nu=nu, storage="f32", scheme="aa")
    lat.init_field(None, u)
    del u
    torch.cuda.empty_cache()
    d0 = lat.diagnostics()
    lat.step(3)
    d1 = lat.diagnostics()
    assert d1["nonfinite_count"] == 0
    assert abs(d1["mass"] - d0["mass"]) / d0["mass"] < 1e-7
    rng = np.random.default_rng(5)
    _sampled_step_check(lat, 24, FP32_STEP_TOL, rng)     # the odd step t = 3 -> 4
    _sampled_step_check(lat, 24, FP32_STEP_TOL, rng)     # the even step t = 4 -> 5


def test_run_logs_diagnostics_as_json_lines(kbc, tmp_path):
    import json
    lat = lattice((16, 16, 16), storage="f32", scheme="aa")
    rho, u = workloads.taylor_green(16, 0.05)
    lat.init_field(rho, u)
    log = tmp_path / "diag.jsonl"
    out = lat.run(120, every=50, log=str(log))
    assert [d["step"] for d in out] == [50, 100, 120]
    lines = [json.loads(l) for l in log.read_text().splitlines()]
    assert [d["step"] for d in lines] == [50, 100, 120]
    assert all(d["mlups"] > 0 and d["nonfinite_count"] == 0 for d in lines)
    assert lines[-1]["kinetic_energy"] < lines[0]["kinetic_energy"]
