"""Pins of the FP64 oracle against what arXiv:1507.02518 and the mathematics fix.

Each check uses a route that does not re-type the oracle's own formula: golden values printed in
the paper, the numerical inverse of the natural-moment basis (numpy), the Lagrange condition of
the entropy maximum, conservation, cube symmetry, and the LBGK / RLB special cases.
"""
import itertools
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
V, W = oracle.lattice()


def near_eq_population(rng, rho=1.0, umax=0.08, amp=0.02):
    u = rng.uniform(-umax, umax, 3)
    feq = oracle.equilibrium(rho, u)
    return feq * (1.0 + amp * rng.uniform(-1, 1, 27))


def monomial_matrix():
    """Mat[m, i] = vix^p viy^q viz^r with m = 9p + 3q + r (eq:natmoments as a matrix)."""
    Mat = np.zeros((27, 27))
    for p, q, r in itertools.product(range(3), repeat=3):
        Mat[9 * p + 3 * q + r] = V[:, 0] ** p * V[:, 1] ** q * V[:, 2] ** r
    return Mat


# ------------------------------------------------------------------ lattice

def test_weights_match_paper_golden():
    table = {}
    for line in open(os.path.join(GOLDEN, "weights_d3q27.txt")):
        if line.startswith("#") or not line.strip():
            continue
        nnz, frac = line.split()
        table[int(nnz)] = float(Fraction(frac))
    for i in range(27):
        assert W[i] == pytest.approx(table[int(np.count_nonzero(V[i]))], rel=1e-15)
    assert W.sum() == pytest.approx(1.0, abs=1e-15)


def test_velocity_order_and_sound_speed():
    for i in range(27):
        assert i == (V[i, 0] + 1) + 3 * (V[i, 1] + 1) + 9 * (V[i, 2] + 1)
    # second moment of the weights is c_s^2 delta_ab with c_s^2 = 1/3 (eq:sound)
    second = np.einsum("i,ia,ib->ab", W, V, V)
    assert np.allclose(second, np.eye(3) / 3.0, atol=1e-16)


def test_beta_inverts_viscosity_relation():
    for nu in (1e-5, 2e-4, 1e-3, 0.1):
        b = oracle.beta(nu)
        assert 0.0 < b < 1.0
        assert (1.0 / 3.0) * (1.0 / (2.0 * b) - 0.5) == pytest.approx(nu, rel=1e-12)


# ------------------------------------------------------------------ equilibrium

def test_equilibrium_conserves_mass_and_momentum():
    rng = np.random.default_rng(1)
    for _ in range(50):
        rho = rng.uniform(0.8, 1.2)
        u = rng.uniform(-0.3, 0.3, 3)
        feq = oracle.equilibrium(rho, u)
        assert feq.sum() == pytest.approx(rho, rel=1e-14)
        assert np.allclose(V.T @ feq, rho * u, atol=1e-14)
        assert np.all(feq > 0)


def test_equilibrium_is_entropy_maximum():
    """Lagrange condition of max S (eq:S) under fixed rho, rho u: ln(f_i/W_i) is affine in v_i."""
    rng = np.random.default_rng(2)
    for _ in range(20):
        u = rng.uniform(-0.2, 0.2, 3)
        feq = oracle.equilibrium(rng.uniform(0.9, 1.1), u)
        X = np.hstack([np.ones((27, 1)), V.astype(float)])
        y = np.log(feq / W)
        coef, res, *_ = np.linalg.lstsq(X, y, rcond=None)
        assert np.max(np.abs(X @ coef - y)) < 1e-13
        # and the entropy drops along any mass- and momentum-free perturbation
        xi = rng.standard_normal(27)
        xi -= X @ np.linalg.lstsq(X, xi, rcond=None)[0]   # project out (1, v) directions
        s0 = oracle.entropy(feq)
        for eps in (1e-3, -1e-3):
            assert oracle.entropy(feq + eps * xi * feq.min()) < s0


def test_equilibrium_second_order_matches_polynomial():
    """eq:polynomial2 is the second-order truncation: the difference is O(u^3)."""
    rng = np.random.default_rng(3)
    d = rng.standard_normal(3)
    d /= np.linalg.norm(d)
    errs = []
    for a in (0.04, 0.02, 0.01):
        u = a * d
        poly = W * (1 + 3 * (V @ u) + 4.5 * (V @ u) ** 2 - 1.5 * u @ u)
        errs.append(np.max(np.abs(oracle.equilibrium(1.0, u) - poly)))
    assert errs[0] / errs[1] == pytest.approx(8.0, rel=0.1)
    assert errs[1] / errs[2] == pytest.approx(8.0, rel=0.1)


# ------------------------------------------------------------------ moments

def test_natural_moments_match_matrix_route():
    rng = np.random.default_rng(4)
    Mat = monomial_matrix()
    f = near_eq_population(rng)
    rho, M = oracle.moments(f)
    assert rho == pytest.approx(f.sum(), rel=1e-15)
    assert np.allclose(M.reshape(27), Mat @ f / rho, atol=1e-15)


def test_moment_representation_inverts_moments():
    """eq:moment_rep (with the Q labels read by counting powers) inverts eq:natmoments."""
    rng = np.random.default_rng(5)
    for _ in range(20):
        f = rng.uniform(0.001, 0.3, 27)
        rho, M = oracle.moments(f)
        assert np.allclose(oracle.moment_rep(M, rho), f, atol=1e-15)


def test_table1_matches_inverse_of_moment_basis():
    """Table 1 parts equal the columns of the numerical inverse of the moment basis."""
    Mat = monomial_matrix()
    C = np.linalg.inv(Mat)           # f = C @ (rho M)
    col = lambda p, q, r: C[:, 9 * p + 3 * q + r]
    rng = np.random.default_rng(6)
    for _ in range(20):
        f = near_eq_population(rng, amp=0.2)
        rho, M = oracle.moments(f)
        k, d, t, q = oracle.table1(M, rho)
        T = M[2, 0, 0] + M[0, 2, 0] + M[0, 0, 2]
        Nxz, Nyz = M[2, 0, 0] - M[0, 0, 2], M[0, 2, 0] - M[0, 0, 2]
        k_ref = rho * (col(0, 0, 0) + M[1, 0, 0] * col(1, 0, 0) + M[0, 1, 0] * col(0, 1, 0)
                       + M[0, 0, 1] * col(0, 0, 1))
        # M200 = (T + 2Nxz - Nyz)/3, M020 = (T - Nxz + 2Nyz)/3, M002 = (T - Nxz - Nyz)/3
        c2x, c2y, c2z = col(2, 0, 0), col(0, 2, 0), col(0, 0, 2)
        t_ref = rho * T * (c2x + c2y + c2z) / 3.0
        d_ref = rho * (Nxz * (2 * c2x - c2y - c2z) / 3.0 + Nyz * (-c2x + 2 * c2y - c2z) / 3.0
                       + M[1, 1, 0] * col(1, 1, 0) + M[1, 0, 1] * col(1, 0, 1)
                       + M[0, 1, 1] * col(0, 1, 1))
        q_ref = rho * sum(M[p, qq, r] * col(p, qq, r) for p, qq, r in
                          [(1, 2, 0), (1, 0, 2), (2, 1, 0), (0, 1, 2), (2, 0, 1), (0, 2, 1),
                           (1, 1, 1)])
        assert np.allclose(k, k_ref, atol=1e-15)
        assert np.allclose(d, d_ref, atol=1e-15)
        assert np.allclose(t, t_ref, atol=1e-15)
        assert np.allclose(q, q_ref, atol=1e-15)
        # d, t, q carry no mass and no momentum (Table 1)
        for part in (d, t, q):
            assert abs(part.sum()) < 1e-15
            assert np.allclose(V.T @ part, 0.0, atol=1e-15)


# ------------------------------------------------------------------ collision

BETA = oracle.beta(1e-3)


@pytest.mark.parametrize("variant", [oracle.S_D, oracle.S_DT, oracle.S_DQ, oracle.S_DTQ])
@pytest.mark.parametrize("mode", [oracle.GAMMA_ESTIMATE, oracle.GAMMA_LBGK, oracle.GAMMA_RLB])
def test_collision_conserves_mass_momentum(variant, mode):
    rng = np.random.default_rng(7 + variant + 10 * mode)
    for _ in range(20):
        f = near_eq_population(rng)
        fo, _, _ = oracle.collide(f, BETA, variant, mode)
        # round-off of 27-term sums of O(0.3) values: a few 1e-16 each
        assert fo.sum() == pytest.approx(f.sum(), abs=4e-15)
        assert np.allclose(V.T @ fo, V.T @ f, atol=4e-15)


def test_equilibrium_is_fixed_point_and_guard():
    rng = np.random.default_rng(8)
    for _ in range(10):
        feq = oracle.equilibrium(rng.uniform(0.9, 1.1), rng.uniform(-0.1, 0.1, 3))
        fo, _, _ = oracle.collide(feq, BETA)
        assert np.allclose(fo, feq, atol=1e-16, rtol=1e-15)
    # at rest the deviations are pure round-off; whatever gamma is, f' = f
    fo, g, guarded = oracle.collide(W.copy(), BETA)
    assert np.isfinite(g) and np.allclose(fo, W, atol=2e-16, rtol=0)


def test_lbgk_special_case():
    """gamma = 2 gives LBGK: f' = f + 2 beta (f_eq - f) (eq:LBGKmirr in eq:Egeneral)."""
    rng = np.random.default_rng(9)
    for variant in range(4):
        f = near_eq_population(rng)
        rho = f.sum()
        u = V.T @ f / rho
        ref = f + 2.0 * BETA * (oracle.equilibrium(rho, u) - f)
        fo, g, _ = oracle.collide(f, BETA, variant, oracle.GAMMA_LBGK)
        assert g == 2.0
        assert np.allclose(fo, ref, atol=1e-16)


def test_rlb_special_case_relaxes_higher_moments_to_equilibrium():
    """gamma = 1/beta: h' = h_eq, i.e. every moment outside k+s takes its equilibrium value."""
    Mat = monomial_matrix()
    rng = np.random.default_rng(10)
    in_s = {oracle.S_DT: [(1, 1, 0), (1, 0, 1), (0, 1, 1), (2, 0, 0), (0, 2, 0), (0, 0, 2)]}
    conserved = [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1)]
    f = near_eq_population(rng)
    fo, g, _ = oracle.collide(f, BETA, oracle.S_DT, oracle.GAMMA_RLB)
    assert g == pytest.approx(1.0 / BETA)
    rho = f.sum()
    feq = oracle.equilibrium(rho, V.T @ f / rho)
    for p, q, r in itertools.product(range(3), repeat=3):
        if (p, q, r) in in_s[oracle.S_DT] or (p, q, r) in conserved:
            continue
        m = Mat[9 * p + 3 * q + r]
        assert m @ fo == pytest.approx(m @ feq, abs=2e-15)
    # and the s moments are over-relaxed: s' - s_eq = (1 - 2 beta)(s - s_eq)
    for p, q, r in in_s[oracle.S_DT]:
        m = Mat[9 * p + 3 * q + r]
        assert m @ fo - m @ feq == pytest.approx((1 - 2 * BETA) * (m @ f - m @ feq), abs=2e-15)


@pytest.mark.parametrize("variant", range(4))
def test_mirror_form_equals_relaxation_form(variant):
    """eq:Egeneral + eq:ksh-mirror built from explicit k, s, h parts == the relaxation form
    f' = f - beta(2 ds + gamma dh) that the two reduce to."""
    rng = np.random.default_rng(11 + variant)
    f = near_eq_population(rng)
    fo, g, _ = oracle.collide(f, BETA, variant)
    assert np.allclose(oracle.collide_mirror(f, BETA, variant, g), fo, atol=1e-16)


def test_generalized_equilibrium_identity():
    """f' = f + 2 beta (f_GE - f), f_GE = f_eq + (gamma - 2)(h_eq - h)/2 (Sec. KBC)."""
    rng = np.random.default_rng(12)
    f = near_eq_population(rng)
    fo, g, _ = oracle.collide(f, BETA, oracle.S_DTQ)
    rho, M = oracle.moments(f)
    feq = oracle.equilibrium(rho, [M[1, 0, 0], M[0, 1, 0], M[0, 0, 1]])
    rq, Mq = oracle.moments(feq)
    k, d, t, q = oracle.table1(M, rho)
    ke, de, te, qe = oracle.table1(Mq, rq)
    h = f - k - (d + t + q)
    heq = feq - ke - (de + te + qe)
    fge = feq + 0.5 * (g - 2.0) * (heq - h)
    assert np.allclose(f + 2 * BETA * (fge - f), fo, atol=1e-16)


def _cube_symmetries():
    for perm in itertools.permutations(range(3)):
        for signs in itertools.product((1, -1), repeat=3):
            R = np.zeros((3, 3), dtype=int)
            for a in range(3):
                R[a, perm[a]] = signs[a]
            yield R


@pytest.mark.parametrize("variant", range(4))
def test_collision_commutes_with_cube_symmetries(variant):
    """All 48 symmetries of the cube: C(R f) = R C(f). Catches mislabelled moments."""
    index = {tuple(v): i for i, v in enumerate(V)}
    rng = np.random.default_rng(13 + variant)
    f = near_eq_population(rng, amp=0.05)
    fo, _, _ = oracle.collide(f, BETA, variant)
    for R in _cube_symmetries():
        perm = np.array([index[tuple(R @ V[i])] for i in range(27)])
        fr = np.empty(27)
        fr[perm] = f                     # population of v_i moves to R v_i
        fro, _, _ = oracle.collide(fr, BETA, variant)
        expect = np.empty(27)
        expect[perm] = fo
        assert np.allclose(fro, expect, atol=1e-16), R


def test_gamma_estimate_tends_to_exact_root():
    """eq:result21 is the first-order expansion of eq:result1: |gamma* - gamma| = O(|deviation|)."""
    rng = np.random.default_rng(14)
    u = rng.uniform(-0.05, 0.05, 3)
    feq0 = oracle.equilibrium(1.0, u)
    xi = rng.uniform(-1, 1, 27)
    gaps = []
    for eps in (1e-2, 5e-3, 2.5e-3, 1.25e-3):
        f = feq0 * (1 + eps * xi)
        feq, ds, dh = oracle.deltas(f)
        _, gstar, _ = oracle.collide(f, BETA)
        gex = oracle.gamma_exact(feq, ds, dh, BETA, gstar)
        gaps.append(abs(gex - gstar))
        # the exact root maximises the post-collision entropy along gamma (Sec. KBC)
        post = lambda gm: f - BETA * (2 * ds + gm * dh)
        s0 = oracle.entropy(post(gex))
        for dg in (1e-2, -1e-2):
            assert oracle.entropy(post(gex + dg)) < s0
    ratios = [gaps[i] / gaps[i + 1] for i in range(3)]
    for r in ratios:
        assert 1.6 < r < 2.4, (gaps, ratios)


@pytest.mark.parametrize("seed,eps,nu", [(21, 1e-2, 1e-3), (22, 5e-2, 1e-4), (23, 2e-1, 1e-2),
                                         (24, 3e-2, 0.3)])
def test_gamma_exact_is_the_entropy_critical_point(seed, eps, nu):
    """gamma* of the oracle equals a bracketing root (Brent) of dS/dgamma written out in numpy.

    S(gamma) = -sum f'_i ln(f'_i / W_i) with f' = f - beta (2 ds + gamma dh) (eq:S, eq:Egeneral);
    dS/dgamma = beta sum dh_i ln(f'_i / W_i) + beta sum dh_i, and sum dh_i = 0. The oracle solves
    eq:result1 (logarithms relative to f_eq) by Newton's method; the two conditions agree because
    ln(f_eq_i / W_i) is linear in (1, v_i) and dh carries no mass or momentum.
    """
    from scipy.optimize import brentq
    rng = np.random.default_rng(seed)
    b = oracle.beta(nu)
    u = rng.uniform(-0.08, 0.08, 3)
    f = oracle.equilibrium(1.0 + rng.uniform(-0.02, 0.02), u) * (1 + eps * rng.uniform(-1, 1, 27))
    feq, ds, dh = oracle.deltas(f)
    _, g0, _ = oracle.collide(f, b)
    gex = oracle.gamma_exact(feq, ds, dh, b, g0)
    _, gmode, _ = oracle.collide(f, b, oracle.S_DTQ, oracle.GAMMA_EXACT)
    assert gmode == gex

    def dsdg(g):
        fp = f - b * (2 * ds + g * dh)
        return float(np.sum(dh * np.log(fp / W)))

    lo, hi = gex - 0.25, gex + 0.25
    while np.any(f - b * (2 * ds + lo * dh) <= 0):
        lo = 0.5 * (lo + gex)
    while np.any(f - b * (2 * ds + hi * dh) <= 0):
        hi = 0.5 * (hi + gex)
    assert dsdg(lo) > 0 > dsdg(hi)          # S rises, then falls: a maximum in between
    root = brentq(dsdg, lo, hi, xtol=1e-15, rtol=4 * np.finfo(float).eps, maxiter=200)
    assert abs(gex - root) <= 1e-11 * (1 + abs(root)), (gex, root, g0)
    assert abs(float(np.sum(dh))) <= 1e-15


# ------------------------------------------------------------------ streaming

def test_streaming_is_periodic_permutation():
    rng = np.random.default_rng(15)
    nx, ny, nz = 5, 7, 9
    f = rng.standard_normal((27, nz, ny, nx))
    g = oracle.stream(f)
    for i in range(27):
        assert sorted(g[i].ravel()) == sorted(f[i].ravel())
        vx, vy, vz = V[i]
        assert np.array_equal(g[i], np.roll(f[i], shift=(vz, vy, vx), axis=(0, 1, 2)))
    h = f
    for _ in range(nx * ny * nz):   # lcm of 5, 7, 9 divides 315
        h = oracle.stream(h)
    assert np.array_equal(h, f)


def test_uniform_flow_is_invariant():
    nz = ny = nx = 4
    rho = np.full((nz, ny, nx), 1.03)
    u = np.zeros((3, nz, ny, nx))
    u[0], u[1], u[2] = 0.04, -0.02, 0.01
    f = oracle.init_equilibrium(rho, u)
    g, _, _ = oracle.run(f, 3, BETA)
    assert np.allclose(g, f, atol=1e-16)
