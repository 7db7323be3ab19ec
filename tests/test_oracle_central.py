"""Pins of the oracle's central-moment KBC variants against the paper's appendix.

The oracle builds the central-basis groups as tensor products of the one-dimensional central
inverse. These tests check them against formulas the paper prints, written out here from the
appendix independently: the natural-to-central mapping (eq:cm1-eq:cm23, a subset) and the
population representation in the central basis (eq:cmf000, eq:cmf for the (s,l,0) and (s,l,d)
classes), split into the groups k~, d~ (Pi~, N~ terms), t~ (T~ term), q~ (Q~ terms).
"""
import itertools

import numpy as np
import pytest

import oracle

V, W = oracle.lattice()
IDX = {tuple(v): i for i, v in enumerate(V)}


def sample(rng, amp=0.05, umax=0.1):
    f = oracle.equilibrium(1.0 + rng.uniform(-0.02, 0.02), rng.uniform(-umax, umax, 3))
    return f * (1 + amp * rng.uniform(-1, 1, 27))


def test_natural_to_central_mapping():
    """eq:cm1-eq:cm6, eq:cm7 (Q~_xyz), eq:cm8 (Q~_xyy), and M~_022 / M~_211 from the appendix."""
    rng = np.random.default_rng(31)
    for _ in range(10):
        f = sample(rng)
        rho, M = oracle.moments(f)
        _, u, Mc = oracle.central_moments(f)
        ux, uy, uz = u
        T = M[2, 0, 0] + M[0, 2, 0] + M[0, 0, 2]
        Nxz, Nyz = M[2, 0, 0] - M[0, 0, 2], M[0, 2, 0] - M[0, 0, 2]
        Pxy, Pxz, Pyz = M[1, 1, 0], M[1, 0, 1], M[0, 1, 1]
        cPxy, cPxz, cPyz = Pxy - ux * uy, Pxz - ux * uz, Pyz - uy * uz
        cNxz = Nxz - ux ** 2 + uz ** 2
        cNyz = Nyz - uy ** 2 + uz ** 2
        cT = T - (ux ** 2 + uy ** 2 + uz ** 2)
        assert Mc[1, 1, 0] == pytest.approx(cPxy, abs=1e-15)
        assert Mc[1, 0, 1] == pytest.approx(cPxz, abs=1e-15)
        assert Mc[0, 1, 1] == pytest.approx(cPyz, abs=1e-15)
        assert Mc[2, 0, 0] - Mc[0, 0, 2] == pytest.approx(cNxz, abs=1e-15)
        assert Mc[0, 2, 0] - Mc[0, 0, 2] == pytest.approx(cNyz, abs=1e-15)
        assert Mc[2, 0, 0] + Mc[0, 2, 0] + Mc[0, 0, 2] == pytest.approx(cT, abs=1e-15)
        cQxyz = M[1, 1, 1] - ux * cPyz - uy * cPxz - uz * cPxy - ux * uy * uz
        assert Mc[1, 1, 1] == pytest.approx(cQxyz, abs=1e-15)
        cQxyy = M[1, 2, 0] - (6 * uy * cPxy + ux * (3 * uy ** 2 + 2 * cNyz - cNxz + cT)) / 3
        assert Mc[1, 2, 0] == pytest.approx(cQxyy, abs=1e-15)
        cQyzz = M[0, 1, 2] - (6 * uz * cPyz + uy * (3 * uz ** 2 - cNxz - cNyz + cT)) / 3
        assert Mc[0, 1, 2] == pytest.approx(cQyzz, abs=1e-15)
        cQxxz = M[2, 0, 1] - (6 * ux * cPxz + uz * (3 * ux ** 2 + 2 * cNxz - cNyz + cT)) / 3
        cQyyz = M[0, 2, 1] - (6 * uy * cPyz + uz * (3 * uy ** 2 + 2 * cNyz - cNxz + cT)) / 3
        assert Mc[2, 0, 1] == pytest.approx(cQxxz, abs=1e-15)
        assert Mc[0, 2, 1] == pytest.approx(cQyyz, abs=1e-15)
        cM022 = M[0, 2, 2] - (uy ** 2 * uz ** 2 + 4 * uy * uz * cPyz + (uy ** 2 + uz ** 2) * cT / 3
                              - (uy ** 2 + uz ** 2) * cNxz / 3 + (-uy ** 2 + 2 * uz ** 2) * cNyz / 3
                              + 2 * uy * cQyzz + 2 * uz * cQyyz)
        assert Mc[0, 2, 2] == pytest.approx(cM022, abs=1e-15)
        cQxxy = M[2, 1, 0] - (6 * ux * cPxy + uy * (3 * ux ** 2 + 2 * cNxz - cNyz + cT)) / 3
        cM211 = M[2, 1, 1] - (ux ** 2 * uy * uz + 2 * ux * uz * cPxy + 2 * ux * uy * cPxz
                              + ux ** 2 * cPyz + uy * uz * cT / 3 + 2 * uy * uz * cNxz / 3
                              - uy * uz * cNyz / 3 + 2 * ux * cQxyz + uz * cQxxy + uy * cQxxz)
        assert Mc[2, 1, 1] == pytest.approx(cM211, abs=1e-15)


def printed_groups(s, l, d, u, Mc):
    """Groups of one population from the appendix's central representation (per unit rho)."""
    ux, uy, uz = u
    cPxy, cPxz, cPyz = Mc[1, 1, 0], Mc[1, 0, 1], Mc[0, 1, 1]
    cT = Mc[2, 0, 0] + Mc[0, 2, 0] + Mc[0, 0, 2]
    cNxz, cNyz = Mc[2, 0, 0] - Mc[0, 0, 2], Mc[0, 2, 0] - Mc[0, 0, 2]
    Qxyz, Qxyy, Qxzz = Mc[1, 1, 1], Mc[1, 2, 0], Mc[1, 0, 2]
    Qxxy, Qyzz, Qxxz, Qyyz = Mc[2, 1, 0], Mc[0, 1, 2], Mc[2, 0, 1], Mc[0, 2, 1]
    if (s, l, d) == (0, 0, 0):                      # eq:cmf000
        k = -(ux**2 - 1) * (uy**2 - 1) * (uz**2 - 1)
        dd = (-4 * ux * uy * (uz**2 - 1) * cPxy - 4 * ux * uz * (uy**2 - 1) * cPxz
              - 4 * uy * uz * (ux**2 - 1) * cPyz
              + (ux**2 * (uy**2 + uz**2 - 2) + uz**2 * (1 - 2 * uy**2) + uy**2) * cNxz / 3
              + (uy**2 * (ux**2 + uz**2 - 2) + uz**2 * (1 - 2 * ux**2) + ux**2) * cNyz / 3)
        t = -(ux**2 * uy**2 + ux**2 * uz**2 + uy**2 * uz**2 - 2 * (ux**2 + uy**2 + uz**2) + 3) * cT / 3
        q = (-8 * ux * uy * uz * Qxyz - 2 * ux * (uz**2 - 1) * Qxyy - 2 * ux * (uy**2 - 1) * Qxzz
             - 2 * uy * (uz**2 - 1) * Qxxy - 2 * uy * (ux**2 - 1) * Qyzz
             - 2 * uz * (uy**2 - 1) * Qxxz - 2 * uz * (ux**2 - 1) * Qyyz)
        return k, dd, t, q
    if d == 0 and s != 0 and l != 0:                # eq:cmf for (sigma, lambda, 0)
        sx, ly = s + ux, l + uy
        k = -ux * uy * (uz**2 - 1) * ly * sx
        dd = (-(uz**2 - 1) * (l + 2 * uy) * (s + 2 * ux) * cPxy
              - 2 * uy * uz * ly * (s + 2 * ux) * cPxz
              # printed without the factor 2 that the (s,0,d) and (0,l,d) entries carry and that
              # exact reconstruction of f needs; read as a typo of the appendix
              - 2 * ux * uz * (l + 2 * uy) * sx * cPyz
              + (s * ux * (uy * ly + uz**2 - 1) + ux**2 * (uy * ly + uz**2 - 1)
                 - 2 * uy * (uz**2 - 1) * ly) * cNxz / 3
              + (s * ux * (uy * ly - 2 * uz**2 + 2) + ux**2 * (uy * ly - 2 * uz**2 + 2)
                 + uy * (uz**2 - 1) * ly) * cNyz / 3)
        t = (-s * ux * (uy * ly + uz**2 - 1) - ux**2 * (uy * ly + uz**2 - 1)
             - uy * (uz**2 - 1) * ly) * cT / 3
        q = (-2 * uz * (l + 2 * uy) * (s + 2 * ux) * Qxyz - (uz**2 - 1) * (s + 2 * ux) * Qxyy
             - uy * ly * (s + 2 * ux) * Qxzz - (uz**2 - 1) * (l + 2 * uy) * Qxxy
             - ux * (l + 2 * uy) * sx * Qyzz - 2 * uy * uz * ly * Qxxz - 2 * ux * uz * sx * Qyyz)
        return k / 4, dd / 4, t / 4, q / 4
    if s != 0 and l != 0 and d != 0:               # eq:cmf for (sigma, lambda, delta)
        sx, ly, dz = s + ux, l + uy, d + uz
        k = ux * uy * uz * dz * ly * sx
        dd = (uz * dz * (l + 2 * uy) * (s + 2 * ux) * cPxy + uy * (d + 2 * uz) * ly * (s + 2 * ux) * cPxz
              + ux * (d + 2 * uz) * (l + 2 * uy) * sx * cPyz
              + (-d * uz * (ux * sx - 2 * uy * ly) - uz**2 * (ux * sx - 2 * uy * ly)
                 - ux * uy * ly * sx) * cNxz / 3
              + (d * uz * (2 * ux * sx - uy * ly) + uz**2 * (2 * ux * sx - uy * ly)
                 - ux * uy * ly * sx) * cNyz / 3)
        t = (d * uz * (uy * ly + ux * sx) + uz**2 * (uy * ly + ux * sx) + ux * uy * ly * sx) * cT / 3
        q = ((d + 2 * uz) * (l + 2 * uy) * (s + 2 * ux) * Qxyz + uz * dz * (s + 2 * ux) * Qxyy
             + uy * ly * (s + 2 * ux) * Qxzz + uz * dz * (l + 2 * uy) * Qxxy
             + ux * (l + 2 * uy) * sx * Qyzz + uy * (d + 2 * uz) * ly * Qxxz
             + ux * (d + 2 * uz) * sx * Qyyz)
        return k / 8, dd / 8, t / 8, q / 8
    raise ValueError


def test_central_groups_match_the_printed_representation():
    rng = np.random.default_rng(32)
    classes = [(0, 0, 0)] + [(s, l, 0) for s in (-1, 1) for l in (-1, 1)] + \
              [(s, l, d) for s in (-1, 1) for l in (-1, 1) for d in (-1, 1)]
    for _ in range(10):
        f = sample(rng)
        rho, u, Mc = oracle.central_moments(f)
        k, d, t, q, h = oracle.central_parts(Mc, rho, u)
        assert np.allclose(k + d + t + q + h, f, atol=1e-16)
        for c in classes:
            i = IDX[c]
            pk, pd, pt, pq = printed_groups(*c, u, Mc)
            assert k[i] == pytest.approx(rho * pk, rel=1e-13, abs=1e-16), ("k", c)
            assert d[i] == pytest.approx(rho * pd, rel=1e-13, abs=1e-16), ("d", c)
            assert t[i] == pytest.approx(rho * pt, rel=1e-13, abs=1e-16), ("t", c)
            assert q[i] == pytest.approx(rho * pq, rel=1e-13, abs=1e-16), ("q", c)


def test_central_groups_carry_no_mass_or_momentum():
    rng = np.random.default_rng(33)
    for _ in range(10):
        f = sample(rng)
        rho, u, Mc = oracle.central_moments(f)
        k, d, t, q, h = oracle.central_parts(Mc, rho, u)
        assert k.sum() == pytest.approx(rho, abs=1e-15)
        assert np.allclose(V.T @ k, rho * u, atol=1e-15)
        for part in (d, t, q, h):
            assert abs(part.sum()) < 1e-15
            assert np.allclose(V.T @ part, 0.0, atol=1e-15)


BETA = oracle.beta(1e-3)
CENTRAL = [oracle.S_CD, oracle.S_CDT, oracle.S_CDQ, oracle.S_CDTQ]


@pytest.mark.parametrize("variant", CENTRAL)
def test_central_collision_conserves_and_commutes_with_symmetries(variant):
    rng = np.random.default_rng(34 + variant)
    f = sample(rng, amp=0.02)
    fo, g, _ = oracle.collide(f, BETA, variant)
    assert fo.sum() == pytest.approx(f.sum(), abs=4e-15)
    assert np.allclose(V.T @ fo, V.T @ f, atol=4e-15)
    feq = oracle.equilibrium(1.01, [0.03, -0.02, 0.05])
    fe, _, _ = oracle.collide(feq, BETA, variant)
    assert np.allclose(fe, feq, atol=1e-16, rtol=1e-15)
    assert np.allclose(oracle.collide_mirror(f, BETA, variant, g), fo, atol=1e-16)
    for perm in itertools.permutations(range(3)):
        for signs in itertools.product((1, -1), repeat=3):
            R = np.zeros((3, 3), dtype=int)
            for a in range(3):
                R[a, perm[a]] = signs[a]
            p = np.array([IDX[tuple(R @ V[i])] for i in range(27)])
            fr = np.empty(27)
            fr[p] = f
            fro, _, _ = oracle.collide(fr, BETA, variant)
            expect = np.empty(27)
            expect[p] = fo
            assert np.allclose(fro, expect, atol=1e-16)


def test_central_and_natural_dt_agree_at_rest_frame():
    """At u = 0 the central and natural moments coincide, so the groups coincide."""
    rng = np.random.default_rng(35)
    f = W * (1 + 0.02 * rng.uniform(-1, 1, 27))
    f = 0.5 * (f + f[::-1])        # f(v) = f(-v): zero momentum up to round-off
    for nat, cen in zip([oracle.S_D, oracle.S_DT, oracle.S_DQ, oracle.S_DTQ], CENTRAL):
        a, _, _ = oracle.collide(f, BETA, nat)
        b, _, _ = oracle.collide(f, BETA, cen)
        assert np.allclose(a, b, atol=1e-16)
