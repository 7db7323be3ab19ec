"""The spectral restriction and interpolation that seed the coarse-to-fine pre-solve: exact for
band-limited periodic fields, and truncating above the coarse box's modes."""
import math

import pytest

torch = pytest.importorskip("torch")

from paper_1507_02518_gb300.table2 import interpolate_periodic, restrict_periodic


def grid(n):
    x = torch.arange(n, dtype=torch.float64) * 2 * math.pi / n
    return torch.meshgrid(x, x, x, indexing="ij")        # Z, Y, X


@pytest.mark.parametrize("m,n", [(8, 16), (9, 18), (10, 30)])
def test_band_limited_fields_round_trip(m, n):
    Z, Y, X = grid(m)
    coarse = torch.sin(X) * torch.cos(2 * Y) + 0.3 * torch.cos(3 * Z) + 0.1
    fine = interpolate_periodic(coarse, n)
    Zf, Yf, Xf = grid(n)
    expect = torch.sin(Xf) * torch.cos(2 * Yf) + 0.3 * torch.cos(3 * Zf) + 0.1
    assert (fine - expect).abs().max() < 1e-13
    assert (restrict_periodic(fine, m) - coarse).abs().max() < 1e-13


def test_restriction_drops_modes_above_the_coarse_box():
    Z, Y, X = grid(16)
    f = torch.stack([torch.sin(X) + torch.sin(7 * X), torch.cos(2 * Y), torch.sin(6 * Z)])
    g = restrict_periodic(f, 8)                              # keeps |k| <= 3
    Z8, Y8, X8 = grid(8)
    assert g.shape == (3, 8, 8, 8)
    assert (g[0] - torch.sin(X8)).abs().max() < 1e-13
    assert (g[1] - torch.cos(2 * Y8)).abs().max() < 1e-13
    assert g[2].abs().max() < 1e-13
