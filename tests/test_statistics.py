"""Table 2's derived scales from its own printed k and epsilon (tab:statistics caption)."""
import os

import pytest

from paper_1507_02518_gb300 import statistics as stt

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table2_kida_statistics.txt")
DERIVED = ("l0N_1e1", "u0_1e2", "tau0N", "Re0", "lamN_1e2", "ulam_1e2", "taulamN", "Relam",
           "etaN_1e3", "ueta_1e3", "tauetaN_1e1")


@pytest.mark.parametrize("run", ["A", "B", "C", "D"])
@pytest.mark.parametrize("t", [0.25, 0.5, 0.75])
def test_derived_scales_reproduce_table2(run, t):
    tab = stt.read_table2(GOLDEN)
    n = stt.RUNS[run]
    nu = 0.05 * n / 6000.0
    diag = {"kinetic_energy": tab[("k_1e4", t)][run] * 1e-4,
            "enstrophy": tab[("OmegaN2", t)][run] / n ** 2,
            "dissipation": tab[("epsN_1e5", t)][run] * 1e-5 / n}
    row = stt.table2_row(diag, n, nu)
    for q in DERIVED:
        # k and epsilon are printed to 4 digits: their rounding moves the derived values by
        # up to ~0.2 %, plus the rounding of the printed value itself
        assert row[q] == pytest.approx(tab[(q, t)][run], rel=3e-3), (q, row[q])


def test_isotropic_identities():
    s = stt.turbulence_scales(8.5e-4, 2.5e-7, 8.3e-4)
    assert s["Re_lambda"] ** 2 == pytest.approx(20.0 / 3.0 * s["Re0"], rel=1e-12)
    assert s["eta"] / s["l0"] == pytest.approx(s["Re0"] ** -0.75, rel=1e-12)
    assert s["u_eta"] * s["eta"] == pytest.approx(8.3e-4, rel=1e-12)   # Re_eta = 1
