"""Turbulence scales of Table 2 (tab:statistics) from the diagnostics k, epsilon and nu.

Host arithmetic on three numbers the library's diagnostics return (lb_diagnostics with
8th-order gradients for the table's values); the definitions are the ones the table's
caption states:
  turbulence:  l0 = k^(3/2) / eps,  u0 = k^(1/2),  tau0 = l0 / u0,  Re0 = l0 u0 / nu
  Taylor:      u' = (2k/3)^(1/2) = u_lambda,  lambda = (15 nu u'^2 / eps)^(1/2),
               tau_lambda = lambda / u_lambda,  Re_lambda = lambda u_lambda / nu
  Kolmogorov:  eta = (nu^3 / eps)^(1/4),  u_eta = (nu eps)^(1/4),  tau_eta = (nu / eps)^(1/2)
"""
from __future__ import annotations

import math


def turbulence_scales(k: float, eps: float, nu: float) -> dict:
    l0 = k ** 1.5 / eps
    u0 = math.sqrt(k)
    ul = math.sqrt(2.0 * k / 3.0)
    lam = math.sqrt(15.0 * nu * ul * ul / eps)
    return {
        "l0": l0, "u0": u0, "tau0": l0 / u0, "Re0": l0 * u0 / nu,
        "lambda": lam, "u_lambda": ul, "tau_lambda": lam / ul, "Re_lambda": lam * ul / nu,
        "eta": (nu ** 3 / eps) ** 0.25, "u_eta": (nu * eps) ** 0.25,
        "tau_eta": math.sqrt(nu / eps),
    }


def table2_row(diag: dict, n: int, nu: float) -> dict:
    """The quantities of one Table 2 column, in the table's scaled units, from a diagnostics
    dict (kinetic_energy, enstrophy, dissipation, skewness[S3..S6]) of an N^3 run."""
    k, om, eps = diag["kinetic_energy"], diag["enstrophy"], diag["dissipation"]
    s = turbulence_scales(k, eps, nu)
    sk = diag.get("skewness", [float("nan")] * 4)
    return {
        "k_1e4": k * 1e4, "OmegaN2": om * n * n, "epsN_1e5": eps * n * 1e5,
        "S3_1e2": sk[0] * 1e2, "S4": sk[1], "S5": sk[2], "S6": sk[3],
        "l0N_1e1": s["l0"] / n * 1e1, "u0_1e2": s["u0"] * 1e2, "tau0N": s["tau0"] / n,
        "Re0": s["Re0"],
        "lamN_1e2": s["lambda"] / n * 1e2, "ulam_1e2": s["u_lambda"] * 1e2,
        "taulamN": s["tau_lambda"] / n, "Relam": s["Re_lambda"],
        "etaN_1e3": s["eta"] / n * 1e3, "ueta_1e3": s["u_eta"] * 1e3,
        "tauetaN_1e1": s["tau_eta"] / n * 1e1,
    }


def read_table2(path: str) -> dict:
    """{(quantity, t): {"A": v, "B": v, "C": v, "D": v}} from the Table 2 text fixture."""
    out = {}
    with open(path) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            q, t, a, b, c, d = line.split()
            out[(q, float(t))] = {"A": float(a), "B": float(b), "C": float(c), "D": float(d)}
    return out


RUNS = {"A": 100, "B": 200, "C": 400, "D": 600}   # N of Table 2's runs (Re = 6000, U0 = 0.05)
