"""Stability sweep of Sec. "Numerical Simulations": the Kida vortex at N = 100, U0 = 0.05 with
the Reynolds number Re = U0 N / nu raised in steps, for LBGK (gamma = 2), the KBC models
(gamma by eq:result21) and the regularized models RLB (gamma = 1/beta), each with any shear
part s of Table 1 or the appendix.

A run is "sensible" while its populations stay finite and its turbulence kinetic energy never
exceeds the initial one by more than 1 % (decaying turbulence cannot gain energy); it is run
until the mean enstrophy has decayed to 5 % of its initial value (the paper's stopping rule)
or a step cap. Diagnostics are checked every ``check_every`` steps. Everything runs through the
library's C ABI; the initial state is either f_eq(1, u0) or the pre-solved state.

Usage::

    python -m paper_1507_02518_gb300.stability --re 500:10000:500 --models lbgk,kbc:d+t+q,rlb:d

A model name with the suffix -poly2 (e.g. lbgk-poly2) collides with the polynomial
equilibrium eq:polynomial2 instead of the product form.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import lb, workloads


def run_one(re_number, model, variant, n=100, U0=0.05, storage="f32", scheme="aa",
            f0=None, max_time=5.0, check_every=100, decay=0.05, equilibrium="product"):
    """One run; returns dict(stable, reason, steps, t, k_max_ratio, omega_ratio).
    model: lbgk, kbc or rlb; equilibrium: product (eq:entropic_eq) or poly2 (eq:polynomial2)."""
    nu = U0 * n / re_number
    gamma = {"lbgk": "lbgk", "kbc": "estimate", "rlb": "rlb"}[model]
    lat = lb.Lattice(n, nu=nu, storage=storage, scheme=scheme, variant=variant, gamma=gamma,
                     equilibrium=equilibrium)
    try:
        if f0 is None:
            rho, u = workloads.kida(n, U0)
            lat.init_field(rho, u)
        else:
            lat.set_populations(f0)
        d0 = lat.diagnostics()
        k0, om0 = d0["kinetic_energy"], d0["enstrophy"]
        max_steps = int(round(max_time * n / U0))
        steps, kmax, reason, om = 0, 1.0, "step cap", om0
        while steps < max_steps:
            c = min(check_every, max_steps - steps)
            lat.step(c)
            steps += c
            d = lat.diagnostics(raise_nonfinite=False)
            if d["nonfinite_count"] > 0 or not np.isfinite(d["kinetic_energy"]):
                return {"stable": False, "reason": "non-finite", "steps": steps,
                        "t": steps * U0 / n, "k_max_ratio": kmax, "omega_ratio": float("nan")}
            kmax = max(kmax, d["kinetic_energy"] / k0)
            om = d["enstrophy"]
            if kmax > 1.01:
                return {"stable": False, "reason": "energy growth", "steps": steps,
                        "t": steps * U0 / n, "k_max_ratio": kmax, "omega_ratio": om / om0}
            if om < decay * om0:
                reason = "decayed"
                break
        return {"stable": True, "reason": reason, "steps": steps, "t": steps * U0 / n,
                "k_max_ratio": kmax, "omega_ratio": om / om0}
    finally:
        lat.close()


def sweep(re_values, models, presolved=False, **kw):
    """{(model, variant): [(Re, result), ...]} over the Reynolds numbers, stopping a model's
    sweep at its first unstable Re (the threshold)."""
    n, U0 = kw.get("n", 100), kw.get("U0", 0.05)
    f0 = None
    if presolved:
        _, u = workloads.kida(n, U0)
        lat = lb.Lattice(n, storage="f64", scheme="aa")
        lat.presolve(u, max_iters=40000, tol=1e-10)
        f0 = lat.get_populations()
        lat.close()
    out = {}
    for model, variant in models:
        res = []
        eq = "product"
        if model.endswith("-poly2"):
            model, eq = model[:-6], "poly2"
        for re_number in re_values:
            r = run_one(re_number, model, variant, f0=f0, equilibrium=eq, **kw)
            res.append((re_number, r))
            if not r["stable"]:
                break
        out[(model + ("-poly2" if eq == "poly2" else ""), variant)] = res
    return out


def _parse_models(text):
    models = []
    for item in text.split(","):
        if ":" in item:
            m, v = item.split(":")
        else:
            m, v = item, "d+t+q"
        models.append((m, v))
    return models


def main(argv=None):
    p = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    p.add_argument("--re", default="500:10000:500", help="start:stop:step (inclusive)")
    p.add_argument("--models", default="lbgk,kbc:d+t+q,kbc:d,rlb:d,rlb:d+t")
    p.add_argument("--storage", default="f32")
    p.add_argument("--max-time", type=float, default=5.0)
    p.add_argument("--presolved", action="store_true")
    a = p.parse_args(argv)
    lo, hi, st = (float(x) for x in a.re.split(":"))
    re_values = list(np.arange(lo, hi + 0.5 * st, st))
    t0 = time.perf_counter()
    res = sweep(re_values, _parse_models(a.models), presolved=a.presolved, storage=a.storage,
                max_time=a.max_time)
    summary = {}
    for (m, v), runs in res.items():
        last = runs[-1]
        summary["%s:%s" % (m, v)] = {
            "stable_up_to": max([r for r, x in runs if x["stable"]], default=None),
            "first_unstable": None if last[1]["stable"] else last[0],
            "reason": last[1]["reason"]}
    print(json.dumps({"wall_s": round(time.perf_counter() - t0, 1), "results": summary}))


if __name__ == "__main__":
    main()
