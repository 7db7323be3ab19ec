"""The second example of Sec. "Numerical Simulations": decaying turbulence from the random
field of eq:E0 (N = 400, u0' = 0.01, nu = 8.16497e-5; Re_lambda = 2000 initially), run to
t = N / u0' * 0.75 with KBC s = d+t+q. Reports Re_lambda(t) from 8th-order gradients and the
energy spectrum E(kappa) at the end with the slope of log E against log kappa over an
inertial range (Kolmogorov: -5/3).

Usage::

    python -m paper_1507_02518_gb300.decay --n 400 --t-end 0.75 --every 0.05 --out e0.json
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import lb, statistics, workloads


def run(n=400, t_end=0.75, every=0.05, storage="f32", scheme="pull", seed=1, presolve=False,
        fit=(3, 20)):
    import torch
    u0p, nu = workloads.E0_U0P, workloads.E0_NU
    steps_per_unit = n / u0p
    _, u = workloads.spectrum_e0(n, u0p, nu, seed=seed, device="cuda")
    lat = lb.Lattice(n, nu=nu, storage=storage, scheme=scheme, variant="d+t+q")
    t0 = time.perf_counter()
    if presolve:
        # coarse-to-fine: the pre-solved density of the truncated field on n/2 seeds the
        # pre-solve on n, which continues from it (FP32 storage: tol at its fixed point)
        from .table2 import interpolate_periodic, presolved_density_of, restrict_periodic
        rho_c = presolved_density_of(restrict_periodic(u, n // 2), storage, 2e-9)
        lat.init_field(interpolate_periodic(rho_c, n), u)
        del rho_c
        lat.presolve(u, tol=2e-9, max_iters=400000, from_current=True)
    else:
        lat.init_field(None, u)
    del u
    torch.cuda.empty_cache()
    lat.set_diag_order(8)
    curve = []

    def record():
        d = lat.diagnostics()
        s = statistics.turbulence_scales(d["kinetic_energy"], d["dissipation"], nu)
        curve.append({"t": lat.t / steps_per_unit, "k": d["kinetic_energy"],
                      "enstrophy": d["enstrophy"], "epsilon": d["dissipation"],
                      "Re_lambda": s["Re_lambda"], "nonfinite": d["nonfinite_count"]})

    record()
    total = int(round(t_end * steps_per_unit))
    chunk = max(1, int(round(every * steps_per_unit)))
    done = 0
    while done < total:
        c = min(chunk, total - done)
        lat.step(c)
        done += c
        record()
    E = lat.spectrum()
    m = np.arange(len(E))
    sel = (m >= fit[0]) & (m <= fit[1]) & (E > 0)
    slope = float(np.polyfit(np.log(m[sel]), np.log(E[sel]), 1)[0])
    wall = time.perf_counter() - t0
    lat.close()
    return {"n": n, "t_end": t_end, "steps": total, "storage": storage, "presolve": presolve,
            "wall_s": wall, "curve": curve, "spectrum": E.tolist(),
            "inertial_fit_shells": list(fit), "spectrum_slope": slope}


def main(argv=None):
    p = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    p.add_argument("--n", type=int, default=400)
    p.add_argument("--t-end", type=float, default=0.75)
    p.add_argument("--every", type=float, default=0.05)
    p.add_argument("--storage", default="f32")
    p.add_argument("--presolve", action="store_true")
    p.add_argument("--out", default=None)
    a = p.parse_args(argv)
    res = run(a.n, a.t_end, a.every, a.storage, presolve=a.presolve)
    if a.out:
        with open(a.out, "w") as fh:
            json.dump(res, fh)
    c0, c1 = res["curve"][0], res["curve"][-1]
    print(json.dumps({"n": res["n"], "steps": res["steps"], "wall_s": round(res["wall_s"], 1),
                      "Re_lambda_0": round(c0["Re_lambda"], 1),
                      "Re_lambda_end": round(c1["Re_lambda"], 1),
                      "k_end_over_k0": c1["k"] / c0["k"],
                      "spectrum_slope": round(res["spectrum_slope"], 3),
                      "finite": all(c["nonfinite"] == 0 for c in res["curve"])}))


if __name__ == "__main__":
    main()
