"""Table 2 (tab:statistics) on the GPU: the Kida vortex at Re = U0 N / nu = 6000, U0 = 0.05,
runs A, B, C with KBC s = d+t+q at N = 100, 200, 400 and the resolved reference run D with
LBGK (gamma = 2) at N = 600, statistics with 8th-order gradients at t = 0.25, 0.5, 0.75
(units of N / U0), compared with the printed values.

The initial state is f_eq(1, u0) or the pre-solved state of lb_presolve (the paper's). For
large N the pre-solve starts from a density interpolated (spectrally, the field is periodic
and smooth) from the pre-solved density of the N/2 box, and continues from it: the slow,
large-scale density modes are then already in place.

Usage::

    python -m paper_1507_02518_gb300.table2 --run C --storage f32 --coarse
    python -m paper_1507_02518_gb300.table2 --run D --storage f32 --coarse
"""
from __future__ import annotations

import argparse
import json
import os
import time

from . import lb, statistics, workloads

GOLDEN = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "tests",
                      "golden", "table2_kida_statistics.txt")
U0 = 0.05
QUANTITIES = ("k_1e4", "OmegaN2", "epsN_1e5", "S3_1e2", "S4", "S5", "S6", "l0N_1e1", "u0_1e2",
              "tau0N", "Re0", "lamN_1e2", "ulam_1e2", "taulamN", "Relam", "etaN_1e3",
              "ueta_1e3", "tauetaN_1e1")


def interpolate_periodic(field, n):
    """Spectral (zero-padding) interpolation of a periodic scalar field [m, m, m] (torch,
    float64) to [n, n, n], n >= m; the coarse Nyquist planes are dropped."""
    import torch
    m = field.shape[0]
    if n == m:
        return field.clone()
    F = torch.fft.rfftn(field)
    G = torch.zeros((n, n, n // 2 + 1), dtype=F.dtype, device=F.device)
    h = (m - 1) // 2                     # modes -h..h survive in y and z, 0..h in x
    G[: h + 1, : h + 1, : h + 1] = F[: h + 1, : h + 1, : h + 1]
    G[: h + 1, n - h:, : h + 1] = F[: h + 1, m - h:, : h + 1]
    G[n - h:, : h + 1, : h + 1] = F[m - h:, : h + 1, : h + 1]
    G[n - h:, n - h:, : h + 1] = F[m - h:, m - h:, : h + 1]
    return torch.fft.irfftn(G, s=(n, n, n)) * (float(n) / m) ** 3


def restrict_periodic(field, m):
    """Spectral truncation of a periodic field [..., n, n, n] (torch, float64) to [..., m, m, m],
    m <= n: the modes -h..h, h = (m - 1) // 2, in each direction."""
    import torch
    n = field.shape[-1]
    if m == n:
        return field.clone()
    F = torch.fft.rfftn(field, dim=(-3, -2, -1))
    h = (m - 1) // 2
    G = torch.zeros(field.shape[:-3] + (m, m, m // 2 + 1), dtype=F.dtype, device=F.device)
    for zs, zd in ((slice(0, h + 1), slice(0, h + 1)), (slice(n - h, n), slice(m - h, m))):
        for ys, yd in ((slice(0, h + 1), slice(0, h + 1)), (slice(n - h, n), slice(m - h, m))):
            G[..., zd, yd, : h + 1] = F[..., zs, ys, : h + 1]
    return torch.fft.irfftn(G, s=(m, m, m), dim=(-3, -2, -1)) * (float(m) / n) ** 3


def _presolved(u, rho_start, storage, tol, log):
    """Pre-solves the velocity field u [3, n, n, n] (torch float64 on the GPU), from rho = 1 or,
    when rho_start [m, m, m] is given, continuing from its spectral interpolation to n; returns
    the pre-solved density [n, n, n] (torch float64 on the GPU)."""
    import torch
    n = u.shape[-1]
    lat = lb.Lattice(n, storage=storage, scheme="aa")
    from_current = rho_start is not None
    if from_current:
        lat.init_field(interpolate_periodic(rho_start, n), u)
    t0 = time.perf_counter()
    it, res = lat.presolve(u, tol=tol, max_iters=400000, from_current=from_current)
    log("pre-solve N = %d (%s, %s): %d iterations, last change %.2e, %.1f s"
        % (n, storage, "from the N/2 density" if from_current else "from rho = 1", it, res,
           time.perf_counter() - t0))
    rho = torch.empty((n, n, n), dtype=torch.float64, device="cuda")
    uu = torch.empty((3, n, n, n), dtype=torch.float64, device="cuda")
    lb.lb_moments(lat.ctx, rho.data_ptr(), uu.data_ptr(), True)
    lat.close()
    return rho


def presolved_density_of(u, storage="f32", tol=2e-9, min_n=100, log=print):
    """rho [n, n, n] (torch float64 on the GPU) of the pre-solved state for the velocity field
    u [3, n, n, n] (torch float64 on the GPU), built coarse to fine: the pre-solve of the
    spectrally truncated field on the n/2 box seeds the one on the n box."""
    n = u.shape[-1]
    rho_c = None
    if n >= 2 * min_n and n % 2 == 0:
        rho_c = presolved_density_of(restrict_periodic(u, n // 2), storage, tol, min_n, log)
    return _presolved(u, rho_c, storage, tol, log)


def presolved_density(n, storage="f32", tol=2e-9, min_n=100, log=print):
    """rho [n, n, n] (torch float64 on the GPU) of the pre-solved Kida state, built coarse to
    fine from min_n upward by factors of 2 when n allows it (each level from the Kida field
    sampled on its own box)."""
    rho_c = None
    if n >= 2 * min_n and n % 2 == 0:
        rho_c = presolved_density(n // 2, storage, tol, min_n, log)
    _, u = workloads.kida_device(n, U0)
    return _presolved(u, rho_c, storage, tol, log)


def run_table2(run, storage="f32", init="presolve", presolve_storage="f64", tol=1e-10,
               coarse=False, log=print, equilibrium="product"):
    """Runs one column of Table 2; returns ({t: row}, table, info). equilibrium: product
    (eq:entropic_eq) or poly2 (eq:polynomial2) for the collision."""
    import torch
    n = statistics.RUNS[run]
    nu = U0 * n / 6000.0
    gamma = "lbgk" if run == "D" else "estimate"
    info = {"run": run, "n": n, "storage": storage, "init": init, "gamma": gamma,
            "equilibrium": equilibrium}
    lat = lb.Lattice(n, nu=nu, storage=storage, scheme="aa", variant="d+t+q", gamma=gamma,
                     equilibrium=equilibrium)
    t0 = time.perf_counter()
    if init == "presolve":
        _, u = workloads.kida_device(n, U0)
        if coarse and n >= 200:
            rho = presolved_density(n // 2, presolve_storage, tol, log=log)
            lat.init_field(interpolate_periodic(rho, n), u)
            del rho
            it, res = lat.presolve(u, tol=tol, max_iters=400000, from_current=True)
        else:
            pre = lb.Lattice(n, storage=presolve_storage, scheme="aa")
            it, res = pre.presolve(u, tol=tol, max_iters=400000)
            f = torch.empty((27, pre.P), dtype=torch.float64, device="cuda")
            lb.lb_get_populations(pre.ctx, f.data_ptr(), True)
            pre.close()
            lb.lb_set_populations(lat.ctx, f.data_ptr(), True)
            del f
        del u
        info.update(presolve_iterations=it, presolve_change=res)
        log("pre-solve N = %d: %d iterations, last change %.2e" % (n, it, res))
    else:
        rho, u = workloads.kida(n, U0)
        lat.init_field(rho, u)
    torch.cuda.empty_cache()
    info["setup_s"] = time.perf_counter() - t0
    lat.set_diag_order(8)
    tab = statistics.read_table2(GOLDEN)
    rows = {}
    done = 0
    t1 = time.perf_counter()
    for t in (0.25, 0.5, 0.75):
        steps = int(round(t * n / U0))
        lat.step(steps - done)
        done = steps
        d = lat.diagnostics()
        if d["nonfinite_count"]:
            raise RuntimeError("non-finite populations at t = %g" % t)
        rows[t] = statistics.table2_row(d, n, nu)
        for q in ("k_1e4", "OmegaN2", "epsN_1e5", "S3_1e2", "S4", "Relam", "etaN_1e3"):
            paper = tab[(q, t)][run]
            log("Table 2 run %s, %s, %s init: t = %.2f  %-9s %9.4g  paper %9.4g  (%+.2f %%)"
                % (run, storage, init, t, q, rows[t][q], paper, 100 * (rows[t][q] / paper - 1)))
    info["run_s"] = time.perf_counter() - t1
    lat.close()
    return rows, tab, info


def main(argv=None):
    p = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    p.add_argument("--run", default="A", choices=["A", "B", "C", "D"])
    p.add_argument("--storage", default="f32")
    p.add_argument("--init", default="presolve", choices=["presolve", "rest"])
    p.add_argument("--presolve-storage", default="f64")
    p.add_argument("--tol", type=float, default=1e-10)
    p.add_argument("--coarse", action="store_true",
                   help="start the pre-solve from the interpolated N/2 density")
    p.add_argument("--equilibrium", default="product", choices=["product", "poly2"])
    p.add_argument("--out", default=None)
    a = p.parse_args(argv)
    rows, tab, info = run_table2(a.run, a.storage, a.init, a.presolve_storage, a.tol, a.coarse,
                                 equilibrium=a.equilibrium)
    dev = {str(t): {q: round(100 * (row[q] / tab[(q, t)][a.run] - 1), 3) for q in QUANTITIES}
           for t, row in rows.items()}
    out = {"info": info, "rows": {str(t): r for t, r in rows.items()}, "deviation_pct": dev}
    if a.out:
        with open(a.out, "w") as fh:
            json.dump(out, fh)
    print(json.dumps({"info": info, "deviation_pct": dev}))


if __name__ == "__main__":
    main()
