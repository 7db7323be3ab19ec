"""Error of reduced-precision storage against FP64 on the same workload.

Runs one workload with FP64 storage (FP64 collision; parity-checked against the CPU oracle by
the test suite) and with FP32 / FP16 storage (FP32 collision), records the diagnostics every
``every`` steps and reports, per precision:

  * the relative error of the energy-decay curve k(t), of the dissipation rate eps(t) and of
    the enstrophy Omega(t), each as the maximum over the recorded times and at the end,
  * the absolute error of <gamma>(t),
  * the velocity error at the end on a sub-lattice taking every ``stride``-th node in each
    direction (the 768^3 -> 256^3 comparison uses stride 3), and, for boxes of at most 256^3
    nodes, the maximum population error max |f - f_FP64| on the same sub-lattice.

The FP64 run is by far the slowest part (the FP64 pipe bounds it), so it can be made once
and stored (``--save-ref``: its diagnostics curve and end velocity sub-lattice, JSON + .npy)
and compared against later (``--ref``).

Usage::

    python -m paper_1507_02518_gb300.precision --n 256 --steps 2000 --every 50 \\
        --field spectrum --out result.json
    python -m paper_1507_02518_gb300.precision --n 512 --field kida --nu 5e-5 --steps 5000 \\
        --precisions none --save-ref kida512_f64
    python -m paper_1507_02518_gb300.precision --n 512 --field kida --nu 5e-5 --steps 5000 \\
        --ref kida512_f64 --precisions f32:aa,f16:aa

Everything runs through the library's C ABI; torch provides device memory.
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import lb, workloads

POP_ERROR_MAX_N = 256  # largest edge for which the end populations are compared


def _field(kind, n, seed, device, urms=0.04):
    import torch
    if kind == "spectrum" and n > 256:
        return workloads.random_spectrum_device(n, 4.0, urms, seed, device)[1]
    if kind == "kida" and n > 256:
        return workloads.kida_device(n, 0.05, device)[1]
    if kind == "spectrum":
        rho, u = workloads.random_spectrum(n, 4.0, urms, seed)
    elif kind == "kida":
        rho, u = workloads.kida(n, 0.05)
    else:
        raise ValueError(kind)
    return torch.from_numpy(u).to(device)


def run_one(n, storage, scheme, nu, u_dev, steps, every, stride):
    import torch
    lat = lb.Lattice(n, nu=nu, storage=storage, scheme=scheme)
    lat.init_field(None, u_dev)
    curve = [lat.diagnostics()]
    t0 = time.perf_counter()
    done = 0
    while done < steps:
        c = min(every, steps - done)
        lat.step(c)
        done += c
        curve.append(lat.diagnostics(raise_nonfinite=False))
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    # the end state, sub-sampled on the device before it comes to the host
    P = lat.P
    rho = torch.empty(P, dtype=torch.float64, device="cuda")
    u = torch.empty((3, P), dtype=torch.float64, device="cuda")
    lb.lb_moments(lat.ctx, rho.data_ptr(), u.data_ptr(), True)
    del rho
    vel = u.view(3, n, n, n)[:, ::stride, ::stride, ::stride].contiguous().cpu().numpy()
    del u
    f = None
    if n <= POP_ERROR_MAX_N:
        fd = torch.empty((27, P), dtype=torch.float64, device="cuda")
        lb.lb_get_populations(lat.ctx, fd.data_ptr(), True)
        f = fd.view(27, n, n, n)[:, ::stride, ::stride, ::stride].contiguous().cpu().numpy()
        del fd
    lat.close()
    del lat
    torch.cuda.empty_cache()
    return {"curve": curve, "u": vel, "f": f, "wall_s": wall}


def _rel(o, r):
    return np.abs(o - r) / np.maximum(np.abs(r), 1e-300)


def compare(ref, other):
    out = {}
    names = {"kinetic_energy": "k", "dissipation": "eps", "enstrophy": "omega"}
    for key, short in names.items():
        r = np.array([d[key] for d in ref["curve"]])
        o = np.array([d[key] for d in other["curve"]])
        e = _rel(o, r)
        out[key + "_max_rel_err"] = float(np.max(e))
        out[short + "_end_rel_err"] = float(e[-1])
    g_r = np.array([d["gamma_mean"] for d in ref["curve"][1:]])
    g_o = np.array([d["gamma_mean"] for d in other["curve"][1:]])
    out["gamma_mean_max_abs_err"] = float(np.max(np.abs(g_o - g_r)))
    if ref.get("f") is not None and other.get("f") is not None:
        out["population_max_abs_err"] = float(np.max(np.abs(other["f"] - ref["f"])))
    ur, uo = ref["u"], other["u"]
    out["velocity_max_abs_err"] = float(np.max(np.abs(uo - ur)))
    out["velocity_rms_rel_err"] = float(np.sqrt(np.mean((uo - ur) ** 2) / np.mean(ur ** 2)))
    out["nonfinite"] = int(max(d["nonfinite_count"] for d in other["curve"]))
    return out


def save_reference(ref, path, meta):
    """Stores the FP64 run: <path>.json (metadata, diagnostics curve) and <path>.npy (end
    velocity sub-lattice, rounded to FP32 to keep the file small)."""
    with open(path + ".json", "w") as fh:
        json.dump({"meta": meta, "wall_s": ref["wall_s"], "curve": ref["curve"]}, fh)
    np.save(path + ".npy", ref["u"].astype(np.float32))


def load_reference(path, meta):
    with open(path + ".json") as fh:
        d = json.load(fh)
    for k, v in meta.items():
        if d["meta"].get(k) != v:
            raise ValueError("stored reference has %s = %r, this run %r"
                             % (k, d["meta"].get(k), v))
    u = np.load(path + ".npy").astype(np.float64)
    return {"curve": d["curve"], "u": u, "f": None, "wall_s": d["wall_s"]}


def study(n=256, steps=2000, every=50, field="spectrum", nu=2e-4, stride=1, seed=1,
          precisions=(("f32", "pull"), ("f32", "aa"), ("f16", "aa")), ref_scheme="aa",
          urms=0.04, ref_path=None, save_ref=None):
    import torch
    lb.load()
    meta = {"n": n, "steps": steps, "every": every, "field": field, "nu": nu, "stride": stride,
            "seed": seed, "urms": urms, "scheme": ref_scheme}
    u = _field(field, n, seed, "cuda", urms)
    if ref_path:
        ref = load_reference(ref_path, meta)
    else:
        ref = run_one(n, "f64", ref_scheme, nu, u, steps, every, stride)
        if save_ref:
            save_reference(ref, save_ref, meta)
    res = dict(meta)
    res["reference"] = {"storage": "f64", "scheme": ref_scheme, "wall_s": ref["wall_s"],
                        "k": [d["kinetic_energy"] for d in ref["curve"]],
                        "eps": [d["dissipation"] for d in ref["curve"]],
                        "omega": [d["enstrophy"] for d in ref["curve"]],
                        "gamma_mean": [d["gamma_mean"] for d in ref["curve"]]}
    res["results"] = {}
    for storage, scheme in precisions:
        o = run_one(n, storage, scheme, nu, u, steps, every, stride)
        r = compare(ref, o)
        r["wall_s"] = o["wall_s"]
        res["results"]["%s_%s" % (storage, scheme)] = r
    del u
    torch.cuda.empty_cache()
    return res


def main(argv=None):
    p = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    p.add_argument("--n", type=int, default=256)
    p.add_argument("--steps", type=int, default=2000)
    p.add_argument("--every", type=int, default=50)
    p.add_argument("--field", choices=["spectrum", "kida"], default="spectrum")
    p.add_argument("--nu", type=float, default=2e-4)
    p.add_argument("--stride", type=int, default=1)
    p.add_argument("--urms", type=float, default=0.04)
    p.add_argument("--precisions", default="f32:pull,f32:aa,f16:aa",
                   help="comma-separated storage:scheme pairs, or 'none'")
    p.add_argument("--ref", default=None, help="compare against a stored FP64 run (path stem)")
    p.add_argument("--save-ref", default=None, help="store the FP64 run (path stem)")
    p.add_argument("--out", default=None)
    a = p.parse_args(argv)
    precs = () if a.precisions == "none" else tuple(
        tuple(x.split(":")) for x in a.precisions.split(","))
    res = study(a.n, a.steps, a.every, a.field, a.nu, a.stride, precisions=precs, urms=a.urms,
                ref_path=a.ref, save_ref=a.save_ref)
    text = json.dumps(res, indent=1)
    if a.out:
        with open(a.out, "w") as fh:
            fh.write(text)
    summary = {k: {kk: (round(vv, 8) if isinstance(vv, float) else vv) for kk, vv in v.items()}
               for k, v in res["results"].items()}
    print(json.dumps({"n": a.n, "steps": a.steps, "field": a.field,
                      "reference_wall_s": res["reference"]["wall_s"], "results": summary}))


if __name__ == "__main__":
    main()
