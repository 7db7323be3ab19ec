"""Benchmark of the D3Q27 KBC step on GB300: MLUPS and fraction of the HBM roofline.

Default workload (one JSON line on rank 0): decaying homogeneous isotropic turbulence on a
periodic 256^3 box (seeded random-phase solenoidal field, E(k) ~ k^4 exp(-2 (k/k0)^2), k0 = 4,
u_rms = 0.04, rho0 = 1, nu = 2e-4), KBC s = d+t+q, FP32 storage of f - W with FP32 collision,
pull streaming, kinetic-energy / enstrophy diagnostics every 50 steps. A "step" is one lattice
update of the whole box. Other storage / scheme / batched variants are reported under
"variants" in the same line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--scaling weak|strong] [--workload NAME]

N > 1 (torchrun) runs, by default, independent replicas, one per GPU (weak scaling, no
data-path collective); value = all ranks' lattice updates / max-over-ranks time. With
--scaling strong the one box of the workload is split along z into one slab per rank, and the
9 populations per face cross between neighbouring ranks every step (NCCL send/recv, overlapped
with the interior planes' update); value = the box's lattice updates / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import signal
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "MLUPS & % HBM roofline, D3Q27 KBC step; FP32/FP16/batched vs FP64 at stated err"
FALLBACK_HBM_GBS = 6800.0
BYTES_PER_LUP = {"f64": 432, "f32": 216, "f16": 108}   # read 27 + write 27 values
MAIN = {"name": "hit256_f32_pull", "n": 256, "field": "spectrum", "k0": 4.0, "urms": 0.04,
        "nu": 2e-4, "seed": 1, "storage": "f32", "scheme": "pull", "diag_every": 50}
VARIANTS = [
    {"name": "hit256_f64_pull", "n": 256, "field": "spectrum", "k0": 4.0, "urms": 0.04,
     "nu": 2e-4, "seed": 1, "storage": "f64", "scheme": "pull", "diag_every": 50, "steps": 100,
     "gap": True},
    {"name": "hit256_f32_aa", "n": 256, "field": "spectrum", "k0": 4.0, "urms": 0.04,
     "nu": 2e-4, "seed": 1, "storage": "f32", "scheme": "aa", "diag_every": 50, "steps": 400},
    {"name": "hit256_f16_aa", "n": 256, "field": "spectrum", "k0": 4.0, "urms": 0.04,
     "nu": 2e-4, "seed": 1, "storage": "f16", "scheme": "aa", "diag_every": 50, "steps": 400},
    # Kida: 1000 of the configuration's 5000 steps, so that the FP64 re-collision of the
    # smooth start (its first ~60 steps) is amortised as over a run, not a 200-step window
    {"name": "kida512_f32_aa", "n": 512, "field": "kida", "U0": 0.05, "nu": 5e-5,
     "storage": "f32", "scheme": "aa", "diag_every": 50, "steps": 1000},
    {"name": "kida512_f16_aa", "n": 512, "field": "kida", "U0": 0.05, "nu": 5e-5,
     "storage": "f16", "scheme": "aa", "diag_every": 50, "steps": 1000},
    {"name": "batch96_f32_pull", "field": "batch", "nbox": 96, "storage": "f32",
     "scheme": "pull", "steps": 200},
    {"name": "hit768_f16_aa", "n": 768, "field": "spectrum", "k0": 4.0, "urms": 0.05,
     "nu": 2e-5, "seed": 1, "storage": "f16", "scheme": "aa", "diag_every": 50, "steps": 100},
    {"name": "hit768_f32_aa", "n": 768, "field": "spectrum", "k0": 4.0, "urms": 0.05,
     "nu": 2e-5, "seed": 1, "storage": "f32", "scheme": "aa", "diag_every": 50, "steps": 100},
    {"name": "hit256_f32_pull_central", "n": 256, "field": "spectrum", "k0": 4.0, "urms": 0.04,
     "nu": 2e-4, "seed": 1, "storage": "f32", "scheme": "pull", "diag_every": 50, "steps": 400,
     "variant": "cd+ct+cq"},
    # exact stabilizer (Newton root of eq:result1 at every node and step) and its gap to the
    # estimate eq:result21 on the final state
    {"name": "hit128_f64_pull_exact", "n": 128, "field": "spectrum", "k0": 4.0, "urms": 0.04,
     "nu": 2e-4, "seed": 1, "storage": "f64", "scheme": "pull", "diag_every": 50, "steps": 50,
     "gamma": "exact", "gap": True},
    {"name": "hit128_f32_pull_exact", "n": 128, "field": "spectrum", "k0": 4.0, "urms": 0.04,
     "nu": 2e-4, "seed": 1, "storage": "f32", "scheme": "pull", "diag_every": 50, "steps": 100,
     "gamma": "exact", "gap": True},
]
# FP64-pipe instructions per lattice update of step_kernel<double> (ncu: the FP64 pipe was
# 86.8 % busy over 2.19 ms for 2,097,152 nodes, 571 instructions per node, on a 128^3 FP64
# pull box) and the GB300 FP64 pipe peak of 2 instructions per SM per cycle.
FP64_INSTR_PER_LUP = 571.0
FP64_PIPE_PER_SM_PER_CYCLE = 2.0
# DRAM bytes per lattice update of the default FP32 pull step kernel (packed FP32x2) from an ncu
# capture, keyed by a hash of the kernel sources; a changed kernel gets no traffic figure until
# it is profiled again.
NCU_TRAFFIC_PER_LUP = {
    # adj_step_kernel<float, MODE_PULL>, the bench's own launch on 256^3: 1812.01 MB read +
    # 1768.59 MB written for 16,777,216 nodes
    "8a587e2711af51ba": 3580.60e6 / 16777216,
}


def parse_workload(name):
    """hit<N>_<storage>_<scheme> (random spectrum, k0=4, u_rms=0.04, nu=2e-4),
    kida<N>_<storage>_<scheme> (U0=0.05, nu=5e-5), e.g. hit128_f32_pull, or (as a variant only)
    batch<K>_<storage>_<scheme>, the first K boxes of the uneven ensemble."""
    for v in [MAIN] + VARIANTS:
        if v["name"] == name:
            return dict(v)
    import re
    m = re.fullmatch(r"batch(\d+)_(f64|f32|f16)_(pull|aa)", name)
    if m:
        return {"name": name, "field": "batch", "nbox": int(m.group(1)), "storage": m.group(2),
                "scheme": m.group(3), "steps": 200}
    m = re.fullmatch(r"(hit|kida)(\d+)_(f64|f32|f16)_(pull|aa)", name)
    if not m:
        raise SystemExit("unknown workload %r" % name)
    fam, n, storage, scheme = m.group(1), int(m.group(2)), m.group(3), m.group(4)
    w = {"name": name, "n": n, "storage": storage, "scheme": scheme, "diag_every": 50}
    if fam == "hit":
        w.update(field="spectrum", k0=4.0, urms=0.04, nu=2e-4, seed=1)
    else:
        w.update(field="kida", U0=0.05, nu=5e-5)
    return w


KERNEL_SOURCES = ("kbc_device.cuh", "kbc_kernels.cuh", "kbc_staged.cuh", "kbc_tma.cuh",
                  "kbc_ops.h", "kbc_f32.cu", "kbc_f16.cu", "lb_api.cu")


def kernel_source_hash() -> str:
    """Hash of every source that decides the step kernels' code and launch shapes (kernel
    bodies, kernel selection and launch configuration)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1507_02518_gb300", "csrc")
    for name in KERNEL_SOURCES:
        path = os.path.join(csrc, name)
        if os.path.exists(path):
            with open(path, "rb") as fh:
                h.update(name.encode())
                h.update(fh.read())
    return h.hexdigest()[:16]


def hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        for key in ("hbm_gbs", "hbm_copy_gbs", "hbm_GBps"):
            if key in d:
                return float(d[key]), "measured"
    except (OSError, ValueError):
        pass
    return FALLBACK_HBM_GBS, "fallback"


# ---------------------------------------------------------------- distributed plumbing

def dist_init(n_gpus):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if os.environ.get("KBC_BENCH_BACKEND", "nccl") == "nccl" else "gloo"
        dist.init_process_group(backend=backend)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


class ClockSampler:
    """nvidia-smi clock / throttle sampling while the timed region runs."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        # the samples of the last run stay in the system temp folder (or BENCH_CLOCKS_DIR)
        folder = os.environ.get("BENCH_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(folder, "kbc_bench_clocks_rank%d.csv" % index)

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.QUERY,
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.fh,
                stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.send_signal(signal.SIGTERM)
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for name, val in zip(names, parts[5:9]):
                    if val.lower().startswith("active"):
                        reasons.add(name)
        except OSError:
            pass
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- workloads

def make_field(w):
    from paper_1507_02518_gb300 import workloads
    if w["field"] == "spectrum" and w["n"] > 512:
        return workloads.random_spectrum_device(w["n"], w["k0"], w["urms"], w["seed"])
    if w["field"] == "spectrum":
        return workloads.random_spectrum(w["n"], w["k0"], w["urms"], w["seed"])
    if w["field"] == "kida" and w["n"] > 512:
        return workloads.kida_device(w["n"], w["U0"])
    if w["field"] == "kida":
        return workloads.kida(w["n"], w["U0"])
    if w["field"] == "tgv":
        return workloads.taylor_green(w["n"], w.get("u0", 0.05))
    raise ValueError(w["field"])


def run_box(w, steps, warmup, want_kernel_time=True):
    """Time `steps` steps of one box (inputs resident in HBM). Returns a dict."""
    import torch
    from paper_1507_02518_gb300 import lb
    rho, u = make_field(w)
    lat = lb.Lattice(w["n"], nu=w["nu"], storage=w["storage"], scheme=w["scheme"],
                     variant=w.get("variant", "d+t+q"), gamma=w.get("gamma", "estimate"))
    st = lat.stream
    u_dev = u if isinstance(u, torch.Tensor) else torch.from_numpy(u).cuda()
    lat.init_field(None, u_dev)
    del rho, u, u_dev
    torch.cuda.empty_cache()
    lat.step(warmup)
    torch.cuda.synchronize()
    every = w.get("diag_every", 0) or steps
    chunks = []
    k = 0
    while k < steps:
        c = min(every, steps - k)
        chunks.append(c)
        k += c
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in chunks]
    e_start, e_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    diags = []
    torch.cuda.synchronize()
    e_start.record(st)
    for (a, b), c in zip(ev, chunks):
        a.record(st)
        lat.step(c)
        b.record(st)
        if w.get("diag_every"):
            diags.append(lat.diagnostics())
    e_end.record(st)
    torch.cuda.synchronize()
    total_ms = e_start.elapsed_time(e_end)
    step_ms = sum(a.elapsed_time(b) for a, b in ev)
    # per step the step kernel, plus the FP64 re-collision pass after it with FP32 storage
    # (estimate of gamma); per diagnostics call two field kernels and two final sums
    per_step = 2 if (w["storage"] == "f32" and w.get("gamma", "estimate") == "estimate") else 1
    launches = steps * per_step + 4 * len(diags)
    out = {"P": lat.P, "steps": steps, "total_ms": total_ms, "step_kernel_ms": step_ms / steps,
           "launches": launches, "diag": diags[-1] if diags else None, "lat": lat}
    return out


def run_batch(w, steps, warmup, rank=0, world=1):
    import torch
    from paper_1507_02518_gb300 import lb, sharding, workloads
    boxes = workloads.batch_boxes(w["nbox"])
    if world > 1:                                 # LPT shard of the ensemble, no exchange
        boxes, _ = sharding.shard_boxes(boxes, rank, world)
    batch = lb.Batch(boxes, storage=w["storage"], scheme=w["scheme"])
    fields = [np.ascontiguousarray(workloads.random_spectrum(b["n"], b["k0"], b["urms"],
                                                             b["seed"])[1]) for b in boxes]

    def init_fields():
        for k in range(len(boxes)):
            lb.lb_init_field(batch.box(k), 0, fields[k].ctypes.data, False)

    # tuned on the initial fields (at rest every FP32 node would take the FP64 re-collision),
    # which are then set again
    init_fields()
    tune = batch.autotune(2)
    init_fields()
    batch.step(warmup)
    torch.cuda.synchronize()
    st = batch.stream
    a, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    batch.step(steps)                             # capture the graphs for this step count
    torch.cuda.synchronize()
    a.record(st)
    batch.step(steps)                             # replay: one graph launch per 64 steps
    b_.record(st)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b_)
    diags = batch.diagnostics()
    # the same boxes stepped one at a time (box-by-box launches, no graph)
    single_ms = 0.0
    lat_steps = max(1, steps // 10)
    for k in range(len(boxes)):
        view = batch.box(k)
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(st)
        lb.lb_step(view, lat_steps)
        s1.record(st)
        torch.cuda.synchronize()
        single_ms += s0.elapsed_time(s1)
    return {"P": batch.nodes, "steps": steps, "total_ms": ms, "tune": tune,
            "single_box_ms_per_step": single_ms / lat_steps, "diags": diags}


def run_strong(w, steps, warmup, rank, world):
    """Time `steps` steps of one box split along z into one slab per rank (strong scaling):
    each step the boundary planes are stepped and their faces packed, the faces travel to the
    neighbouring ranks (NCCL point-to-point, periodic ring) while the interior planes are
    stepped, and the received faces are unpacked. No diagnostics in the timed region."""
    import torch
    from paper_1507_02518_gb300 import sharding
    from paper_1507_02518_gb300 import slab as slabmod
    dist = None
    if world > 1:
        import torch.distributed as dist
    n = w["n"]
    z0, z1 = sharding.slab_bounds(n, rank, world)
    rho, u = make_field(w)
    u_dev = u if isinstance(u, torch.Tensor) else torch.from_numpy(u).cuda()
    u_mine = u_dev[:, z0:z1].contiguous()
    del rho, u, u_dev
    torch.cuda.empty_cache()
    s = slabmod.Slab(n, n, n, z0, z1 - z0, nu=w["nu"], storage=w["storage"],
                     scheme=w["scheme"])
    s.init_field(None, u_mine)
    del u_mine
    torch.cuda.empty_cache()
    slabmod.step_distributed(s, rank, world, dist, warmup)
    torch.cuda.synchronize()
    barrier(world)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(s.stream)
    slabmod.step_distributed(s, rank, world, dist, steps)
    b.record(s.stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    nz_local = z1 - z0
    per_kernel = 2 if w["storage"] == "f32" else 1   # step kernel (+ FP64 re-collision pass)
    launches = steps * (per_kernel * ((2 if nz_local > 1 else 1) + (1 if nz_local > 2 else 0))
                        + 2)
    s.close()
    return {"P": n * n * nz_local, "P_box": n ** 3, "total_ms": ms, "launches": launches,
            "planes": [z0, z1], "face_bytes": 9 * n * n * {"f64": 8, "f32": 4, "f16": 2}[
                w["storage"]]}


def main_strong(args, rank, world, local):
    import torch
    torch.cuda.set_device(local)
    from paper_1507_02518_gb300 import lb
    lb.load()
    w = parse_workload(args.workload)
    if w["field"] == "batch":
        raise SystemExit("strong scaling splits one box; a batch shards without exchange")
    barrier(world)
    with ClockSampler(local) as clk:
        res = run_strong(w, args.steps, args.warmup, rank, world)
    barrier(world)
    ms_max = max_over_ranks(res["total_ms"], world)
    value = res["P_box"] * args.steps / (ms_max / 1e3) / 1e6
    out = None
    if rank == 0:
        peak, peak_kind = hbm_peak()
        out = {
            "metric": METRIC, "value": round(value, 1), "unit": "MLUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(ms_max / args.steps, 5), "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": w["storage"], "data": "synthetic",
            "config": {"workload": workload_text(w) + " (no diagnostics in the timed region)",
                       "box": [w["n"]] * 3, "storage": w["storage"], "scheme": w["scheme"],
                       "parallelism": "%d slabs along z, face exchange per step" % world,
                       "face_bytes_per_step_per_rank": 2 * res["face_bytes"],
                       "l2": "populations %.2f GB per rank per step vs 129 MB L2 (no flush)"
                             % (BYTES_PER_LUP[w["storage"]] * res["P"] / 1e9)},
            "roofline": roofline(w["storage"], value / world, peak, peak_kind),
            "gpu_launches": res["launches"], "clocks": clk.summary()}
        print(json.dumps(out), flush=True)
    barrier(world)
    return out


def run_e2e(w, steps):
    """Same metric through the public API with host buffers: H2D of the initial fields, the
    steps with diagnostics, D2H of the final rho and u, all inside the timed region."""
    import torch
    from paper_1507_02518_gb300 import lb
    rho, u = make_field(w)
    lat = lb.Lattice(w["n"], nu=w["nu"], storage=w["storage"], scheme=w["scheme"])
    # inputs and outputs in pinned host memory (allocated and filled before the timed region)
    rho_t = torch.from_numpy(np.ascontiguousarray(rho)).pin_memory()
    u_t = torch.from_numpy(np.ascontiguousarray(u)).pin_memory()
    rho_o = torch.empty_like(rho_t).pin_memory()
    u_o = torch.empty_like(u_t).pin_memory()
    rho, u, rho_out, u_out = rho_t.numpy(), u_t.numpy(), rho_o.numpy(), u_o.numpy()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lat.init_field(rho, u)                        # returns after its copies and kernels
    t1 = time.perf_counter()
    every = w.get("diag_every", 0) or steps
    k = 0
    while k < steps:
        c = min(every, steps - k)
        lat.step(c)
        k += c
        if w.get("diag_every"):
            lat.diagnostics()
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    lb.lb_moments(lat.ctx, rho_out.ctypes.data, u_out.ctypes.data, False)
    torch.cuda.synchronize()
    t3 = time.perf_counter()
    dt = t3 - t0
    h2d = rho.nbytes + u.nbytes
    d2h = rho_out.nbytes + u_out.nbytes + (steps // every) * (16 * 8 + 8)
    return {"value": lat.P * steps / dt / 1e6, "unit": "MLUPS",
            "h2d_bytes_per_step": h2d / steps, "d2h_bytes_per_step": d2h / steps,
            "phase_ms": {"h2d_and_init": round(1e3 * (t1 - t0), 2),
                         "steps_and_diagnostics": round(1e3 * (t2 - t1), 2),
                         "moments_and_d2h": round(1e3 * (t3 - t2), 2)}}


def cpu_baseline(w, budget_s=12.0):
    """The FP64 oracle (as it stands) on a bounded sample of the workload: a 64^3 box of the
    same field family and parameters, stepped until about budget_s seconds of CPU work."""
    import oracle
    from paper_1507_02518_gb300 import workloads
    n = 64
    if w["field"] == "spectrum":
        rho, u = workloads.random_spectrum(n, w["k0"], w["urms"], w["seed"])
    elif w["field"] == "kida":
        rho, u = workloads.kida(n, w["U0"])
    else:
        rho, u = workloads.taylor_green(n, 0.05)
    f = oracle.init_equilibrium(rho, u)
    beta = oracle.beta(w["nu"])
    steps = 0
    t0 = time.perf_counter()
    while True:
        f, _, _ = oracle.run(f, 1, beta)
        steps += 1
        if time.perf_counter() - t0 >= budget_s:
            break
    dt = time.perf_counter() - t0
    return {"value": n ** 3 * steps / dt / 1e6, "unit": "MLUPS", "cores": oracle.num_threads(),
            "kind": "oracle",
            "sample": "%d steps of a %d^3 box of the same field family (FP64 oracle, %.1f s)"
                      % (steps, n, dt)}


def workload_text(w):
    if w["field"] == "spectrum":
        fld = ("decaying HIT, seeded random solenoidal field E(k)~k^4 exp(-2(k/k0)^2), k0=%g, "
               "u_rms=%g, rho0=1, nu=%g" % (w["k0"], w["urms"], w["nu"]))
    else:
        fld = "Kida vortex U0=%g, rho0=1, nu=%g" % (w["U0"], w["nu"])
    st = {"f64": "FP64 storage + FP64 collision", "f32": "FP32 (f-W) storage + FP32 collision",
          "f16": "FP16 (f-W)/W storage + FP32 collision"}[w["storage"]]
    return "%s: periodic %d^3 %s, KBC s=d+t+q, %s, %s streaming, diagnostics every %s steps" % (
        w["name"], w["n"], fld, st, w["scheme"], w.get("diag_every"))


def roofline(storage, mlups, peak, peak_kind, traffic=None):
    bpl = BYTES_PER_LUP[storage]
    achieved = bpl * mlups * 1e6 / 1e9
    return {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "traffic": traffic,
            "peak_source": "of %s" % peak_kind, "bytes_per_lup": bpl}


# ---------------------------------------------------------------- arms

def main_ours(args, rank, world, local):
    w = parse_workload(args.workload)
    if w["field"] == "batch":
        raise SystemExit("a batch workload runs as a variant: --variants %s" % w["name"])
    import torch
    torch.cuda.set_device(local)
    from paper_1507_02518_gb300 import lb
    lb.load()
    peak, peak_kind = hbm_peak()
    # warm-up and timed region (max over ranks)
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        res = run_box(w, args.steps, args.warmup)
    barrier(world)
    torch.cuda.synchronize()
    ms_max = max_over_ranks(res["total_ms"], world)
    total_lups = sum_over_ranks(float(res["P"] * args.steps), world)
    value = total_lups / (ms_max / 1e3) / 1e6
    kernel_ms = res["step_kernel_ms"]
    kernel_mlups = res["P"] / (kernel_ms / 1e3) / 1e6
    h = kernel_source_hash()
    traffic = NCU_TRAFFIC_PER_LUP.get(h)
    if w["name"] != MAIN["name"]:
        traffic = None
    rl = roofline(w["storage"], kernel_mlups, peak, peak_kind,
                  None if traffic is None else traffic * res["P"])
    rl["kernel"] = "kbc::%s<%s, %s>" % (
        "step_kernel" if w["storage"] == "f64" else
        ("adj_step_kernel" if w["n"] % 2 == 0 else "pair_step_kernel"),
        {"f64": "double", "f32": "float", "f16": "uint16 (half bits)"}[w["storage"]],
        "MODE_PULL" if w["scheme"] == "pull" else "MODE_AA_EVEN/ODD")
    rl["kernel_ms"] = round(kernel_ms, 5)
    del res["lat"]
    torch.cuda.empty_cache()

    variants = {}
    clk_mhz = clk.summary().get("sm_mhz")
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    if not args.no_variants:
        chosen = VARIANTS if args.variants is None else [
            parse_workload(name) for name in args.variants.split(",") if name]
        for v in chosen:
            try:
                vs = v.get("steps", 200)
                if v["field"] == "batch":
                    r = run_batch(v, vs, 3, rank, world)
                    mlups = r["P"] * vs / (r["total_ms"] / 1e3) / 1e6
                    single = r["P"] / (r["single_box_ms_per_step"] / 1e3) / 1e6
                    variants[v["name"]] = {
                        "MLUPS": round(mlups, 1), "nodes": r["P"], "steps": vs,
                        "single_box_MLUPS": round(single, 1),
                        "autotune": {"threads": r["tune"][0], "tile": r["tune"][1]},
                        "frac_hbm": roofline(v["storage"], mlups, peak, peak_kind)["frac"],
                        "finite": all(d["nonfinite_count"] == 0 for d in r["diags"])}
                else:
                    r = run_box(v, vs, 3)
                    mlups = r["P"] * vs / (r["total_ms"] / 1e3) / 1e6
                    kml = r["P"] / (r["step_kernel_ms"] / 1e3) / 1e6
                    d = r["diag"]
                    variants[v["name"]] = {
                        "MLUPS": round(mlups, 1), "kernel_MLUPS": round(kml, 1), "steps": vs,
                        "frac_hbm": roofline(v["storage"], kml, peak, peak_kind)["frac"],
                        "kinetic_energy": d["kinetic_energy"], "gamma_mean": d["gamma_mean"]}
                    if v.get("gap"):
                        gp = r["lat"].stabilizer_gap()
                        variants[v["name"]]["gamma_gap"] = {
                            k: gp[k] for k in ("mean_abs", "max_abs", "mean_estimate",
                                               "mean_exact", "unconverged", "skipped")}
                    if v.get("gamma") == "exact":
                        variants[v["name"]]["bound"] = "alu (Newton iterations)"
                    elif v["storage"] == "f64":
                        sm_mhz = clk_mhz or 2070.0
                        pipe_peak = FP64_PIPE_PER_SM_PER_CYCLE * sms * sm_mhz * 1e6
                        variants[v["name"]]["bound"] = "alu (FP64 pipe)"
                        variants[v["name"]]["frac_fp64_pipe"] = round(
                            kml * 1e6 * FP64_INSTR_PER_LUP / pipe_peak, 4)
                    del r["lat"]
                torch.cuda.empty_cache()
            except Exception as e:  # report, do not hide
                variants[v["name"]] = {"error": str(e)[:200]}

    e2e = run_e2e(w, args.steps) if not args.no_e2e else None
    out = None
    if rank == 0:
        cpu = cpu_baseline(w) if (world == 1 and not args.no_cpu) else None
        out = {
            "metric": METRIC, "value": round(value, 1), "unit": "MLUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_max / args.steps, 5),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": w["storage"], "data": "synthetic",
            "config": {"workload": workload_text(w),
                       "box": [w["n"]] * 3, "storage": w["storage"], "scheme": w["scheme"],
                       "variant": "d+t+q", "diag_every": w.get("diag_every"),
                       "l2": "populations %.2f GB read+written per step vs 129 MB L2 (no flush)"
                             % (BYTES_PER_LUP[w["storage"]] * res["P"] / 1e9),
                       "parallelism": "replicas" if world > 1 else "single"},
            "roofline": rl, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": res["launches"],
            "clocks": clk.summary(),
            "diag_last": {k: res["diag"][k] for k in ("step", "kinetic_energy", "enstrophy",
                                                      "dissipation", "gamma_mean", "gamma_std",
                                                      "nonfinite_count")} if res["diag"] else None,
            "variants": variants, "kernel_hash": h,
        }
        print(json.dumps(out), flush=True)
    barrier(world)
    return out


def main_reference(args, rank, world):
    """The reference arm: the FP64 CPU oracle, as it stands, on the machine's host cores."""
    if rank != 0:
        return None
    w = dict(MAIN)
    import oracle
    from paper_1507_02518_gb300 import workloads
    # each step is a bounded sample of the workload: an n^3 sub-box of the same field family,
    # n chosen so that warm-up + timed steps stay around a minute of oracle time
    n = int(round((40e6 / max(1, args.steps + args.warmup)) ** (1.0 / 3.0)))
    n = max(8, min(64, n))
    rho, u = workloads.random_spectrum(n, w["k0"], w["urms"], w["seed"])
    f = oracle.init_equilibrium(rho, u)
    beta = oracle.beta(w["nu"])
    for _ in range(args.warmup):
        f, _, _ = oracle.run(f, 1, beta)
    t0 = time.perf_counter()
    f, _, _ = oracle.run(f, args.steps, beta)
    dt = time.perf_counter() - t0
    value = n ** 3 * args.steps / dt / 1e6
    sample = ("%d steps (after %d warm-up) of a %d^3 box of the hit256 field family "
              "(random spectrum k0=4, u_rms=0.04, nu=2e-4), FP64 oracle"
              % (args.steps, args.warmup, n))
    out = {"impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": "MLUPS",
           "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": round(dt / args.steps * 1e3, 3), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": "hit256 field family on a bounded %d^3 sample (CPU oracle)" % n,
                      "box": [n, n, n]},
           "cpu_baseline": {"value": round(value, 4), "unit": "MLUPS",
                            "cores": oracle.num_threads(), "kind": "oracle", "sample": sample},
           "e2e": {"value": round(value, 4), "unit": "MLUPS", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return out


def parse_args(argv=None):
    p = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=None)
    p.add_argument("--warmup", type=int, default=None)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", default=MAIN["name"],
                   help="hit<N>_<f64|f32|f16>_<pull|aa> or kida<N>_..., default %s" % MAIN["name"])
    p.add_argument("--no-variants", action="store_true")
    p.add_argument("--variants", default=None,
                   help="comma-separated workloads to run as variants instead of the default "
                        "list (names as for --workload, or batch<K>_<storage>_<scheme>)")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--scaling", choices=["weak", "strong"], default="weak",
                   help="weak: one box per rank (replicas); strong: one box split along z")
    a = p.parse_args(argv)
    if a.impl == "reference":
        a.steps = 3 if a.steps is None else a.steps
        a.warmup = 1 if a.warmup is None else a.warmup
    else:
        a.steps = 2000 if a.steps is None else a.steps
        a.warmup = 10 if a.warmup is None else a.warmup
        if a.warmup < 3:
            a.warmup = 3
    return a


def main(argv=None):
    args = parse_args(argv)
    rank, world, local = dist_init(args.gpus)
    try:
        if args.impl == "reference":
            main_reference(args, rank, world)
        elif args.scaling == "strong":
            main_strong(args, rank, world, local)
        else:
            main_ours(args, rank, world, local)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
