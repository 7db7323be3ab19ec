"""Python binding of the C ABI in ``include/kbc_lb.h`` (argument marshalling only).

Every function here has the name of the C entry point it calls; all lattice-Boltzmann work runs
in ``libkbc.so`` (CUDA, sm_103a). PyTorch is used only for device memory and streams in the
``Lattice`` / ``Batch`` convenience classes. There is no CPU fallback: if the library is missing
or cannot be loaded, ``load()`` raises.
"""
from __future__ import annotations

import ctypes
import math
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libkbc.so")

LB_OK, LB_ERR_INVALID_ARG, LB_ERR_OOM, LB_ERR_CUDA, LB_ERR_NONFINITE, LB_ERR_TIMEOUT, \
    LB_ERR_UNSUPPORTED = range(7)
LB_S_D, LB_S_DT, LB_S_DQ, LB_S_DTQ, LB_S_CD, LB_S_CDT, LB_S_CDQ, LB_S_CDTQ = range(8)
LB_GAMMA_ESTIMATE, LB_GAMMA_LBGK, LB_GAMMA_RLB, LB_GAMMA_EXACT = range(4)
LB_F64, LB_F32, LB_F16 = range(3)
LB_PULL, LB_AA = range(2)
LB_EQ_PRODUCT, LB_EQ_POLY2 = range(2)
LB_KERNEL_AUTO, LB_KERNEL_DIRECT, LB_KERNEL_STAGED, LB_KERNEL_PERSISTENT, \
    LB_KERNEL_PACKED, LB_KERNEL_ROWS, LB_KERNEL_ADJ = range(7)
KERNEL = {"auto": LB_KERNEL_AUTO, "direct": LB_KERNEL_DIRECT, "staged": LB_KERNEL_STAGED,
          "persistent": LB_KERNEL_PERSISTENT, "packed": LB_KERNEL_PACKED,
          "rows": LB_KERNEL_ROWS, "adj": LB_KERNEL_ADJ}

STORAGE = {"f64": LB_F64, "f32": LB_F32, "f16": LB_F16}
SCHEME = {"pull": LB_PULL, "aa": LB_AA}
VARIANT = {"d": LB_S_D, "d+t": LB_S_DT, "d+q": LB_S_DQ, "d+t+q": LB_S_DTQ,
           "cd": LB_S_CD, "cd+ct": LB_S_CDT, "cd+cq": LB_S_CDQ, "cd+ct+cq": LB_S_CDTQ}
GAMMA = {"estimate": LB_GAMMA_ESTIMATE, "lbgk": LB_GAMMA_LBGK, "rlb": LB_GAMMA_RLB,
         "exact": LB_GAMMA_EXACT}
EQUILIBRIUM = {"product": LB_EQ_PRODUCT, "poly2": LB_EQ_POLY2}
BYTES_PER_VALUE = {LB_F64: 8, LB_F32: 4, LB_F16: 2}


class lb_config(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("nu", ctypes.c_double), ("variant", ctypes.c_int32),
                ("gamma_mode", ctypes.c_int32), ("storage", ctypes.c_int32),
                ("scheme", ctypes.c_int32), ("equilibrium", ctypes.c_int32)]


class lb_diag(ctypes.Structure):
    _fields_ = [("step", ctypes.c_int64), ("nodes", ctypes.c_int64), ("mass", ctypes.c_double),
                ("momentum", ctypes.c_double * 3), ("kinetic_energy", ctypes.c_double),
                ("enstrophy", ctypes.c_double), ("dissipation", ctypes.c_double),
                ("gamma_mean", ctypes.c_double), ("gamma_std", ctypes.c_double),
                ("nonfinite_count", ctypes.c_int64), ("den_guard_count", ctypes.c_int64),
                ("grad_order", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("dudx2", ctypes.c_double), ("skewness", ctypes.c_double * 4)]

    def as_dict(self):
        return {"step": self.step, "nodes": self.nodes, "mass": self.mass,
                "momentum": list(self.momentum), "kinetic_energy": self.kinetic_energy,
                "enstrophy": self.enstrophy, "dissipation": self.dissipation,
                "gamma_mean": self.gamma_mean, "gamma_std": self.gamma_std,
                "nonfinite_count": self.nonfinite_count,
                "den_guard_count": self.den_guard_count, "grad_order": self.grad_order,
                "dudx2": self.dudx2, "skewness": list(self.skewness)}


class lb_gap(ctypes.Structure):
    _fields_ = [("step", ctypes.c_int64), ("nodes", ctypes.c_int64),
                ("mean_abs", ctypes.c_double), ("max_abs", ctypes.c_double),
                ("mean_estimate", ctypes.c_double), ("mean_exact", ctypes.c_double),
                ("unconverged", ctypes.c_int64), ("skipped", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None
_lock = threading.Lock()

# exported C entry points (kept in step with include/kbc_lb.h; a test checks both ways)
SYMBOLS = ["lb_required_bytes", "lb_create", "lb_destroy", "lb_last_error", "lb_init_field",
           "lb_step", "lb_moments", "lb_diagnostics", "lb_get_populations",
           "lb_set_populations", "lb_time", "lb_beta", "lb_set_time", "lb_set_block",
           "lb_set_kernel", "lb_set_prefetch", "lb_set_wait_budget",
           "lb_batch_required_bytes", "lb_batch_create", "lb_batch_destroy",
           "lb_batch_last_error", "lb_batch_box", "lb_batch_step", "lb_batch_diagnostics",
           "lb_batch_autotune", "lb_batch_set_tile", "lb_batch_set_kernel",
           "lb_diagnostics_noalloc", "lb_stabilizer_gap", "lb_presolve", "lb_set_diag_order",
           "lb_spectrum_work_bytes", "lb_spectrum", "lb_get_gamma", "lb_slab_required_bytes",
           "lb_slab_create", "lb_slab_faces", "lb_slab_step_faces", "lb_slab_step_interior",
           "lb_slab_unpack"]


class LBError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("lb status %d: %s" % (status, msg))
        self.status = status


def load(path: str = LIB_PATH):
    """Load libkbc.so (raises if it is missing: build it with paper_1507_02518_gb300.build)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError("libkbc.so not found at %s: run "
                               "`python -m paper_1507_02518_gb300.build` (needs nvcc)" % path)
        L = ctypes.CDLL(path)
        vp, i32, i64, d = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        cfgp = ctypes.POINTER(lb_config)
        L.lb_required_bytes.restype = ctypes.c_size_t
        L.lb_required_bytes.argtypes = [cfgp]
        L.lb_create.restype = i32
        L.lb_create.argtypes = [cfgp, vp, ctypes.c_size_t, vp, ctypes.POINTER(vp)]
        L.lb_destroy.restype = i32
        L.lb_destroy.argtypes = [vp]
        L.lb_last_error.restype = ctypes.c_char_p
        L.lb_last_error.argtypes = [vp]
        L.lb_init_field.restype = i32
        L.lb_init_field.argtypes = [vp, vp, vp, ctypes.c_int]
        L.lb_step.restype = i32
        L.lb_step.argtypes = [vp, i64]
        L.lb_moments.restype = i32
        L.lb_moments.argtypes = [vp, vp, vp, ctypes.c_int]
        L.lb_diagnostics.restype = i32
        L.lb_diagnostics.argtypes = [vp, ctypes.POINTER(lb_diag)]
        L.lb_get_populations.restype = i32
        L.lb_get_populations.argtypes = [vp, vp, ctypes.c_int]
        L.lb_get_gamma.restype = i32
        L.lb_get_gamma.argtypes = [vp, vp, ctypes.c_int]
        L.lb_slab_required_bytes.restype = ctypes.c_size_t
        L.lb_slab_required_bytes.argtypes = [cfgp, i32]
        L.lb_slab_create.restype = i32
        L.lb_slab_create.argtypes = [cfgp, i32, i32, vp, ctypes.c_size_t, vp, ctypes.POINTER(vp)]
        L.lb_slab_faces.restype = i32
        L.lb_slab_faces.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp),
                                    ctypes.POINTER(vp), ctypes.POINTER(vp),
                                    ctypes.POINTER(ctypes.c_size_t)]
        L.lb_slab_step_faces.restype = i32
        L.lb_slab_step_faces.argtypes = [vp, i32]
        L.lb_slab_step_interior.restype = i32
        L.lb_slab_step_interior.argtypes = [vp]
        L.lb_slab_unpack.restype = i32
        L.lb_slab_unpack.argtypes = [vp]
        L.lb_set_populations.restype = i32
        L.lb_set_populations.argtypes = [vp, vp, ctypes.c_int]
        L.lb_time.restype = i64
        L.lb_time.argtypes = [vp]
        L.lb_beta.restype = d
        L.lb_beta.argtypes = [vp]
        L.lb_set_time.restype = i32
        L.lb_set_time.argtypes = [vp, i64]
        L.lb_set_block.restype = i32
        L.lb_set_block.argtypes = [vp, i32, i32]
        L.lb_set_kernel.restype = i32
        L.lb_set_kernel.argtypes = [vp, i32]
        L.lb_set_prefetch.restype = i32
        L.lb_set_prefetch.argtypes = [vp, i32]
        L.lb_set_wait_budget.restype = i32
        L.lb_set_wait_budget.argtypes = [vp, ctypes.c_uint64, i32]
        L.lb_batch_required_bytes.restype = ctypes.c_size_t
        L.lb_batch_required_bytes.argtypes = [cfgp, i32]
        L.lb_batch_create.restype = i32
        L.lb_batch_create.argtypes = [cfgp, i32, vp, ctypes.c_size_t, vp, ctypes.POINTER(vp)]
        L.lb_batch_destroy.restype = i32
        L.lb_batch_destroy.argtypes = [vp]
        L.lb_batch_last_error.restype = ctypes.c_char_p
        L.lb_batch_last_error.argtypes = [vp]
        L.lb_batch_box.restype = vp
        L.lb_batch_box.argtypes = [vp, i32]
        L.lb_batch_step.restype = i32
        L.lb_batch_step.argtypes = [vp, i64]
        L.lb_batch_diagnostics.restype = i32
        L.lb_batch_diagnostics.argtypes = [vp, ctypes.POINTER(lb_diag)]
        L.lb_batch_autotune.restype = i32
        L.lb_batch_autotune.argtypes = [vp, i32, ctypes.POINTER(i32), ctypes.POINTER(i32),
                                        ctypes.POINTER(d)]
        L.lb_batch_set_tile.restype = i32
        L.lb_batch_set_tile.argtypes = [vp, i32, i32]
        L.lb_batch_set_kernel.restype = i32
        L.lb_batch_set_kernel.argtypes = [vp, i32]
        L.lb_diagnostics_noalloc.restype = i32
        L.lb_diagnostics_noalloc.argtypes = [i32, i32, i32, d, vp, vp, ctypes.POINTER(lb_diag)]
        L.lb_spectrum_work_bytes.restype = ctypes.c_size_t
        L.lb_spectrum_work_bytes.argtypes = [vp, i32]
        L.lb_spectrum.restype = i32
        L.lb_spectrum.argtypes = [vp, vp, ctypes.c_size_t, i32, vp]
        L.lb_set_diag_order.restype = i32
        L.lb_set_diag_order.argtypes = [vp, i32]
        L.lb_presolve.restype = i32
        L.lb_presolve.argtypes = [vp, vp, ctypes.c_int, d, i64, d, i32, ctypes.POINTER(i64),
                                  ctypes.POINTER(d)]
        L.lb_stabilizer_gap.restype = i32
        L.lb_stabilizer_gap.argtypes = [vp, ctypes.POINTER(lb_gap)]
        _lib = L
        return L


def _check(status, ctx=None, batch=False):
    if status != LB_OK:
        L = load()
        msg = (L.lb_batch_last_error(ctx) if batch else L.lb_last_error(ctx)) or b""
        raise LBError(status, msg.decode(errors="replace"))


def make_config(nx, ny=None, nz=None, nu=1e-3, variant="d+t+q", gamma="estimate", storage="f32",
                scheme="pull", equilibrium="product") -> lb_config:
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    return lb_config(int(nx), int(ny), int(nz), float(nu),
                     VARIANT[variant] if isinstance(variant, str) else int(variant),
                     GAMMA[gamma] if isinstance(gamma, str) else int(gamma),
                     STORAGE[storage] if isinstance(storage, str) else int(storage),
                     SCHEME[scheme] if isinstance(scheme, str) else int(scheme),
                     EQUILIBRIUM[equilibrium] if isinstance(equilibrium, str) else int(equilibrium))


# ---------------------------------------------------------------- 1:1 wrappers of the C ABI

def lb_required_bytes(cfg: lb_config) -> int:
    return int(load().lb_required_bytes(ctypes.byref(cfg)))


def lb_create(cfg: lb_config, dev_buf: int, nbytes: int, stream: int = 0):
    out = ctypes.c_void_p()
    _check(load().lb_create(ctypes.byref(cfg), ctypes.c_void_p(dev_buf), nbytes,
                            ctypes.c_void_p(stream), ctypes.byref(out)))
    return out.value


def lb_destroy(ctx):
    _check(load().lb_destroy(ctx), ctx)


def lb_last_error(ctx=None) -> str:
    return (load().lb_last_error(ctx) or b"").decode(errors="replace")


def lb_init_field(ctx, rho_ptr: int, u_ptr: int, on_device: bool):
    _check(load().lb_init_field(ctx, ctypes.c_void_p(rho_ptr), ctypes.c_void_p(u_ptr),
                                int(on_device)), ctx)


def lb_spectrum_work_bytes(ctx, nbins: int) -> int:
    return int(load().lb_spectrum_work_bytes(ctx, int(nbins)))


def lb_spectrum(ctx, work_ptr: int, work_bytes: int, nbins: int) -> np.ndarray:
    E = np.zeros(int(nbins))
    _check(load().lb_spectrum(ctx, ctypes.c_void_p(work_ptr), int(work_bytes), int(nbins),
                              E.ctypes.data), ctx)
    return E


def lb_set_diag_order(ctx, order: int):
    _check(load().lb_set_diag_order(ctx, int(order)), ctx)


def lb_presolve(ctx, u0_ptr: int, on_device: bool, nu_pre: float, max_iters: int, tol: float,
                from_current: bool = False):
    it, res = ctypes.c_int64(), ctypes.c_double()
    _check(load().lb_presolve(ctx, ctypes.c_void_p(u0_ptr), int(on_device), float(nu_pre),
                              int(max_iters), float(tol), int(bool(from_current)),
                              ctypes.byref(it), ctypes.byref(res)), ctx)
    return it.value, res.value


def lb_step(ctx, n: int):
    _check(load().lb_step(ctx, int(n)), ctx)


def lb_moments(ctx, rho_ptr: int, u_ptr: int, on_device: bool):
    _check(load().lb_moments(ctx, ctypes.c_void_p(rho_ptr), ctypes.c_void_p(u_ptr),
                             int(on_device)), ctx)


def lb_diagnostics(ctx, raise_nonfinite: bool = True) -> lb_diag:
    d = lb_diag()
    s = load().lb_diagnostics(ctx, ctypes.byref(d))
    if s == LB_ERR_NONFINITE and not raise_nonfinite:
        return d
    _check(s, ctx)
    return d


def lb_diagnostics_noalloc(nx: int, ny: int, nz: int, nu: float, f_dev_ptr: int, stream: int = 0,
                           raise_nonfinite: bool = True) -> lb_diag:
    """Diagnostics of a canonical FP64 population field already on the device, computed with
    the library's static work space (no allocation; at most 65,536 nodes)."""
    d = lb_diag()
    s = load().lb_diagnostics_noalloc(int(nx), int(ny), int(nz), float(nu),
                                      ctypes.c_void_p(f_dev_ptr), ctypes.c_void_p(stream),
                                      ctypes.byref(d))
    if s == LB_ERR_NONFINITE and not raise_nonfinite:
        return d
    if s != LB_OK:
        raise LBError(s, lb_last_error(None))
    return d


def lb_stabilizer_gap(ctx) -> lb_gap:
    g = lb_gap()
    _check(load().lb_stabilizer_gap(ctx, ctypes.byref(g)), ctx)
    return g


def lb_get_populations(ctx, f_ptr: int, on_device: bool):
    _check(load().lb_get_populations(ctx, ctypes.c_void_p(f_ptr), int(on_device)), ctx)


def lb_get_gamma(ctx, gamma_ptr: int, on_device: bool):
    _check(load().lb_get_gamma(ctx, ctypes.c_void_p(gamma_ptr), int(on_device)), ctx)


def lb_slab_required_bytes(cfg: lb_config, nz_local: int) -> int:
    return int(load().lb_slab_required_bytes(ctypes.byref(cfg), int(nz_local)))


def lb_slab_create(cfg: lb_config, z0: int, nz_local: int, dev_buf: int, nbytes: int,
                   stream: int = 0):
    out = ctypes.c_void_p()
    _check(load().lb_slab_create(ctypes.byref(cfg), int(z0), int(nz_local),
                                 ctypes.c_void_p(dev_buf), nbytes, ctypes.c_void_p(stream),
                                 ctypes.byref(out)))
    return out


def lb_slab_faces(ctx):
    """(send_up, send_down, recv_below, recv_above) device addresses and the face size."""
    p = [ctypes.c_void_p() for _ in range(4)]
    n = ctypes.c_size_t()
    _check(load().lb_slab_faces(ctx, *[ctypes.byref(x) for x in p], ctypes.byref(n)), ctx)
    return [x.value for x in p], n.value


def lb_slab_step_faces(ctx, record: bool = False):
    _check(load().lb_slab_step_faces(ctx, int(bool(record))), ctx)


def lb_slab_step_interior(ctx):
    _check(load().lb_slab_step_interior(ctx), ctx)


def lb_slab_unpack(ctx):
    _check(load().lb_slab_unpack(ctx), ctx)


def lb_set_populations(ctx, f_ptr: int, on_device: bool):
    _check(load().lb_set_populations(ctx, ctypes.c_void_p(f_ptr), int(on_device)), ctx)


def lb_time(ctx) -> int:
    return int(load().lb_time(ctx))


def lb_beta(ctx) -> float:
    return float(load().lb_beta(ctx))


def lb_set_time(ctx, t: int):
    _check(load().lb_set_time(ctx, int(t)), ctx)


def lb_set_block(ctx, bx: int, by: int):
    _check(load().lb_set_block(ctx, int(bx), int(by)), ctx)


def lb_set_kernel(ctx, kind):
    _check(load().lb_set_kernel(ctx, KERNEL[kind] if isinstance(kind, str) else int(kind)), ctx)


def lb_set_prefetch(ctx, items_ahead: int):
    _check(load().lb_set_prefetch(ctx, int(items_ahead)), ctx)


def lb_set_wait_budget(ctx, cycles: int, stall_copies: bool = False):
    _check(load().lb_set_wait_budget(ctx, int(cycles), int(bool(stall_copies))), ctx)


def lb_batch_required_bytes(cfgs) -> int:
    arr = (lb_config * len(cfgs))(*cfgs)
    return int(load().lb_batch_required_bytes(arr, len(cfgs)))


def lb_batch_create(cfgs, dev_buf: int, nbytes: int, stream: int = 0):
    arr = (lb_config * len(cfgs))(*cfgs)
    out = ctypes.c_void_p()
    s = load().lb_batch_create(arr, len(cfgs), ctypes.c_void_p(dev_buf), nbytes,
                               ctypes.c_void_p(stream), ctypes.byref(out))
    if s != LB_OK:
        raise LBError(s, lb_last_error(None))
    return out.value


def lb_batch_destroy(b):
    _check(load().lb_batch_destroy(b), b, batch=True)


def lb_batch_box(b, box: int):
    v = load().lb_batch_box(b, int(box))
    if not v:
        raise LBError(LB_ERR_INVALID_ARG, "no box %d" % box)
    return v


def lb_batch_step(b, n: int):
    _check(load().lb_batch_step(b, int(n)), b, batch=True)


def lb_batch_diagnostics(b, nbox: int, raise_nonfinite: bool = True):
    arr = (lb_diag * nbox)()
    s = load().lb_batch_diagnostics(b, arr)
    if not (s == LB_ERR_NONFINITE and not raise_nonfinite):
        _check(s, b, batch=True)
    return list(arr)


def lb_batch_autotune(b, trial_steps: int):
    th, tl, ms = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_double()
    _check(load().lb_batch_autotune(b, int(trial_steps), ctypes.byref(th), ctypes.byref(tl),
                                    ctypes.byref(ms)), b, batch=True)
    return th.value, tl.value, ms.value


def lb_batch_set_kernel(b, kind):
    _check(load().lb_batch_set_kernel(b, KERNEL[kind] if isinstance(kind, str) else int(kind)),
           b, batch=True)


def lb_batch_set_tile(b, threads: int, tile: int):
    _check(load().lb_batch_set_tile(b, int(threads), int(tile)), b, batch=True)


# ---------------------------------------------------------------- convenience classes

def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("a CUDA device is required")
    return torch


def _device_buffer(torch, nbytes, device, stream):
    """The caller-owned device buffer of a context: a torch uint8 tensor. When the library's
    stream is not the one torch allocated on, the tensor is recorded on it, so that the caching
    allocator does not hand the memory out again while kernels enqueued there may still run."""
    buf = torch.empty(nbytes, dtype=torch.uint8, device=device)
    if stream != torch.cuda.current_stream(device):
        buf.record_stream(stream)
    return buf


class Lattice:
    """One periodic box. Device memory is a torch uint8 tensor owned by this object."""

    def __init__(self, nx, ny=None, nz=None, nu=1e-3, variant="d+t+q", gamma="estimate",
                 storage="f32", scheme="pull", stream=None, device=None, equilibrium="product"):
        torch = _torch()
        self.cfg = make_config(nx, ny, nz, nu, variant, gamma, storage, scheme, equilibrium)
        self.shape = (self.cfg.nz, self.cfg.ny, self.cfg.nx)
        self.P = self.cfg.nx * self.cfg.ny * self.cfg.nz
        self.nbytes = lb_required_bytes(self.cfg)
        if self.nbytes == 0:
            raise LBError(LB_ERR_INVALID_ARG, "invalid configuration")
        self.device = torch.device(device or "cuda")
        self.stream = stream or torch.cuda.current_stream(self.device)
        self.buf = _device_buffer(torch, self.nbytes, self.device, self.stream)
        self.ctx = lb_create(self.cfg, self.buf.data_ptr(), self.nbytes, self.stream.cuda_stream)

    def close(self):
        if getattr(self, "ctx", None):
            lb_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def t(self) -> int:
        return lb_time(self.ctx)

    @property
    def nu(self) -> float:
        return self.cfg.nu

    @property
    def beta(self) -> float:
        return lb_beta(self.ctx)

    def init_field(self, rho, u):
        """rho [nz,ny,nx] (or None), u [3,nz,ny,nx]: numpy (host copy path) or CUDA tensors."""
        torch = _torch()
        if isinstance(u, torch.Tensor) and u.is_cuda:
            u = u.to(torch.float64).contiguous()
            r = None if rho is None else rho.to(torch.float64).contiguous()
            lb_init_field(self.ctx, 0 if r is None else r.data_ptr(), u.data_ptr(), True)
        else:
            u = np.ascontiguousarray(u, dtype=np.float64)
            r = None if rho is None else np.ascontiguousarray(rho, dtype=np.float64)
            lb_init_field(self.ctx, 0 if r is None else r.ctypes.data, u.ctypes.data, False)

    def presolve(self, u0, nu_pre=1.0 / 6.0, max_iters=20000, tol=1e-9, from_current=False):
        """Consistent initial state for the velocity u0 ([3,nz,ny,nx], numpy or CUDA tensor):
        see lb_presolve. Returns (iterations, last change of rho)."""
        torch = _torch()
        if isinstance(u0, torch.Tensor) and u0.is_cuda:
            u0 = u0.to(torch.float64).contiguous()
            return lb_presolve(self.ctx, u0.data_ptr(), True, nu_pre, max_iters, tol,
                               from_current)
        u0 = np.ascontiguousarray(u0, dtype=np.float64)
        return lb_presolve(self.ctx, u0.ctypes.data, False, nu_pre, max_iters, tol, from_current)

    def step(self, n=1):
        lb_step(self.ctx, n)

    def run(self, steps, every=50, log=None):
        """Advance `steps` steps with lb_diagnostics every `every` steps (and at the end).
        Returns the list of diagnostics dicts, each with the MLUPS of its interval (wall clock
        between two synchronising diagnostics); with `log`, also appends them as JSON lines."""
        import json
        import time
        out = []
        fh = open(log, "a") if log else None
        try:
            done = 0
            t0 = time.perf_counter()
            while done < steps:
                c = min(every, steps - done)
                lb_step(self.ctx, c)
                done += c
                d = lb_diagnostics(self.ctx, raise_nonfinite=False).as_dict()
                t1 = time.perf_counter()
                d["mlups"] = self.P * c / max(t1 - t0, 1e-12) / 1e6
                t0 = t1
                out.append(d)
                if fh:
                    fh.write(json.dumps(d) + "\n")
                    fh.flush()
        finally:
            if fh:
                fh.close()
        return out

    def moments(self):
        rho = np.empty(self.shape)
        u = np.empty((3,) + self.shape)
        lb_moments(self.ctx, rho.ctypes.data, u.ctypes.data, False)
        return rho, u

    def diagnostics(self, raise_nonfinite=True) -> dict:
        return lb_diagnostics(self.ctx, raise_nonfinite).as_dict()

    def spectrum(self, nbins=None):
        """Shell-summed kinetic-energy spectrum E[m] (kappa = 2 pi m / N) of the current state;
        nbins defaults to every shell of the cube. Work space comes from torch's allocator."""
        torch = _torch()
        if nbins is None:
            nbins = int(math.sqrt(3.0) * self.shape[0] / 2.0) + 2
        need = lb_spectrum_work_bytes(self.ctx, nbins)
        if need == 0:
            cubic = self.shape[0] == self.shape[1] == self.shape[2]
            raise LBError(LB_ERR_INVALID_ARG if cubic else LB_ERR_UNSUPPORTED,
                          lb_last_error(self.ctx))
        with torch.cuda.stream(self.stream):
            work = torch.empty(need + 256, dtype=torch.uint8, device="cuda")
            ptr = (work.data_ptr() + 255) // 256 * 256
            return lb_spectrum(self.ctx, ptr, need, nbins)

    def set_diag_order(self, order):
        """Central-difference order (2 or 8) of the velocity gradients in diagnostics()."""
        lb_set_diag_order(self.ctx, order)

    def stabilizer_gap(self) -> dict:
        """<|gamma_est - gamma*|>, max, means and solver counts on the current state."""
        return lb_stabilizer_gap(self.ctx).as_dict()

    def get_populations(self) -> np.ndarray:
        f = np.empty((27,) + self.shape)
        lb_get_populations(self.ctx, f.ctypes.data, False)
        return f

    def gamma(self) -> np.ndarray:
        """The stabilizer of every node in the last collision (FP32, [nz, ny, nx])."""
        g = np.empty(self.shape, dtype=np.float32)
        lb_get_gamma(self.ctx, g.ctypes.data, False)
        return g

    def set_populations(self, f):
        f = np.ascontiguousarray(f, dtype=np.float64)
        assert f.shape == (27,) + self.shape
        lb_set_populations(self.ctx, f.ctypes.data, False)

    def set_block(self, bx, by):
        lb_set_block(self.ctx, bx, by)

    def set_kernel(self, kind):
        lb_set_kernel(self.ctx, kind)

    def save_checkpoint(self, path):
        """Raw little-endian FP64 canonical populations with a one-line JSON header."""
        import json
        f = self.get_populations()
        hdr = {"nx": self.cfg.nx, "ny": self.cfg.ny, "nz": self.cfg.nz, "nu": self.cfg.nu,
               "variant": self.cfg.variant, "gamma_mode": self.cfg.gamma_mode,
               "storage": self.cfg.storage, "scheme": self.cfg.scheme, "t": self.t}
        with open(path, "wb") as fh:
            fh.write((json.dumps(hdr) + "\n").encode())
            fh.write(f.astype("<f8").tobytes())

    def load_checkpoint(self, path):
        import json
        with open(path, "rb") as fh:
            hdr = json.loads(fh.readline().decode())
            data = np.frombuffer(fh.read(), dtype="<f8")
        if (hdr["nx"], hdr["ny"], hdr["nz"]) != (self.cfg.nx, self.cfg.ny, self.cfg.nz):
            raise LBError(LB_ERR_INVALID_ARG, "checkpoint box does not match")
        if data.size != 27 * self.P:
            raise LBError(LB_ERR_INVALID_ARG, "checkpoint is truncated or corrupt")
        lb_set_time(self.ctx, hdr["t"])
        self.set_populations(data.reshape((27,) + self.shape))


class Batch:
    """An ensemble of boxes stepped together (one work-list kernel per step, CUDA graph)."""

    def __init__(self, boxes, variant="d+t+q", gamma="estimate", storage="f32", scheme="pull",
                 stream=None, device=None):
        torch = _torch()
        self.cfgs = [make_config(b["n"], b.get("ny"), b.get("nz"), b["nu"], variant, gamma,
                                 storage, scheme) for b in boxes]
        self.nbox = len(self.cfgs)
        self.nbytes = lb_batch_required_bytes(self.cfgs)
        if self.nbytes == 0:
            raise LBError(LB_ERR_INVALID_ARG, "invalid batch configuration")
        self.device = torch.device(device or "cuda")
        self.stream = stream or torch.cuda.current_stream(self.device)
        self.buf = _device_buffer(torch, self.nbytes, self.device, self.stream)
        self.handle = lb_batch_create(self.cfgs, self.buf.data_ptr(), self.nbytes,
                                      self.stream.cuda_stream)
        self.nodes = sum(c.nx * c.ny * c.nz for c in self.cfgs)

    def close(self):
        if getattr(self, "handle", None):
            lb_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def box(self, k):
        """A ctx handle aliasing box k (use with the lb_* functions)."""
        return lb_batch_box(self.handle, k)

    def step(self, n=1):
        lb_batch_step(self.handle, n)

    def diagnostics(self, raise_nonfinite=True):
        return [d.as_dict() for d in lb_batch_diagnostics(self.handle, self.nbox, raise_nonfinite)]

    def autotune(self, trial_steps=3):
        return lb_batch_autotune(self.handle, trial_steps)

    def set_tile(self, threads, tile):
        lb_batch_set_tile(self.handle, threads, tile)

    def set_kernel(self, kind):
        lb_batch_set_kernel(self.handle, kind)
