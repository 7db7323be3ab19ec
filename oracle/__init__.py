"""FP64 CPU oracle of the D3Q27 KBC step (arXiv:1507.02518).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()`` and by the
CPU-baseline leg of ``bench.py``. The product package never imports it, and the two share no
code. The arithmetic lives in ``kbc_oracle.c`` (plain C, FP64, compiled with
``-O2 -ffp-contract=off``); this module only builds it and marshals numpy arrays.

Field layout: ``f[27, nz, ny, nx]`` (plane i contiguous, x fastest), velocity index
``i = (vx+1) + 3(vy+1) + 9(vz+1)``; macroscopic ``rho[nz, ny, nx]``, ``u[3, nz, ny, nx]``.

Parity pins: every function here is pinned by ``tests/test_oracle_*.py`` against properties the
paper and the mathematics fix (conservation, fixed point, LBGK/RLB limits, the moment-basis
inverse, cube symmetry, entropy maximum, analytic decay rates, closed-form diagnostics). The
exact-stabilizer root (``gamma_exact``) is pinned by a bracketing root of the entropy
derivative and its limit toward eq:result21; the density pre-solve (``presolve``) by mass
conservation, its fixed points and the closed-form pressure of the Taylor-Green vortex.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kbc_oracle.c")
_HDR = os.path.join(_HERE, "kbc_oracle.h")
_LIB = os.path.join(_HERE, "liborc.so")
_lock = threading.Lock()
_lib = None

S_D, S_DT, S_DQ, S_DTQ = 0, 1, 2, 3
S_CD, S_CDT, S_CDQ, S_CDTQ = 4, 5, 6, 7      # the same groups in the central-moment basis
GAMMA_ESTIMATE, GAMMA_LBGK, GAMMA_RLB, GAMMA_EXACT = 0, 1, 2, 3
EQ_POLY2 = 16          # OR'ed into a variant: the polynomial equilibrium eq:polynomial2
DEN_GUARD = 1e-300


def build(force: bool = False) -> str:
    """Compile ``liborc.so`` with gcc (OpenMP if available). Returns the library path."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= newest:
        return _LIB
    base = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11", "-fPIC", "-shared"]
    tmp = _LIB + ".tmp%d" % os.getpid()
    try:
        subprocess.run(base + ["-fopenmp", _SRC, "-o", tmp, "-lm"], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base + [_SRC, "-o", tmp, "-lm"], check=True)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            d, i32, i64, vp = ctypes.c_double, ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p
            L.orc_beta.restype = d
            L.orc_beta.argtypes = [d]
            L.orc_lattice.argtypes = [vp, vp]
            L.orc_equilibrium.argtypes = [d, vp, vp]
            L.orc_equilibrium_poly2.argtypes = [d, vp, vp]
            L.orc_moments.argtypes = [vp, vp, vp]
            L.orc_table1.argtypes = [vp, d, vp, vp, vp, vp]
            L.orc_moment_rep.argtypes = [vp, d, vp]
            L.orc_central_moments.argtypes = [vp, vp, vp, vp]
            L.orc_central_parts.argtypes = [vp, d, vp, vp, vp, vp, vp, vp]
            L.orc_collide.restype = ctypes.c_int
            L.orc_collide.argtypes = [vp, d, ctypes.c_int, ctypes.c_int, vp, vp]
            L.orc_collide_mirror.argtypes = [vp, d, ctypes.c_int, d, vp]
            L.orc_deltas.argtypes = [vp, ctypes.c_int, vp, vp, vp]
            L.orc_gamma_exact.restype = d
            L.orc_gamma_exact.argtypes = [vp, vp, vp, d, d]
            L.orc_entropy.restype = d
            L.orc_entropy.argtypes = [vp]
            L.orc_stream.argtypes = [i32, i32, i32, vp, vp]
            L.orc_collide_field.restype = i64
            L.orc_collide_field.argtypes = [i32, i32, i32, vp, d, ctypes.c_int, ctypes.c_int, vp]
            L.orc_init_equilibrium.argtypes = [i32, i32, i32, vp, vp, vp]
            L.orc_macroscopic.argtypes = [i32, i32, i32, vp, vp, vp]
            L.orc_diagnostics.argtypes = [i32, i32, i32, vp, vp, d, ctypes.c_int, vp]
            L.orc_run.restype = i64
            L.orc_run.argtypes = [i32, i32, i32, vp, vp, i64, d, ctypes.c_int, ctypes.c_int,
                                       vp]
            L.orc_presolve.restype = i64
            L.orc_presolve.argtypes = [i32, i32, i32, vp, vp, vp, d, i64, d, vp]
            L.orc_num_threads.restype = ctypes.c_int
            _lib = L
    return _lib


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _null():
    return ctypes.c_void_p(0)


# ---------------------------------------------------------------- single node

def lattice():
    """(v[27,3] int, W[27]) in the order i = (vx+1) + 3(vy+1) + 9(vz+1)."""
    v = np.zeros((27, 3), dtype=np.int32)
    w = np.zeros(27)
    lib().orc_lattice(v.ctypes.data_as(ctypes.c_void_p), _p(w))
    return v.astype(np.int64), w


def beta(nu: float) -> float:
    return lib().orc_beta(nu)


def equilibrium(rho: float, u) -> np.ndarray:
    u = _f64(u)
    out = np.zeros(27)
    lib().orc_equilibrium(float(rho), _p(u), _p(out))
    return out


def equilibrium_poly2(rho: float, u) -> np.ndarray:
    """The second-order polynomial equilibrium eq:polynomial2."""
    u = _f64(u)
    out = np.zeros(27)
    lib().orc_equilibrium_poly2(float(rho), _p(u), _p(out))
    return out


def moments(f):
    """(rho, M[3,3,3]) with M[p,q,r] = sum f v^p v^q v^r / rho (eq:natmoments)."""
    f = _f64(f)
    rho = np.zeros(1)
    M = np.zeros(27)
    lib().orc_moments(_p(f), _p(rho), _p(M))
    return float(rho[0]), M.reshape(3, 3, 3)


def table1(M, rho):
    """(k, d, t, q) parts of Table 1 for unit-density moments M[3,3,3]."""
    M = _f64(M).reshape(27)
    k, d, t, q = (np.zeros(27) for _ in range(4))
    lib().orc_table1(_p(M), float(rho), _p(k), _p(d), _p(t), _p(q))
    return k, d, t, q


def moment_rep(M, rho):
    M = _f64(M).reshape(27)
    f = np.zeros(27)
    lib().orc_moment_rep(_p(M), float(rho), _p(f))
    return f


def central_moments(f):
    """(rho, u[3], Mc[3,3,3]) with Mc[p,q,r] = sum f (vx-ux)^p (vy-uy)^q (vz-uz)^r / rho."""
    f = _f64(f)
    rho, u, Mc = np.zeros(1), np.zeros(3), np.zeros(27)
    lib().orc_central_moments(_p(f), _p(rho), _p(u), _p(Mc))
    return float(rho[0]), u, Mc.reshape(3, 3, 3)


def central_parts(Mc, rho, u):
    """(k~, d~, t~, q~, h~) of the central-moment representation (appendix)."""
    Mc, u = _f64(Mc).reshape(27), _f64(u)
    parts = [np.zeros(27) for _ in range(5)]
    lib().orc_central_parts(_p(Mc), float(rho), _p(u), *[_p(x) for x in parts])
    return tuple(parts)


def collide(f, beta_, variant=S_DTQ, gamma_mode=GAMMA_ESTIMATE):
    """One KBC collision of a single node. Returns (f', gamma, guarded)."""
    f = _f64(f)
    out = np.zeros(27)
    g = np.zeros(1)
    guarded = lib().orc_collide(_p(f), float(beta_), int(variant), int(gamma_mode), _p(out),
                                _p(g))
    return out, float(g[0]), bool(guarded)


def collide_mirror(f, beta_, variant, gamma):
    f = _f64(f)
    out = np.zeros(27)
    lib().orc_collide_mirror(_p(f), float(beta_), int(variant), float(gamma), _p(out))
    return out


def deltas(f, variant=S_DTQ):
    """(f_eq, ds, dh) of Sec. KBC: the equilibrium, ds = s - s_eq and dh = f - f_eq - ds."""
    f = _f64(f)
    feq, ds, dh = np.zeros(27), np.zeros(27), np.zeros(27)
    lib().orc_deltas(_p(f), int(variant), _p(feq), _p(ds), _p(dh))
    return feq, ds, dh


def gamma_exact(feq, ds, dh, beta_, gamma0):
    feq, ds, dh = _f64(feq), _f64(ds), _f64(dh)
    return lib().orc_gamma_exact(_p(feq), _p(ds), _p(dh), float(beta_), float(gamma0))


def entropy(f) -> float:
    f = _f64(f)
    return lib().orc_entropy(_p(f))


# ---------------------------------------------------------------- fields

def _shape(f):
    assert f.ndim == 4 and f.shape[0] == 27
    nz, ny, nx = f.shape[1:]
    return int(nx), int(ny), int(nz)


def stream(f) -> np.ndarray:
    """Periodic propagation g_i(x) = f_i(x - v_i)."""
    f = _f64(f)
    nx, ny, nz = _shape(f)
    out = np.empty_like(f)
    lib().orc_stream(nx, ny, nz, _p(f), _p(out))
    return out


def collide_field(f, beta_, variant=S_DTQ, gamma_mode=GAMMA_ESTIMATE, want_gamma=False):
    """Collide every node. Returns (f', gamma_field or None, guarded_count)."""
    f = _f64(f).copy()
    nx, ny, nz = _shape(f)
    g = np.zeros((nz, ny, nx)) if want_gamma else None
    guarded = lib().orc_collide_field(nx, ny, nz, _p(f), float(beta_), int(variant),
                                      int(gamma_mode), _p(g) if want_gamma else _null())
    return f, g, int(guarded)


def init_equilibrium(rho, u) -> np.ndarray:
    rho, u = _f64(rho), _f64(u)
    nz, ny, nx = rho.shape
    f = np.empty((27, nz, ny, nx))
    lib().orc_init_equilibrium(nx, ny, nz, _p(rho), _p(u), _p(f))
    return f


def macroscopic(f):
    f = _f64(f)
    nx, ny, nz = _shape(f)
    rho = np.empty((nz, ny, nx))
    u = np.empty((3, nz, ny, nx))
    lib().orc_macroscopic(nx, ny, nz, _p(f), _p(rho), _p(u))
    return rho, u


def diagnostics(rho, u, nu, order=2):
    """dict(mass, momentum[3], kinetic_energy, enstrophy, dissipation, dudx2, skewness[S3..S6])
    from rho, u; derivatives by central differences of order 2 or 8."""
    assert order in (2, 8)
    rho, u = _f64(rho), _f64(u)
    nz, ny, nx = rho.shape
    out = np.zeros(13)
    lib().orc_diagnostics(nx, ny, nz, _p(rho), _p(u), float(nu), int(order), _p(out))
    return {"mass": out[0], "momentum": out[1:4].copy(), "kinetic_energy": out[4],
            "enstrophy": out[5], "dissipation": out[6], "dudx2": out[8],
            "skewness": out[9:13].copy()}


def spectrum(u, nbins):
    """Shell-summed kinetic-energy spectrum of u' = u - <u> on a periodic N^3 grid (Sec.
    "Numerical Simulations": E(kappa) with k = integral of E, D(kappa) = 2 nu kappa^2 E).

    E[m] = sum over integer wave vectors n != 0 with round(|n|) == m of 1/2 |u_hat(n)|^2,
    u_hat(n) = (1/P) sum_x u(x) exp(-2 pi i n.x / N), so that sum_m E[m] = k (Parseval).
    Shell m holds kappa = 2 pi m / N. A plain full complex FFT per component and a loop-free
    binning; numpy's FFT is the library step."""
    u = _f64(u)
    _, nz, ny, nx = u.shape
    assert nx == ny == nz, "cubic boxes only"
    n = nx
    P = n ** 3
    idx = np.fft.fftfreq(n, 1.0 / n)                 # 0, 1, ..., -1 (integers)
    NZ, NY, NX = np.meshgrid(idx, idx, idx, indexing="ij")
    shell = np.rint(np.sqrt(NX ** 2 + NY ** 2 + NZ ** 2)).astype(np.int64)
    e = np.zeros((nz, ny, nx))
    for a in range(3):
        uh = np.fft.fftn(u[a]) / P
        e += 0.5 * np.abs(uh) ** 2
    e[0, 0, 0] = 0.0                                  # the mean flow is not part of u'
    E = np.zeros(nbins)
    keep = shell < nbins
    np.add.at(E, shell[keep], e[keep])
    return E


def presolve(u0, beta_pre, max_iters, tol=-1.0, f=None):
    """Consistent initial state: the iteration of ``orc_presolve`` from f (default
    f_eq(1, u0)). Returns (f, iterations run, last change of rho)."""
    u0 = _f64(u0)
    _, nz, ny, nx = u0.shape
    if f is None:
        f = init_equilibrium(np.ones((nz, ny, nx)), u0)
    f = _f64(f).copy()
    fb = np.empty_like(f)
    res = ctypes.c_double()
    it = lib().orc_presolve(nx, ny, nz, _p(f), _p(fb), _p(u0), float(beta_pre), int(max_iters),
                            float(tol), ctypes.byref(res))
    if it < 0:
        raise MemoryError("orc_presolve could not allocate its work array")
    return f, int(it), res.value


def run(f, nsteps, beta_, variant=S_DTQ, gamma_mode=GAMMA_ESTIMATE, want_gamma=False):
    """nsteps of collide-then-stream from the pre-collision field f(t).

    Returns (f(t + nsteps), gamma of the last collision or None, guarded count).
    """
    fa = _f64(f).copy()
    nx, ny, nz = _shape(fa)
    fb = np.empty_like(fa)
    g = np.zeros((nz, ny, nx)) if want_gamma else None
    guarded = lib().orc_run(nx, ny, nz, _p(fa), _p(fb), int(nsteps), float(beta_),
                            int(variant), int(gamma_mode), _p(g) if want_gamma else _null())
    return fa, g, int(guarded)


def num_threads() -> int:
    return int(lib().orc_num_threads())
