"""CPU oracle for the RSWR wave-equation hot path (TEST INFRASTRUCTURE).

Python face of ``oracle/rswr_oracle.c``: a plain, slow, obviously correct
reference.  Only the test suite, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package; the CUDA library and its
binding never do, and this package never imports them.

Functions (each cites the paper passage it follows in the C source):

* ``coeffs``       grid/stencil coefficients from (xa, xb, a, nx, dt)
* ``leapfrog``     monolithic leapfrog, the "true solution" (Sec. 2.1)
* ``rswr_mask``    serial RSWR with select as an index mask (Sec. 2.2-2.6, Sec. 3)
* ``rswr_paper``   serial RSWR with the paper's adaptive select and
                   flux-exchange update (Sec. 2.3-2.6)
* ``adjoint``      discrete adjoint of the canonical leapfrog for a receiver
                   trace cotangent (gradient workload; not in the paper)
* ``misfit_grad``  loss ||trace - target||^2 and its gradients via ``adjoint``

Parity status: every function is pinned by ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rswr_oracle.c")
_HDR = os.path.join(_HERE, "leapfrog_body.h")
_LIB = os.path.join(_HERE, "_build", "librswr_oracle.so")

CANONICAL = 0
INCREMENT = 1


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, no fast-math)."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= newest:
        return _LIB
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    tmp = _LIB + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True, cwd=_HERE)
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _declare(_lib)
    return _lib


_i64 = ctypes.c_int64
_dbl = ctypes.c_double
_flt = ctypes.c_float
_vp = ctypes.c_void_p


def _declare(L):
    L.oracle_coeffs.argtypes = [_dbl, _dbl, _dbl, _i64, _dbl] + [_vp] * 7
    L.oracle_coeffs.restype = None
    L.oracle_set_threads.argtypes = [ctypes.c_int]
    L.oracle_set_threads.restype = None
    for suf, R in (("f64", _dbl), ("f32", _flt)):
        f = getattr(L, f"oracle_leapfrog_{suf}")
        f.argtypes = [ctypes.c_int, _i64, _i64, R, R, _vp, _vp, _vp, _vp, _vp, _vp,
                      _i64, _vp, _vp, _i64, _vp, R, _vp, _i64, _vp, _vp]
        f.restype = ctypes.c_int
        g = getattr(L, f"oracle_rswr_mask_{suf}")
        g.argtypes = [ctypes.c_int, _i64, _i64, R, R, _vp, _vp, _vp, _vp, _i64, _i64, _i64,
                      _vp, _vp, R, _vp, _i64, _vp, _vp]
        g.restype = ctypes.c_int
    L.oracle_rswr_paper.argtypes = [ctypes.c_int, _i64, _i64, _dbl, _dbl, _dbl, _dbl, _vp, _vp,
                                    _i64, _i64, _i64, _dbl, _vp, _vp, _vp, _vp]
    L.oracle_rswr_paper.restype = ctypes.c_int
    L.oracle_adjoint.argtypes = [_i64, _i64, _dbl, _dbl, _vp, _vp, _i64, _vp, _vp, _vp, _vp]
    L.oracle_adjoint.restype = ctypes.c_int


def _ptr(a):
    return None if a is None else a.ctypes.data


def _arr(a, dtype):
    if a is None:
        return None
    return np.ascontiguousarray(a, dtype=dtype)


@dataclass
class Coeffs:
    c: float
    c2: float
    k: float
    inv2dx: float
    c2f: np.float32
    kf: np.float32
    inv2dxf: np.float32
    dx: float


def set_threads(n: int) -> None:
    """Threads of the monolithic leapfrog's interior loop (default 1).  The
    result is the same bit for bit for any count (pinned by the tests)."""
    lib().oracle_set_threads(int(n))


def coeffs(xa: float, xb: float, a: float, nx: int, dt: float) -> Coeffs:
    out = [ctypes.c_double() for _ in range(4)] + [ctypes.c_float() for _ in range(3)]
    lib().oracle_coeffs(xa, xb, a, nx, dt, *[ctypes.addressof(o) for o in out])
    return Coeffs(out[0].value, out[1].value, out[2].value, out[3].value,
                  np.float32(out[4].value), np.float32(out[5].value), np.float32(out[6].value),
                  (xb - xa) / (nx - 1))


def _prec(prec: str):
    if prec == "f64":
        return np.float64, "f64"
    if prec == "f32":
        return np.float32, "f32"
    raise ValueError(prec)


def _cf(cf: Coeffs, prec: str):
    if prec == "f64":
        return cf.c2, cf.k, cf.inv2dx
    return float(cf.c2f), float(cf.kf), float(cf.inv2dxf)


def _sources(src_j, src, T, dt_):
    """(count, points, samples[count, T+1]) from one point (int, src 1-D) or a list."""
    if src is None:
        return 0, None, None
    src = np.asarray(src, dtype=dt_)
    if np.ndim(src_j) == 0:
        j = np.array([int(src_j)], dtype=np.int64)
        src = src.reshape(1, -1)
    else:
        j = np.ascontiguousarray(src_j, dtype=np.int64)
    src = np.ascontiguousarray(src.reshape(len(j), -1), dtype=dt_)
    assert src.shape == (len(j), T + 1)
    return len(j), j, src


def leapfrog(nx, T, a, dt, fA, fB, *, form=CANONICAL, prec="f64", q0=None, q1=None,
             rec_j=(), flux_j=(), xa=0.0, xb=1.0, nx_run=None, src_j=-1, src=None):
    """Monolithic leapfrog.  Returns dict(u=final q0, w=final q1, rec, flux, coeffs).

    The coefficients come from the grid (xa, xb, nx); ``nx_run`` < nx runs the
    same grid truncated to its first nx_run points (see ``causal_extent``).
    Interior point sources (the paper's pulse sources, Sec. 4; one of them is
    also the source term of the discrete adjoint): ``src_j`` one point or a list
    of K points, ``src`` T+1 samples or a (K, T+1) array; sample n is added at
    the point when level n is formed, in list order."""
    dt_, suf = _prec(prec)
    cf = coeffs(xa, xb, a, nx, dt)
    nx = nx if nx_run is None else int(nx_run)
    c2, k, inv2dx = _cf(cf, prec)
    fA = _arr(fA, dt_)
    fB = _arr(fB, dt_)
    assert fA.shape == (T + 1,) and fB.shape == (T + 1,)
    q0 = _arr(q0, dt_)
    q1 = _arr(q1, dt_)
    out0 = np.empty(nx, dt_)
    out1 = np.empty(nx, dt_)
    rj = np.ascontiguousarray(rec_j, dtype=np.int64)
    fj = np.ascontiguousarray(flux_j, dtype=np.int64)
    rec = np.empty((len(rj), T + 1), dt_)
    flux = np.empty((len(fj), T + 1), dt_)
    ns, sj, sv = _sources(src_j, src, T, dt_)
    rc = getattr(lib(), f"oracle_leapfrog_{suf}")(form, nx, T, c2, k, _ptr(fA), _ptr(fB), _ptr(q0), _ptr(q1),
                                                  _ptr(out0), _ptr(out1), len(rj), _ptr(rj), _ptr(rec),
                                                  len(fj), _ptr(fj), inv2dx, _ptr(flux), ns, _ptr(sj), _ptr(sv))
    if rc:
        raise RuntimeError(f"oracle_leapfrog failed ({rc})")
    return {"u": out0, "w": out1, "rec": rec, "flux": flux, "coeffs": cf}


def rswr_mask(nx, T, a, dt, fA, fB, N, ov, *, S=None, form=CANONICAL, prec="f64", q0=None, q1=None,
              xa=0.0, xb=1.0, traces=True, src_j=(), src=None):
    """Serial RSWR (index-mask select).  Returns dict(u, w, traces[(N-1),2,T+1]).
    Point sources as in ``leapfrog``, applied inside every window that holds them."""
    dt_, suf = _prec(prec)
    cf = coeffs(xa, xb, a, nx, dt)
    c2, k, inv2dx = _cf(cf, prec)
    if S is None:
        S = ov // 2
    fA = _arr(fA, dt_)
    fB = _arr(fB, dt_)
    q0 = _arr(q0, dt_)
    q1 = _arr(q1, dt_)
    out0 = np.empty(nx, dt_)
    out1 = np.empty(nx, dt_)
    tr = np.zeros((max(N - 1, 0), 2, T + 1), dt_) if traces else None
    ns, sj, sv = _sources(src_j, src, T, dt_)
    rc = getattr(lib(), f"oracle_rswr_mask_{suf}")(form, nx, T, c2, k, _ptr(fA), _ptr(fB), _ptr(q0), _ptr(q1),
                                                   N, ov, S, _ptr(out0), _ptr(out1), inv2dx,
                                                   _ptr(tr) if (traces and N > 1) else None, ns, _ptr(sj), _ptr(sv))
    if rc:
        raise RuntimeError(f"oracle_rswr_mask failed ({rc})")
    return {"u": out0, "w": out1, "traces": tr, "coeffs": cf}


def rswr_paper(nx, T, a, dt, fA, fB, N, ov, *, form=CANONICAL, tau0=0, beta=0.1, xa=0.0, xb=1.0):
    """Paper-literal serial RSWR (FP64).  Returns dict(u, w, spans)."""
    cf = coeffs(xa, xb, a, nx, dt)
    fA = _arr(fA, np.float64)
    fB = _arr(fB, np.float64)
    out0 = np.empty(nx)
    out1 = np.empty(nx)
    spans = np.zeros(max(T, 1), np.int64)
    ns = ctypes.c_int64()
    rc = lib().oracle_rswr_paper(form, nx, T, cf.c, cf.c2, cf.k, cf.dx, _ptr(fA), _ptr(fB), N, ov, tau0, beta,
                                 _ptr(out0), _ptr(out1), _ptr(spans), ctypes.addressof(ns))
    if rc:
        raise RuntimeError(f"oracle_rswr_paper failed ({rc})")
    return {"u": out0, "w": out1, "spans": spans[: ns.value].copy(), "coeffs": cf}


def adjoint(nx, T, a, dt, fA, fB, j_r, wbar, *, xa=0.0, xb=1.0, nx_run=None):
    """Gradients of <wbar, trace> w.r.t. fA and a (canonical FP64 leapfrog).

    Returns dict(dg[T+1], dc2, da, abs_dc2, abs_da)."""
    cf = coeffs(xa, xb, a, nx, dt)
    nx = nx if nx_run is None else int(nx_run)
    fA = _arr(fA, np.float64)
    fB = _arr(fB, np.float64)
    wbar = _arr(wbar, np.float64)
    dg = np.empty(T + 1)
    dc2 = ctypes.c_double()
    adc2 = ctypes.c_double()
    rc = lib().oracle_adjoint(nx, T, cf.c2, cf.k, _ptr(fA), _ptr(fB), j_r, _ptr(wbar), _ptr(dg),
                              ctypes.addressof(dc2), ctypes.addressof(adc2))
    if rc:
        raise RuntimeError(f"oracle_adjoint failed ({rc})")
    scale = 2.0 * cf.c2 / a
    return {"dg": dg, "dc2": dc2.value, "da": dc2.value * scale, "abs_dc2": adc2.value,
            "abs_da": adc2.value * scale, "coeffs": cf}


def misfit_grad(nx, T, a, dt, fA, fB, j_r, target, *, xa=0.0, xb=1.0, nx_run=None):
    """loss = sum_n (u^n_{j_r} - target^n)^2 and its gradients w.r.t. fA and a."""
    fw = leapfrog(nx, T, a, dt, fA, fB, rec_j=[j_r], xa=xa, xb=xb, nx_run=nx_run)
    trace = fw["rec"][0]
    r = trace - np.asarray(target, np.float64)
    loss = float(np.dot(r, r))
    g = adjoint(nx, T, a, dt, fA, fB, j_r, 2.0 * r, xa=xa, xb=xb, nx_run=nx_run)
    g.update(loss=loss, trace=trace)
    return g


def causal_extent(T: int, nx: int, extra: int = 0) -> int:
    """Points needed to reproduce a zero-initial-data run with a quiet right
    boundary exactly: the solution vanishes for j > n at level n (one cell per
    step), so a grid truncated to T + 2 (+extra) points with Dirichlet 0 at its
    end gives the same values on its points.  Pinned by the oracle tests."""
    return int(min(nx, T + 2 + extra))
