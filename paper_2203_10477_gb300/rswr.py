"""Python binding of librswr (the C ABI in include/rswr.h).

Argument marshalling only: every step of the RSWR path runs in the CUDA
library.  PyTorch supplies device memory and streams.  The raw entry points
keep their C names (``rswr_plan_create``, ``rswr_run``, ``rswr_adjoint``, ...)
on the loaded library object ``lib()``; ``Plan``, ``Batch`` and
``RSWRFunction`` are thin conveniences over them.

There is no fallback: if the library is missing or fails to load, every call
raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "librswr.so")

F32, F64 = 0, 1
FORM_DEFAULT, FORM_CANONICAL, FORM_INCREMENT = 0, 1, 2
MODE_PERSISTENT, MODE_PER_SPAN = 0, 1

STATUS = {0: "RSWR_OK", 1: "RSWR_EINVAL", 2: "RSWR_ECFL", 3: "RSWR_EOVERLAP", 4: "RSWR_ENOMEM",
          5: "RSWR_ECUDA", 6: "RSWR_ETIMEOUT", 7: "RSWR_ENOTSUP"}


class RSWRError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class PlanInfo(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int64), ("dtype", ctypes.c_int32), ("form", ctypes.c_int32),
                ("n_sub", ctypes.c_int32), ("overlap", ctypes.c_int32),
                ("c", ctypes.c_double), ("c2", ctypes.c_double), ("k", ctypes.c_double), ("inv2dx", ctypes.c_double),
                ("c2f", ctypes.c_float), ("kf", ctypes.c_float), ("inv2dxf", ctypes.c_float),
                ("span_steps", ctypes.c_int32), ("halo", ctypes.c_int32), ("core", ctypes.c_int32),
                ("window", ctypes.c_int32), ("points_per_thread", ctypes.c_int32),
                ("threads_per_cta", ctypes.c_int32), ("variant", ctypes.c_int32), ("mode", ctypes.c_int32),
                ("ntiles", ctypes.c_int64), ("state_len", ctypes.c_int64), ("workspace_bytes", ctypes.c_int64)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


class Problem(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int64), ("xa", ctypes.c_double), ("xb", ctypes.c_double),
                ("a", ctypes.c_double), ("dt", ctypes.c_double), ("n_sub", ctypes.c_int32),
                ("overlap", ctypes.c_int32)]


_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_i32 = ctypes.c_int32
_dbl = ctypes.c_double
_st = ctypes.c_int

# name -> (restype, argtypes); names are the C ABI's
SIGNATURES = {
    "rswr_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "rswr_last_error_message": (ctypes.c_char_p, []),
    "rswr_version": (_i32, []),
    "rswr_plan_create": (_st, [ctypes.POINTER(_vp), _dbl, _dbl, _dbl, _i64, _dbl, _i32, _i32, _i32, _i32,
                               ctypes.c_uint32]),
    "rswr_plan_create_part": (_st, [ctypes.POINTER(_vp), _dbl, _dbl, _dbl, _i64, _dbl, _i64, _i64, _i32, _i32, _i32,
                                    _i32, ctypes.c_uint32]),
    "rswr_plan_destroy": (None, [_vp]),
    "rswr_plan_get_info": (_st, [_vp, ctypes.POINTER(PlanInfo)]),
    "rswr_plan_set_span": (_st, [_vp, _i32]),
    "rswr_plan_set_variant": (_st, [_vp, _i32]),
    "rswr_plan_set_mode": (_st, [_vp, _i32]),
    "rswr_plan_set_wait_limit": (_st, [_vp, _dbl]),
    "rswr_plan_set_checkpoint_spacing": (_st, [_vp, _i64]),
    "rswr_plan_set_sources": (_st, [_vp, _i64, _vp, _vp, _i64]),
    "rswr_plan_inject_missing_flag": (_st, [_vp, _i32, _i32]),
    "rswr_plan_autotune": (_st, [_vp, _i64, ctypes.POINTER(_i32), _vp]),
    "rswr_plan_set_kernel_events": (_st, [_vp, _vp, _vp]),
    "rswr_plan_set_graph": (_st, [_vp, _i32]),
    "rswr_batch_set_graph": (_st, [_vp, _i32]),
    "rswr_batch_autotune": (_st, [_vp, _i64, ctypes.POINTER(_i32), _vp]),
    "rswr_batch_set_kernel_events": (_st, [_vp, _vp, _vp]),
    "rswr_batch_set_sources": (_st, [_vp, _i64, _vp, _vp, _vp, _i64]),
    "rswr_plan_check": (_st, [_vp, _vp, ctypes.POINTER(_i32), ctypes.POINTER(_i32), ctypes.POINTER(_i32)]),
    "rswr_run": (_st, [_vp, _vp, _vp, _i64, _vp, _vp, _vp, _vp, _vp, _i64, _vp, _vp]),
    "rswr_run_host": (_st, [_vp, _vp, _vp, _i64, _vp, _vp, _vp, _vp, _vp, _i64, _vp, _vp]),
    "rswr_mono": (_st, [_vp, _vp, _vp, _i64, _vp, _vp, _vp, _vp, _vp, _i64, _vp, _vp]),
    "rswr_run_paper": (_st, [_vp, _vp, _vp, _i64, _vp, _vp, _vp, _vp, _vp, _i64, _vp, _vp]),
    "rswr_adjoint": (_st, [_vp, _vp, _vp, _i64, _i64, _vp, _vp, _vp, _vp]),
    "rswr_run_keep": (_st, [_vp, _vp, _vp, _i64, _i64, _vp, _vp, _vp, _vp]),
    "rswr_batch_create": (_st, [ctypes.POINTER(_vp), _i32, ctypes.POINTER(Problem), _i32, _i32, ctypes.c_uint32]),
    "rswr_batch_destroy": (None, [_vp]),
    "rswr_batch_offsets": (_st, [_vp, _vp]),
    "rswr_batch_get_info": (_st, [_vp, ctypes.POINTER(PlanInfo)]),
    "rswr_batch_set_mode": (_st, [_vp, _i32]),
    "rswr_batch_set_variant": (_st, [_vp, _i32]),
    "rswr_batch_set_wait_limit": (_st, [_vp, _dbl]),
    "rswr_batch_set_checkpoint_spacing": (_st, [_vp, _i64]),
    "rswr_batch_check": (_st, [_vp, _vp, ctypes.POINTER(_i32), ctypes.POINTER(_i32), ctypes.POINTER(_i32)]),
    "rswr_batch_run": (_st, [_vp, _vp, _vp, _i64, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "rswr_batch_adjoint": (_st, [_vp, _vp, _vp, _i64, _vp, _vp, _vp, _vp, _vp]),
    "rswr_fma_probe": (_st, [_i32, _i64, _i32, _i32, _vp, _vp]),
    "rswr_variant_count": (_i32, []),
    "rswr_variant_get_kind": (_st, [_i32, ctypes.POINTER(_i32)]),
    "rswr_variant_get": (_st, [_i32, ctypes.POINTER(_i32), ctypes.POINTER(_i32), ctypes.POINTER(_i32),
                               ctypes.POINTER(_i32)]),
    "rswr_variant_get_tiling": (_st, [_i32, ctypes.POINTER(_i32), ctypes.POINTER(_i32), ctypes.POINTER(_i32),
                                      ctypes.POINTER(_i32)]),
}

_lib: Optional[ctypes.CDLL] = None


def lib() -> ctypes.CDLL:
    """The loaded library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"librswr is not built ({LIB_PATH}); run paper_2203_10477_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def check(status: int) -> None:
    if status != 0:
        raise RSWRError(status, lib().rswr_last_error_message().decode())


# ----------------------------------------------------------------------------
# torch marshalling
# ----------------------------------------------------------------------------

def _torch():
    import torch

    return torch


def _tdtype(dtype: int):
    torch = _torch()
    return torch.float64 if dtype == F64 else torch.float32


def _ptr(t) -> Optional[int]:
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return t.data_ptr()


def _stream(stream) -> Optional[int]:
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _as_dev(x, dtype: int, device):
    """Host data (numpy / list) -> contiguous device tensor of the plan's dtype."""
    if x is None:
        return None
    torch = _torch()
    if isinstance(x, torch.Tensor):
        t = x.to(device=device, dtype=_tdtype(dtype))
    else:
        t = torch.as_tensor(np.asarray(x), dtype=_tdtype(dtype), device=device)
    return t.contiguous()


def _set_sources(call, dtype, device, problem, j, samples):
    # marshals a source set; returns the device tensors the library reads (kept by the caller)
    torch = _torch()
    if j is None or len(j) == 0:
        check(call(0, None, None, 0) if problem is None else call(0, None, None, None, 0))
        return None
    jj = np.ascontiguousarray(np.asarray(j, dtype=np.int64).reshape(-1))
    sm = _as_dev(samples, dtype, device)
    if sm.dim() != 2 or sm.shape[0] != jj.size:
        raise ValueError("samples must be a 2-D array with one row per source")
    sm = sm.contiguous()
    if problem is None:
        check(call(int(jj.size), jj.ctypes.data, _ptr(sm), int(sm.stride(0))))
        return sm
    pp = np.ascontiguousarray(np.asarray(problem, dtype=np.int32).reshape(-1))
    if pp.size != jj.size:
        raise ValueError("one problem index per source")
    check(call(int(jj.size), pp.ctypes.data, jj.ctypes.data, _ptr(sm), int(sm.stride(0))))
    return sm


def variants() -> list[dict]:
    out = []
    for v in range(lib().rswr_variant_count()):
        d, f, p, n = _i32(), _i32(), _i32(), _i32()
        check(lib().rswr_variant_get(v, ctypes.byref(d), ctypes.byref(f), ctypes.byref(p), ctypes.byref(n)))
        kh, w, ms, th = _i32(), _i32(), _i32(), _i32()
        check(lib().rswr_variant_get_tiling(v, ctypes.byref(kh), ctypes.byref(w), ctypes.byref(ms), ctypes.byref(th)))
        kind = _i32()
        check(lib().rswr_variant_get_kind(v, ctypes.byref(kind)))
        out.append({"variant": v, "dtype": d.value, "form": f.value, "P": p.value, "NT": n.value,
                    "KH": kh.value, "window": w.value, "max_span": ms.value, "threads": th.value,
                    "kind": kind.value, "resident": kind.value == 2})
    return out


def fma_rate(dtype, device=None, target_ms=60.0, reps=3) -> dict:
    """Fused multiply-adds per second of the FP64 (dtype F64) or FP32 (F32)
    pipe on `device`, measured with rswr_fma_probe: 8 blocks of 256 threads
    per SM, the iteration count sized to about `target_ms`, best of `reps`
    launches timed with CUDA events on the current stream."""
    torch = _torch()
    dev = torch.device("cuda" if device is None else device)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    blocks, threads = 8 * sms, 256
    td = torch.float64 if dtype == F64 else torch.float32  # dtypes 2, 3: packed FP32 pairs
    with torch.cuda.device(dev):
        sink = torch.empty(blocks * threads, dtype=td, device=dev)
        stream = torch.cuda.current_stream(dev)

        def launch(iters):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            check(lib().rswr_fma_probe(dtype, iters, blocks, threads, _ptr(sink), _stream(stream)))
            e1.record(stream)
            e1.synchronize()
            return e0.elapsed_time(e1)

        iters = 256
        ms = launch(iters)
        while ms < 5.0:
            iters *= 4
            ms = launch(iters)
        iters = max(1, int(iters * target_ms / ms))
        best = min(launch(iters) for _ in range(reps))
    fmas = 8.0 * iters * blocks * threads * (2 if dtype in (2, 3) else 1)
    return {"fma_per_s": fmas / (best / 1e3), "ms": best, "iters": iters, "blocks": blocks, "threads": threads,
            "sms": sms, "finite": bool(torch.isfinite(sink).all())}


class Plan:
    """One problem (paper Sec. 2.1) split into n_sub overlapping subdomains."""

    def __init__(self, xa, xb, a, nx, dt, n_sub, overlap, dtype=F64, form=FORM_DEFAULT, device=None):
        torch = _torch()
        self.device = torch.device("cuda" if device is None else device)
        self.dtype = dtype
        h = _vp()
        with torch.cuda.device(self.device):
            check(lib().rswr_plan_create(ctypes.byref(h), xa, xb, a, nx, dt, n_sub, overlap, dtype, form, 0))
        self.h = h
        self.nx = nx
        self.n_sub = n_sub
        self.a = a

    @classmethod
    def from_problem(cls, p, dtype=F64, form=FORM_DEFAULT, device=None):
        return cls(p.xa, p.xb, p.a, p.nx, p.dt, p.n_sub, p.overlap, dtype, form, device)

    @classmethod
    def part(cls, xa, xb, a, nx, dt, lo, hi, n_sub, overlap, dtype=F64, form=FORM_DEFAULT, device=None):
        """A plan for the points [lo, hi) of the grid (xa, xb, nx) with the whole
        grid's coefficients (rswr_plan_create_part)."""
        torch = _torch()
        self = cls.__new__(cls)
        self.device = torch.device("cuda" if device is None else device)
        self.dtype = dtype
        h = _vp()
        with torch.cuda.device(self.device):
            check(lib().rswr_plan_create_part(ctypes.byref(h), xa, xb, a, nx, dt, lo, hi, n_sub, overlap, dtype,
                                              form, 0))
        self.h = h
        self.nx = hi - lo
        self.n_sub = n_sub
        self.a = a
        return self

    def close(self):
        if getattr(self, "h", None):
            lib().rswr_plan_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self) -> dict:
        i = PlanInfo()
        check(lib().rswr_plan_get_info(self.h, ctypes.byref(i)))
        return i.as_dict()

    def set_span(self, S: int):
        check(lib().rswr_plan_set_span(self.h, S))

    def set_variant(self, v: int):
        check(lib().rswr_plan_set_variant(self.h, v))

    def set_mode(self, mode: int):
        check(lib().rswr_plan_set_mode(self.h, mode))

    def set_wait_limit(self, seconds: float):
        check(lib().rswr_plan_set_wait_limit(self.h, seconds))

    def set_checkpoint_spacing(self, spans: int):
        """Adjoint checkpoint every `spans` spans (0: automatic)."""
        check(lib().rswr_plan_set_checkpoint_spacing(self.h, spans))

    def set_graph(self, enable: bool):
        check(lib().rswr_plan_set_graph(self.h, int(enable)))

    def set_sources(self, j=None, samples=None):
        """Point sources: source q at grid point j[q] with samples[q, n] (n = 0..T) added when level n
        is formed (rswr_plan_set_sources).  samples: a 2-D array, copied to the plan's device; None clears."""
        self._src_keep = _set_sources(lambda *a: lib().rswr_plan_set_sources(self.h, *a), self.dtype,
                                      self.device, None, j, samples)

    def inject_missing_flag(self, tile: int, span: int):
        check(lib().rswr_plan_inject_missing_flag(self.h, tile, span))

    def set_kernel_events(self, start=None, stop=None):
        """torch.cuda.Event pair recorded around the kernels of every run (None clears)."""
        h = lambda ev: None if ev is None else ev.cuda_event
        if start is not None and (not h(start) or not h(stop)):
            raise ValueError("record the events once before handing them over (torch creates them lazily)")
        check(lib().rswr_plan_set_kernel_events(self.h, h(start), h(stop)))

    def autotune(self, probe_steps: int, stream=None) -> int:
        v = _i32()
        check(lib().rswr_plan_autotune(self.h, probe_steps, ctypes.byref(v), _stream(stream)))
        return v.value

    def check(self, stream=None):
        c, t, s = _i32(), _i32(), _i32()
        st = lib().rswr_plan_check(self.h, _stream(stream), ctypes.byref(c), ctypes.byref(t), ctypes.byref(s))
        check(st)
        return c.value, t.value, s.value

    def _run(self, fn, fA, fB, T, q0=None, q1=None, traces=False, j_r=None, out=None, stream=None):
        torch = _torch()
        dev = self.device
        fA_ = _as_dev(fA, self.dtype, dev)
        fB_ = _as_dev(fB, self.dtype, dev)
        q0_ = _as_dev(q0, self.dtype, dev)
        q1_ = _as_dev(q1, self.dtype, dev)
        td = _tdtype(self.dtype)
        if out is None:
            out = (torch.empty(self.nx, dtype=td, device=dev), torch.empty(self.nx, dtype=td, device=dev))
        tr = torch.empty((max(self.n_sub - 1, 0), 2, T + 1), dtype=td, device=dev) if traces else None
        rec = torch.empty(T + 1, dtype=td, device=dev) if j_r is not None else None
        with torch.cuda.device(dev):
            check(fn(self.h, _ptr(fA_), _ptr(fB_), T, _ptr(q0_), _ptr(q1_), _ptr(out[0]), _ptr(out[1]),
                     _ptr(tr) if (tr is not None and tr.numel()) else None, -1 if j_r is None else int(j_r),
                     _ptr(rec), _stream(stream)))
        return {"u": out[0], "w": out[1], "traces": tr, "recv": rec, "_keep": (fA_, fB_, q0_, q1_)}

    def run(self, fA, fB, T, **kw):
        """RSWR run (the hot path).  Returns dict(u, w, traces, recv) of device tensors."""
        return self._run(lib().rswr_run, fA, fB, T, **kw)

    def run_keep(self, fA, fB, T, j_r=None, out=None, stream=None):
        """A forward run that keeps its span states for the next adjoint with
        dL/da (rswr_run_keep).  Returns dict(u, w, recv) like run()."""
        torch = _torch()
        dev = self.device
        fA_ = _as_dev(fA, self.dtype, dev)
        fB_ = _as_dev(fB, self.dtype, dev)
        td = _tdtype(self.dtype)
        if out is None:
            out = (torch.empty(self.nx, dtype=td, device=dev), torch.empty(self.nx, dtype=td, device=dev))
        rec = torch.empty(T + 1, dtype=td, device=dev) if j_r is not None else None
        with torch.cuda.device(dev):
            check(lib().rswr_run_keep(self.h, _ptr(fA_), _ptr(fB_), T, -1 if j_r is None else int(j_r), _ptr(rec),
                                      _ptr(out[0]), _ptr(out[1]), _stream(stream)))
        return {"u": out[0], "w": out[1], "recv": rec, "_keep": (fA_, fB_)}

    def run_paper(self, fA, fB, T, q0=None, q1=None, out=None, stream=None):
        """The paper-literal RSWR (data-chosen spans).  Returns dict(u, w, spans)."""
        torch = _torch()
        dev = self.device
        fA_ = _as_dev(fA, self.dtype, dev)
        fB_ = _as_dev(fB, self.dtype, dev)
        q0_ = _as_dev(q0, self.dtype, dev)
        q1_ = _as_dev(q1, self.dtype, dev)
        td = _tdtype(self.dtype)
        if out is None:
            out = (torch.empty(self.nx, dtype=td, device=dev), torch.empty(self.nx, dtype=td, device=dev))
        spans = np.zeros(max(T, 1), np.int64)
        ns = ctypes.c_int64()
        with torch.cuda.device(dev):
            check(lib().rswr_run_paper(self.h, _ptr(fA_), _ptr(fB_), T, _ptr(q0_), _ptr(q1_), _ptr(out[0]),
                                       _ptr(out[1]), spans.ctypes.data, len(spans), ctypes.addressof(ns),
                                       _stream(stream)))
        return {"u": out[0], "w": out[1], "spans": spans[: ns.value].copy()}

    def mono(self, fA, fB, T, **kw):
        """Monolithic comparator with the same arguments and results as run()."""
        return self._run(lib().rswr_mono, fA, fB, T, **kw)

    def run_host(self, fA, fB, T, q0=None, q1=None, traces=False, j_r=None, out=None):
        """rswr_run_host on host (numpy or pinned torch CPU) buffers; synchronous."""
        torch = _torch()
        td = _tdtype(self.dtype)

        def host(x):
            if x is None:
                return None
            if isinstance(x, torch.Tensor):
                return x.to(td).contiguous()
            return torch.as_tensor(np.ascontiguousarray(x), dtype=td)

        fA_, fB_, q0_, q1_ = host(fA), host(fB), host(q0), host(q1)
        if out is None:
            out = (torch.empty(self.nx, dtype=td), torch.empty(self.nx, dtype=td))
        tr = torch.empty((max(self.n_sub - 1, 0), 2, T + 1), dtype=td) if traces else None
        rec = torch.empty(T + 1, dtype=td) if j_r is not None else None
        hp = lambda t: None if t is None else t.data_ptr()
        with torch.cuda.device(self.device):
            check(lib().rswr_run_host(self.h, hp(fA_), hp(fB_), T, hp(q0_), hp(q1_), hp(out[0]), hp(out[1]),
                                      hp(tr) if (tr is not None and tr.numel()) else None,
                                      -1 if j_r is None else int(j_r), hp(rec), _stream(None)))
        return {"u": out[0], "w": out[1], "traces": tr, "recv": rec}

    def adjoint(self, fA, fB, T, j_r, wbar, want_a=False, stream=None):
        """grad_fA (and dL/da if want_a) of <wbar, receiver trace>."""
        torch = _torch()
        dev = self.device
        fA_ = _as_dev(fA, self.dtype, dev)
        fB_ = _as_dev(fB, self.dtype, dev)
        w_ = _as_dev(wbar, self.dtype, dev)
        g = torch.empty(T + 1, dtype=_tdtype(self.dtype), device=dev)
        ga = torch.zeros(1, dtype=torch.float64, device=dev) if want_a else None
        with torch.cuda.device(dev):
            check(lib().rswr_adjoint(self.h, _ptr(fA_), _ptr(fB_), T, int(j_r), _ptr(w_), _ptr(g), _ptr(ga),
                                     _stream(stream)))
        return {"grad_fA": g, "grad_a": ga}


class Batch:
    """Many independent problems advanced in one persistent launch."""

    def __init__(self, problems, dtype=F32, form=FORM_DEFAULT, device=None):
        torch = _torch()
        self.device = torch.device("cuda" if device is None else device)
        self.dtype = dtype
        arr = (Problem * len(problems))()
        for i, p in enumerate(problems):
            arr[i] = Problem(p.nx, p.xa, p.xb, p.a, p.dt, p.n_sub, p.overlap)
        h = _vp()
        with torch.cuda.device(self.device):
            check(lib().rswr_batch_create(ctypes.byref(h), len(problems), arr, dtype, form, 0))
        self.h = h
        self.n = len(problems)
        off = np.zeros(self.n + 1, np.int64)
        check(lib().rswr_batch_offsets(self.h, off.ctypes.data))
        self.offsets = off

    def close(self):
        if getattr(self, "h", None):
            lib().rswr_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self) -> dict:
        i = PlanInfo()
        check(lib().rswr_batch_get_info(self.h, ctypes.byref(i)))
        return i.as_dict()

    def set_mode(self, mode: int):
        check(lib().rswr_batch_set_mode(self.h, mode))

    def set_variant(self, v: int):
        check(lib().rswr_batch_set_variant(self.h, v))

    def set_wait_limit(self, seconds: float):
        check(lib().rswr_batch_set_wait_limit(self.h, seconds))

    def set_checkpoint_spacing(self, spans: int):
        check(lib().rswr_batch_set_checkpoint_spacing(self.h, spans))

    def set_sources(self, problem=None, j=None, samples=None):
        """Point sources of the batch: source q belongs to problem[q] and sits at its point j[q]
        (rswr_batch_set_sources); samples as in Plan.set_sources."""
        self._src_keep = _set_sources(lambda *a: lib().rswr_batch_set_sources(self.h, *a), self.dtype,
                                      self.device, problem, j, samples)

    def set_graph(self, enable: bool):
        check(lib().rswr_batch_set_graph(self.h, int(enable)))

    def autotune(self, probe_steps: int, stream=None) -> int:
        v = _i32()
        check(lib().rswr_batch_autotune(self.h, probe_steps, ctypes.byref(v), _stream(stream)))
        return v.value

    def set_kernel_events(self, start=None, stop=None):
        h = lambda ev: None if ev is None else ev.cuda_event
        check(lib().rswr_batch_set_kernel_events(self.h, h(start), h(stop)))

    def check(self, stream=None):
        c, t, s = _i32(), _i32(), _i32()
        check(lib().rswr_batch_check(self.h, _stream(stream), ctypes.byref(c), ctypes.byref(t), ctypes.byref(s)))
        return c.value, t.value, s.value

    def run(self, fA, fB, T, q0=None, q1=None, j_r=None, out=None, stream=None):
        torch = _torch()
        dev = self.device
        td = _tdtype(self.dtype)
        fA_ = _as_dev(fA, self.dtype, dev)
        fB_ = _as_dev(fB, self.dtype, dev)
        q0_ = _as_dev(q0, self.dtype, dev)
        q1_ = _as_dev(q1, self.dtype, dev)
        n = int(self.offsets[-1])
        if out is None:
            out = (torch.empty(n, dtype=td, device=dev), torch.empty(n, dtype=td, device=dev))
        jr = None
        rec = None
        if j_r is not None:
            jr = np.ascontiguousarray(j_r, dtype=np.int64)
            rec = torch.empty((self.n, T + 1), dtype=td, device=dev)
        with torch.cuda.device(dev):
            check(lib().rswr_batch_run(self.h, _ptr(fA_), _ptr(fB_), T, _ptr(q0_), _ptr(q1_), _ptr(out[0]),
                                       _ptr(out[1]), None if jr is None else jr.ctypes.data, _ptr(rec),
                                       _stream(stream)))
        return {"u": out[0], "w": out[1], "recv": rec, "_keep": (fA_, fB_, q0_, q1_, jr)}

    def adjoint(self, fA, fB, T, j_r, wbar, want_a=False, stream=None):
        torch = _torch()
        dev = self.device
        td = _tdtype(self.dtype)
        fA_ = _as_dev(fA, self.dtype, dev)
        fB_ = _as_dev(fB, self.dtype, dev)
        w_ = _as_dev(wbar, self.dtype, dev)
        jr = np.ascontiguousarray(j_r, dtype=np.int64)
        g = torch.empty((self.n, T + 1), dtype=td, device=dev)
        ga = torch.zeros(self.n, dtype=torch.float64, device=dev) if want_a else None
        with torch.cuda.device(dev):
            check(lib().rswr_batch_adjoint(self.h, _ptr(fA_), _ptr(fB_), T, jr.ctypes.data, _ptr(w_), _ptr(g),
                                           _ptr(ga), _stream(stream)))
        return {"grad_fA": g, "grad_a": ga}


def _make_function():
    torch = _torch()

    class RSWRFunction(torch.autograd.Function):
        """recv = RSWRFunction.apply(fA, a, plan, T, j_r[, fB]): the receiver trace
        of an RSWR run as a differentiable function of the left boundary waveform
        fA and of the wave speed a (a one-element tensor equal to the plan's
        speed).  The right boundary waveform fB (T+1 samples, default 0) enters
        the forward run and the gradient w.r.t. a, but is data: a fB that
        requires a gradient is refused.  Backward calls rswr_adjoint (the
        library's adjoint kernels)."""

        @staticmethod
        def forward(ctx, fA, a, plan: Plan, T: int, j_r: int, fB=None):
            if a is not None and abs(float(a) - plan.a) > 1e-15 * max(1.0, abs(plan.a)):
                raise ValueError("a must equal the plan's wave speed")
            if fB is not None and fB.requires_grad:
                raise ValueError("gradients w.r.t. the right boundary waveform fB are not provided")
            # the plan's dtype on its device, so that backward passes the very
            # arrays the forward run read
            fA_d = _as_dev(fA.detach(), plan.dtype, plan.device)
            fB_d = None if fB is None else _as_dev(fB.detach(), plan.dtype, plan.device)
            want_a = a is not None and a.requires_grad
            # with dL/da wanted, the forward run keeps its span states for backward
            res = (plan.run_keep if want_a else plan.run)(fA_d, fB_d, T, j_r=j_r)
            ctx.save_for_backward(fA_d, fB_d)
            ctx.plan, ctx.T, ctx.j_r, ctx.want_a = plan, T, j_r, want_a
            ctx.a_shape = None if a is None else a.shape
            ctx.n_inputs = 6 if fB is not None else 5
            return res["recv"]

        @staticmethod
        def backward(ctx, grad_out):
            fA, fB = ctx.saved_tensors
            g = ctx.plan.adjoint(fA, fB, ctx.T, ctx.j_r, grad_out.contiguous(), want_a=ctx.want_a)
            ga = None
            if ctx.want_a:
                ga = g["grad_a"].reshape(ctx.a_shape).to(grad_out.dtype)
            return (g["grad_fA"], ga, None, None, None, None)[: ctx.n_inputs]

    return RSWRFunction


_fn_cache = None


def rswr_function():
    global _fn_cache
    if _fn_cache is None:
        _fn_cache = _make_function()
    return _fn_cache
