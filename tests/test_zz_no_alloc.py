"""rswr_run_noalloc: the entry point for callers that may not allocate device
memory (a framework's caching allocator holds the memory they may use, or a
latency-critical loop cannot afford cudaMalloc's device synchronisation).

Checked through the C ABI, bit for bit (the bar of every parity test of the
library), against the CPU oracle running the same operation order and against
the plan-based rswr_run on the same inputs, on two calls in a row, so that
leftovers of the first call in the shared scratch area would show.  One case
has a right Dirichlet waveform and an explicit second state component.  This
file is collected last on purpose.
"""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

from paper_2203_10477_gb300 import inputs

torch = pytest.importorskip("torch")

F32, F64 = 0, 1
ORACLE = {F64: (0, "f64"), F32: (1, "f32")}  # canonical FP64, increment FP32


@pytest.fixture(scope="module")
def L():
    from paper_2203_10477_gb300 import build, rswr

    build.build()
    lib = rswr.lib()
    f = lib.rswr_run_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int64, ctypes.c_double,
                  ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                  ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                  ctypes.c_void_p]
    return lib, rswr


def test_rejects_problems_larger_than_the_scratch_area(L):
    lib, _ = L
    out = ctypes.c_void_p(16)  # never touched: the size check comes first
    st = lib.rswr_run_noalloc(0.0, 1.0, 1.0, 1 << 22, 0.5 / ((1 << 22) - 1), 4, 64, F64, None, None, 10,
                              None, None, out, out, None)
    assert st == 1
    assert b"scratch" in lib.rswr_last_error_message()


def _ptr(t):
    return None if t is None else t.data_ptr()


@pytest.mark.gpu
@pytest.mark.parametrize("dtype", [F64, F32])
def test_noalloc_matches_oracle_and_plan_run_on_two_calls(L, oracle_mod, dtype):
    lib, rswr = L
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    td = torch.float64 if dtype == F64 else torch.float32
    npd = np.float64 if dtype == F64 else np.float32
    oform, oprec = ORACLE[dtype]
    stream = torch.cuda.current_stream()
    cases = [
        # nx, N, ov, T, cfl, seed, right Dirichlet waveform and explicit q1
        (50_021, 5, 48, 333, 0.9, 1, False),
        (9_001, 2, 16, 120, 0.6, 2, True),
    ]
    for nx, N, ov, T, cfl, seed, full in cases:
        dt = cfl / (nx - 1)
        fA_h = inputs.ramped_sine(T, dt, freq=9.0 + seed).astype(npd)
        q0_h = inputs.smooth_random_state(nx, seed=seed).astype(npd)
        fB_h = inputs.ramped_sine(T, dt, freq=4.0).astype(npd) * npd(0.5) if full else None
        if full:
            # a second component that is not the default (u^{-1} = u^0, v^0 = 0)
            q1_h = (inputs.smooth_random_state(nx, seed=seed + 7) * 1e-3).astype(npd)
            if oform == 0:
                q1_h = (q0_h + q1_h).astype(npd)
        else:
            q1_h = None
        dev = lambda a: None if a is None else torch.tensor(a, dtype=td, device="cuda")
        fA, fB, q0, q1 = dev(fA_h), dev(fB_h), dev(q0_h), dev(q1_h)
        out0 = torch.empty(nx, dtype=td, device="cuda")
        out1 = torch.empty(nx, dtype=td, device="cuda")
        st = lib.rswr_run_noalloc(0.0, 1.0, 1.0, nx, dt, N, ov, dtype, _ptr(fA), _ptr(fB), T, _ptr(q0),
                                  _ptr(q1), out0.data_ptr(), out1.data_ptr(), stream.cuda_stream)
        assert st == 0, lib.rswr_last_error_message()
        zb = np.zeros(T + 1, npd)
        ref = oracle_mod.leapfrog(nx, T, 1.0, dt, fA_h, zb if fB_h is None else fB_h, form=oform, prec=oprec,
                                  q0=q0_h, q1=q1_h)
        got0, got1 = out0.cpu().numpy(), out1.cpu().numpy()
        assert np.array_equal(got0, ref["u"]), f"u differs from the oracle (nx={nx})"
        assert np.array_equal(got1, ref["w"]), f"second component differs from the oracle (nx={nx})"
        assert np.abs(got0).max() > 0.0
        plan = rswr.Plan(0.0, 1.0, 1.0, nx, dt, N, ov, dtype=dtype)
        pr = plan.run(fA, fB, T, q0=q0, q1=q1)
        torch.cuda.synchronize()
        assert torch.equal(out0, pr["u"]) and torch.equal(out1, pr["w"]), f"differs from rswr_run (nx={nx})"
