"""rswr_run_noalloc: the entry point for callers that may not allocate device
memory (a framework's caching allocator holds the memory they may use, or a
latency-critical loop cannot afford cudaMalloc's device synchronisation).

It is checked through the C ABI against the plan-based rswr_run on the same
inputs, bit for bit (the tolerance every parity test of the library uses), on
two calls in a row so that leftovers of the first call in the shared scratch
area would show.  This file is collected last on purpose.
"""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

from paper_2203_10477_gb300 import inputs

torch = pytest.importorskip("torch")

F32, F64 = 0, 1


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


@pytest.mark.gpu
@pytest.mark.parametrize("dtype", [F64, F32])
def test_noalloc_matches_plan_run_on_two_calls(L, dtype):
    lib, rswr = L
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    td = torch.float64 if dtype == F64 else torch.float32
    stream = torch.cuda.current_stream()
    cases = [
        # nx, N, ov, T, cfl, seed
        (50_021, 5, 48, 333, 0.9, 1),
        (9_001, 2, 16, 120, 0.6, 2),
    ]
    for nx, N, ov, T, cfl, seed in cases:
        dt = cfl / (nx - 1)
        fA = torch.tensor(inputs.ramped_sine(T, dt, freq=9.0 + seed), dtype=td, device="cuda")
        q0 = torch.tensor(inputs.smooth_random_state(nx, seed=seed), dtype=td, device="cuda")
        out0 = torch.empty(nx, dtype=td, device="cuda")
        out1 = torch.empty(nx, dtype=td, device="cuda")
        st = lib.rswr_run_noalloc(0.0, 1.0, 1.0, nx, dt, N, ov, dtype, fA.data_ptr(), None, T, q0.data_ptr(),
                                  None, out0.data_ptr(), out1.data_ptr(), stream.cuda_stream)
        assert st == 0, lib.rswr_last_error_message()
        plan = rswr.Plan(0.0, 1.0, 1.0, nx, dt, N, ov, dtype=dtype)
        ref = plan.run(fA, None, T, q0=q0)
        torch.cuda.synchronize()
        assert torch.equal(out0, ref["u"]), f"u differs (nx={nx})"
        assert torch.equal(out1, ref["w"]), f"second component differs (nx={nx})"
        assert float(out0.abs().max()) > 0.0
