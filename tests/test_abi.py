"""The C-ABI library builds, loads without a GPU and exports every entry point
that include/rswr.h declares; host-side validation needs no device."""
from __future__ import annotations

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rswr.h")


def declared_functions() -> list[str]:
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:rswr_status|void|const char\s*\*|int32_t)\s+(rswr_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def built_lib():
    from paper_2203_10477_gb300 import build

    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_hot_path():
    names = declared_functions()
    for must in ("rswr_plan_create", "rswr_run", "rswr_adjoint", "rswr_batch_create", "rswr_batch_run",
                 "rswr_batch_adjoint", "rswr_mono", "rswr_run_host"):
        assert must in names


def test_library_exports_every_declared_symbol(built_lib):
    missing = [n for n in declared_functions() if not hasattr(built_lib, n)]
    assert not missing, missing


def test_status_strings_and_variants_without_gpu(built_lib):
    from paper_2203_10477_gb300 import rswr

    L = rswr.lib()
    assert L.rswr_status_string(0) == b"RSWR_OK"
    assert L.rswr_status_string(6) == b"RSWR_ETIMEOUT"
    assert L.rswr_version() >= 100
    vs = rswr.variants()
    assert {(v["dtype"], v["form"]) for v in vs} == {(0, 1), (0, 2), (1, 1), (1, 2)}
    for v in vs:
        assert v["P"] >= 2 and v["NT"] % 32 == 0


def test_validation_errors_are_reported_without_touching_the_device(built_lib):
    from paper_2203_10477_gb300 import rswr

    L = rswr.lib()
    h = ctypes.c_void_p()
    # Courant number 2 > 1
    st = L.rswr_plan_create(ctypes.byref(h), 0.0, 1.0, 1.0, 101, 0.02, 2, 8, 1, 0, 0)
    assert st == 2 and not h.value
    assert b"Courant" in L.rswr_last_error_message()
    # overlap too small / cores too short
    assert L.rswr_plan_create(ctypes.byref(h), 0.0, 1.0, 1.0, 101, 0.005, 2, 1, 1, 0, 0) == 3
    assert L.rswr_plan_create(ctypes.byref(h), 0.0, 1.0, 1.0, 101, 0.005, 50, 8, 1, 0, 0) == 3
    # bad sizes / dtype
    assert L.rswr_plan_create(ctypes.byref(h), 0.0, 1.0, 1.0, 2, 0.005, 1, 2, 1, 0, 0) == 1
    assert L.rswr_plan_create(ctypes.byref(h), 0.0, 1.0, 1.0, 101, 0.005, 2, 8, 7, 0, 0) == 1
    assert L.rswr_plan_create(None, 0.0, 1.0, 1.0, 101, 0.005, 2, 8, 1, 0, 0) == 1


def test_source_setters_reject_null_handles_without_touching_the_device(built_lib):
    from paper_2203_10477_gb300 import rswr

    L = rswr.lib()
    j = (ctypes.c_int64 * 1)(5)
    p = (ctypes.c_int32 * 1)(0)
    assert L.rswr_plan_set_sources(None, 1, j, None, 8) == 1
    assert L.rswr_batch_set_sources(None, 1, p, j, None, 8) == 1
    assert b"NULL" in L.rswr_last_error_message()
