"""The stored oracle values of tests/golden/ (regression fixtures, written by
tests/golden/make_golden.py from oracle/ only) are reproduced bit for bit."""
from __future__ import annotations

import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))

import make_golden  # noqa: E402


def test_c1_fixture_regenerates_bit_for_bit():
    stored = make_golden.read(os.path.join(HERE, "golden", "c1_fp64.txt"))
    fresh = make_golden.c1_values()
    assert set(stored) == set(fresh)
    for key, rows in fresh.items():
        assert [(i, float(v)) for i, v in rows] == stored[key], key
