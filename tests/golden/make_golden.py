"""Writes the stored expected values of tests/golden/ from the CPU oracle.

Only oracle/ computes the values (and inputs.py, which draws the seeded
workload data); nothing here or in the fixtures comes from the CUDA path.  The
fixtures are regression values of the oracle, not pins of it: the pins are in
tests/test_oracle_pins.py.

    python tests/golden/make_golden.py
"""
from __future__ import annotations

import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2203_10477_gb300 import inputs  # noqa: E402

RECV_J = 500
U_POINTS = list(range(0, 1001, 50))
LEVELS = list(range(0, 2001, 100))


def problem():
    """The c1 grid (nx = 1001 on [0, 1], a = 1, CFL 0.5, 2000 steps, N = 2,
    overlap 16) with a boundary pulse built from additions and products only,
    64 s^3 (1 - s)^3 with s = min(n / 400, 1), so that the stored values do not
    depend on a platform's sin / exp."""
    p = inputs.c1()
    s = np.minimum(np.arange(p.T + 1, dtype=np.float64) / 400.0, 1.0)
    q = s * (1.0 - s)
    p.fA = 64.0 * (q * q * q)
    return p


def c1_values():
    """FP64 canonical leapfrog of problem(): the monolithic solve that RSWR
    reproduces (Sec. 2.4), and the serial RSWR's interface output waveforms."""
    p = problem()
    ref = oracle.leapfrog(p.nx, p.T, p.a, p.dt, p.fA, p.fB, rec_j=[RECV_J])
    rs = oracle.rswr_mask(p.nx, p.T, p.a, p.dt, p.fA, p.fB, p.n_sub, p.overlap)
    return {
        "u_T": [(j, ref["u"][j]) for j in U_POINTS],
        "recv": [(n, ref["rec"][0][n]) for n in LEVELS],
        "trace_left": [(n, rs["traces"][0, 0, n]) for n in LEVELS],
        "trace_right": [(n, rs["traces"][0, 1, n]) for n in LEVELS],
    }


def write(path, vals):
    with open(path, "w") as f:
        f.write("# c1 grid (nx = 1001, N = 2, overlap 16, CFL 0.5, 2000 steps, FP64 canonical) with the\n")
        f.write("# boundary pulse 64 s^3 (1 - s)^3, s = min(n / 400, 1) (make_golden.problem):\n")
        f.write("# oracle values written by tests/golden/make_golden.py (oracle/ only).\n")
        f.write(f"# u_T: final level at grid point j; recv: u at j = {RECV_J} per level n;\n")
        f.write("# trace_left / trace_right: the interface output waveforms of Sec. 2.2 per level n.\n")
        f.write("# columns: series index value(hex) value(decimal)\n")
        for key, rows in vals.items():
            for i, v in rows:
                f.write(f"{key} {i} {float(v).hex()} {float(v):.17g}\n")


def read(path):
    out = {}
    with open(path) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            key, i, h, _ = line.split()
            out.setdefault(key, []).append((int(i), float.fromhex(h)))
    return out


if __name__ == "__main__":
    write(os.path.join(HERE, "c1_fp64.txt"), c1_values())
