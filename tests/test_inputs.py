"""The synthetic workload recipes: seeded, reproducible, and shaped as stated."""
from __future__ import annotations

import numpy as np

from paper_2203_10477_gb300 import inputs


def test_recipes_are_reproducible_and_sized():
    a, b = inputs.c3_table(64), inputs.c3_table(64)
    for k in ("nx", "a", "f"):
        assert np.array_equal(a[k], b[k])
    assert a["nx"].min() >= 1 << 10 and a["nx"].max() <= 1 << 18
    p = inputs.c2(T=100, nx=1 << 12)
    assert p.fA.shape == (101,) and p.n_sub == 1024 and p.overlap == 64
    assert abs(p.a * p.dt / inputs.grid_dx(p.nx) - 0.9) < 1e-15
    c4 = inputs.c4()
    assert c4.meta["j_r"] == int(np.floor(0.7 * (c4.nx - 1)))


def test_pulse_sources_follow_their_recipe():
    nx, T = 100_001, 2000
    dt = inputs.dt_for_cfl(nx, 1.0, 0.9)
    j, s = inputs.pulse_sources(nx, T, dt, K=10)
    j2, s2 = inputs.pulse_sources(nx, T, dt, K=10)
    assert np.array_equal(j, j2) and np.array_equal(s, s2)
    # one source at the centre of each of ten equal cells
    assert np.array_equal(j, [(2 * q + 1) * (nx - 1) // 20 for q in range(10)])
    assert s.shape == (10, T + 1)
    # Gaussian pulses of width 30 dt centred within [4, 6] widths, amplitude at most 1/30
    peak = np.argmax(np.abs(s), axis=1)
    assert np.all((peak >= 4 * 30 - 1) & (peak <= 6 * 30 + 1))
    assert np.abs(s).max() <= 1.0 / 30.0 + 1e-15
    p, jj, ss = inputs.pulse_experiment(nx=4096, T=50)
    assert p.n_sub == 10 and p.overlap == 64 and not p.fA.any() and not p.fB.any()
    assert jj.shape == (10,) and ss.shape == (10, 51)
