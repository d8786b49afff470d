"""Seeded synthetic inputs for the RSWR wave-equation workloads.

This module only *describes problems*: grid sizes, wave speeds, time steps,
boundary waveforms (Dirichlet data f_A(t), f_B(t) of the paper's problem
statement, Sec. 2.1) and smooth random initial states used by the tests.
It holds none of the method's arithmetic (no stencil, no decomposition, no
stability coefficients): both the CUDA library and the CPU oracle derive their
own coefficients from the numbers produced here.

Every random draw uses numpy's PCG64 with an explicit seed; the draw order is
part of the recipe and must not change.

The paper's experiments (Sec. 4) give no grid, source placement or data, so
these five workloads stand in for them:

* ``c1``  nx=1001 on [0,1], a=1, CFL 0.5, 2000 steps, N=2 subdomains,
          16-point overlap, left boundary a ramped 5 Hz sine, right boundary 0.
* ``c2``  nx=2**24, a=1, CFL 0.9, 10**4 steps, N=1024, overlap 64,
          left boundary Gaussian pulse (sigma = 50 dt, t0 = 4 sigma).
* ``c3``  4096 independent problems, nx uniform in [2**10, 2**18], a uniform in
          [0.5, 2], CFL 0.8, 4096 steps, N_p = ceil(nx/2048), overlap 32,
          left boundary sin(2 pi f t), f uniform in [1, 20].
* ``c4``  adjoint workload: nx=2**20, a=1.3, CFL 0.9, 8192 steps, N=256,
          overlap 64, left boundary low-passed white noise, receiver at x=0.7,
          target trace produced with a=1.0 on the same grid and time step.
* ``c5``  nx=2**28, N=8192, overlap 64, 2**15 steps, plus 512 uneven problems
          with nx in [2**12, 2**20] carrying boundary-waveform gradients.

The paper's N = 10 experiment (Sec. 4) inserts ten pulse sources and splits
the domain into ten subdomains without stating where the sources sit or what
they emit; ``pulse_sources`` / ``pulse_experiment`` fix that choice (one
Gaussian pulse at the centre of each of K equal cells, staggered onsets,
random amplitudes).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED = 10477


def rng(seed: int = SEED) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


@dataclass
class Problem:
    """One 1-D wave problem u_tt = a^2 u_xx on [xa, xb] with nx grid points.

    ``dt`` is the time step; ``T`` the number of steps; ``n_sub`` and
    ``overlap`` the overlapping decomposition (overlap = number of grid
    points shared by two neighbouring subdomains).  ``fA``/``fB`` hold the
    Dirichlet samples at t_n = n*dt for n = 0..T (float64).
    """

    nx: int
    a: float
    dt: float
    T: int
    n_sub: int
    overlap: int
    fA: np.ndarray
    fB: np.ndarray
    xa: float = 0.0
    xb: float = 1.0
    meta: dict = field(default_factory=dict)


def grid_dx(nx: int, xa: float = 0.0, xb: float = 1.0) -> float:
    return (xb - xa) / (nx - 1)


def dt_for_cfl(nx: int, a: float, cfl: float, xa: float = 0.0, xb: float = 1.0) -> float:
    """Time step giving Courant number ``cfl`` = a*dt/dx on the uniform grid."""
    return cfl * grid_dx(nx, xa, xb) / a


def times(T: int, dt: float) -> np.ndarray:
    return np.arange(T + 1, dtype=np.float64) * dt


def ramped_sine(T: int, dt: float, freq: float = 5.0, ramp: float = 0.05) -> np.ndarray:
    """sin(2 pi freq t) * (1 - exp(-(t/ramp)^2)), t = n dt, n = 0..T."""
    t = times(T, dt)
    return np.sin(2.0 * np.pi * freq * t) * (1.0 - np.exp(-((t / ramp) ** 2)))


def gaussian_pulse(T: int, dt: float, sigma_steps: float = 50.0, t0_sigmas: float = 4.0) -> np.ndarray:
    """exp(-((t - t0)/sigma)^2) with sigma = sigma_steps*dt and t0 = t0_sigmas*sigma."""
    t = times(T, dt)
    sigma = sigma_steps * dt
    t0 = t0_sigmas * sigma
    return np.exp(-(((t - t0) / sigma) ** 2))


def sine(T: int, dt: float, freq: float) -> np.ndarray:
    return np.sin(2.0 * np.pi * freq * times(T, dt))


def lowpass_noise(T: int, seed: int = SEED, keep_frac: float = 0.1) -> np.ndarray:
    """N(0,1) samples (T+1 of them) with every rfft bin above keep_frac*Nyquist zeroed."""
    g = rng(seed).standard_normal(T + 1)
    G = np.fft.rfft(g)
    nyq_bin = len(G) - 1
    G[np.arange(len(G)) > keep_frac * nyq_bin] = 0.0
    return np.fft.irfft(G, n=T + 1)


def smooth_random_state(nx: int, seed: int = SEED, modes: int = 24) -> np.ndarray:
    """A smooth random field on nx points (sum of low sine modes), zero at both ends."""
    r = rng(seed)
    x = np.linspace(0.0, 1.0, nx)
    amp = r.standard_normal(modes) / (1.0 + np.arange(modes))
    u = np.zeros(nx)
    for m in range(modes):
        u += amp[m] * np.sin(np.pi * (m + 1) * x)
    u[0] = 0.0
    u[-1] = 0.0
    return u


def receiver_index(nx: int, x_r: float, xa: float = 0.0, xb: float = 1.0) -> int:
    return int(math.floor((x_r - xa) / (xb - xa) * (nx - 1)))


# ----------------------------------------------------------------------------
# The five workloads
# ----------------------------------------------------------------------------

def c1() -> Problem:
    nx, a, cfl, T = 1001, 1.0, 0.5, 2000
    dt = dt_for_cfl(nx, a, cfl)
    return Problem(nx, a, dt, T, 2, 16, ramped_sine(T, dt), np.zeros(T + 1),
                   meta={"name": "c1", "cfl": cfl})


def c2(T: int = 10_000, nx: int = 1 << 24) -> Problem:
    a, cfl = 1.0, 0.9
    dt = dt_for_cfl(nx, a, cfl)
    return Problem(nx, a, dt, T, 1024, 64, gaussian_pulse(T, dt), np.zeros(T + 1),
                   meta={"name": "c2", "cfl": cfl})


def c3_table(P: int = 4096, seed: int = SEED) -> dict:
    """Draws (in this order) nx_p, a_p, f_p for P problems."""
    r = rng(seed)
    nx = r.integers(1 << 10, 1 << 18, size=P, endpoint=True)
    a = r.uniform(0.5, 2.0, size=P)
    f = r.uniform(1.0, 20.0, size=P)
    return {"nx": nx.astype(np.int64), "a": a, "f": f}


def c3_problems(P: int = 4096, T: int = 4096, seed: int = SEED, cfl: float = 0.8,
                overlap: int = 32, sub_len: int = 2048) -> list[Problem]:
    tab = c3_table(P, seed)
    out = []
    for p in range(P):
        nx = int(tab["nx"][p])
        a = float(tab["a"][p])
        dt = dt_for_cfl(nx, a, cfl)
        n_sub = -(-nx // sub_len)
        out.append(Problem(nx, a, dt, T, n_sub, overlap, sine(T, dt, float(tab["f"][p])),
                           np.zeros(T + 1), meta={"name": f"c3[{p}]", "cfl": cfl, "f": float(tab["f"][p])}))
    return out


def c4(T: int = 8192, nx: int = 1 << 20, j_r: int | None = None) -> Problem:
    """Adjoint workload.  ``meta['j_r']`` is the receiver grid index (x_r = 0.7
    unless given) and ``meta['a_target']`` the speed that made the target."""
    a, cfl = 1.3, 0.9
    dt = dt_for_cfl(nx, a, cfl)
    jr = receiver_index(nx, 0.7) if j_r is None else int(j_r)
    return Problem(nx, a, dt, T, 256, 64, lowpass_noise(T), np.zeros(T + 1),
                   meta={"name": "c4", "cfl": cfl, "j_r": jr, "a_target": 1.0})


def c5_big(T: int = 1 << 15, nx: int = 1 << 28) -> Problem:
    a, cfl = 1.0, 0.9
    dt = dt_for_cfl(nx, a, cfl)
    return Problem(nx, a, dt, T, 8192, 64, gaussian_pulse(T, dt), np.zeros(T + 1),
                   meta={"name": "c5", "cfl": cfl})


def c5_uneven(P: int = 512, T: int = 1 << 15, seed: int = SEED + 5, cfl: float = 0.9,
              overlap: int = 64, sub_len: int = 2048) -> list[Problem]:
    r = rng(seed)
    nx = r.integers(1 << 12, 1 << 20, size=P, endpoint=True)
    a = r.uniform(0.5, 2.0, size=P)
    out = []
    for p in range(P):
        n = int(nx[p])
        ap = float(a[p])
        dt = dt_for_cfl(n, ap, cfl)
        jr = min(receiver_index(n, 0.7), T // 2)
        out.append(Problem(n, ap, dt, T, -(-n // sub_len), overlap, gaussian_pulse(T, dt),
                           np.zeros(T + 1), meta={"name": f"c5u[{p}]", "cfl": cfl, "j_r": jr,
                                                  "a_target": 0.8 * ap}))
    return out


def pulse_sources(nx: int, T: int, dt: float, K: int = 10, seed: int = SEED + 10,
                  sigma_steps: float = 30.0) -> tuple[np.ndarray, np.ndarray]:
    """K interior pulse sources.  Source q sits at j_q = floor((q + 1/2)(nx - 1)/K),
    the centre of the q-th of K equal cells, and emits
    A_q / sigma_steps * exp(-((t - t_q)/sigma)^2) with sigma = sigma_steps*dt,
    t_q = (4 + 2 s_q) sigma; s_q uniform in [0, 1), A_q uniform in [-1, 1]
    (draw order: all s, then all A).  Returns (j[K] int64, samples[K, T+1])."""
    r = rng(seed)
    s = r.uniform(0.0, 1.0, size=K)
    A = r.uniform(-1.0, 1.0, size=K)
    t = times(T, dt)
    sigma = sigma_steps * dt
    j = np.array([((2 * q + 1) * (nx - 1)) // (2 * K) for q in range(K)], dtype=np.int64)
    samples = np.empty((K, T + 1))
    for q in range(K):
        samples[q] = A[q] / sigma_steps * np.exp(-(((t - (4.0 + 2.0 * s[q]) * sigma) / sigma) ** 2))
    return j, samples


def pulse_experiment(nx: int = 1 << 24, T: int = 10_000, K: int = 10) -> tuple[Problem, np.ndarray, np.ndarray]:
    """The N = 10 pulse-source experiment: a=1 on [0, 1], CFL 0.9, N = 10
    subdomains, overlap 64, zero Dirichlet data, K pulse sources from
    ``pulse_sources``.  Returns (problem, j, samples)."""
    a, cfl = 1.0, 0.9
    dt = dt_for_cfl(nx, a, cfl)
    j, samples = pulse_sources(nx, T, dt, K)
    return (Problem(nx, a, dt, T, 10, 64, np.zeros(T + 1), np.zeros(T + 1),
                    meta={"name": "pulse10", "cfl": cfl, "sources": K}), j, samples)
