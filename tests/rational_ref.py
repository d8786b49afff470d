"""Exact rational brute force of the leapfrog and of serial RSWR (tiny grids).

Test-only.  Written independently of ``oracle/`` (pure Python ``Fraction``
arithmetic, no rounding) so that the oracle can be pinned against it: any
floating-point result of the oracle must lie within rounding of these values,
and the method's exactness claims (Decomposition / Prediction Validation /
Global Maximum Waveform Time Span theorems, paper Sec. 2.2, 2.4, 3) can be
checked without any rounding at all.
"""
from __future__ import annotations

from fractions import Fraction


def _sources(new, n, nx, sources, lo=1, hi=None):
    """Point sources (j, samples): samples[n + 1] joins level n + 1 at interior point j."""
    hi = nx - 2 if hi is None else hi
    for j, smp in sources:
        if 0 < j < nx - 1 and lo <= j <= hi:
            new[j] += Fraction(smp[n + 1])


def leapfrog(nx, T, c2, k, fA, fB, u0=None, up=None, sources=()):
    """u^{n+1}_j = c2 (u^n_{j-1} + u^n_{j+1}) + k u^n_j - u^{n-1}_j on interior j,
    Dirichlet fA/fB; zero initial data with u^{-1} = u^0 unless given; point
    sources [(j, samples)] add samples[n+1] at j when level n+1 is formed.
    Returns the list of all levels u^0..u^T."""
    u = [Fraction(0)] * nx if u0 is None else [Fraction(x) for x in u0]
    u[0], u[-1] = Fraction(fA[0]), Fraction(fB[0])
    prev = list(u) if up is None else [Fraction(x) for x in up]
    levels = [list(u)]
    for n in range(T):
        new = [Fraction(0)] * nx
        for j in range(1, nx - 1):
            new[j] = c2 * (u[j - 1] + u[j + 1]) + k * u[j] - prev[j]
        _sources(new, n, nx, sources)
        new[0], new[-1] = Fraction(fA[n + 1]), Fraction(fB[n + 1])
        prev, u = u, new
        levels.append(list(u))
    return levels


def rswr_mask(nx, T, c2, k, fA, fB, N, ov, S, u0=None, up=None, sources=()):
    """Serial RSWR with zero-flux (mirror) predictions and core write-back.
    Windows extend ceil(ov/2) left and floor(ov/2) right of the cores
    b_i = floor(i nx / N); each window applies the point sources it contains.
    Returns the final level pair (u^T, u^{T-1})."""
    el, er = (ov + 1) // 2, ov // 2
    u = [Fraction(0)] * nx if u0 is None else [Fraction(x) for x in u0]
    u[0], u[-1] = Fraction(fA[0]), Fraction(fB[0])
    prev = list(u) if up is None else [Fraction(x) for x in up]
    n0 = 0
    while n0 < T:
        steps = min(S, T - n0)
        nu = [None] * nx
        nprev = [None] * nx
        for i in range(N):
            b0, b1 = i * nx // N, (i + 1) * nx // N
            L, R = max(b0 - el, 0), min(b1 - 1 + er, nx - 1)
            cu = {j: u[j] for j in range(L, R + 1)}
            cp = {j: prev[j] for j in range(L, R + 1)}
            for s in range(steps):
                n = n0 + s
                new = {}
                for j in range(L, R + 1):
                    if j == 0:
                        new[j] = Fraction(fA[n + 1])
                    elif j == nx - 1:
                        new[j] = Fraction(fB[n + 1])
                    else:
                        left = cu[j + 1] if j == L else cu[j - 1]
                        right = cu[j - 1] if j == R else cu[j + 1]
                        new[j] = c2 * (left + right) + k * cu[j] - cp[j]
                for j, smp in sources:
                    if 0 < j < nx - 1 and L <= j <= R:
                        new[j] += Fraction(smp[n + 1])
                cp, cu = cu, new
            for j in range(b0, b1):
                nu[j] = cu[j]
                nprev[j] = cp[j]
        u, prev = nu, nprev
        n0 += steps
    return u, prev


def tangent_dc2(nx, T, c2, fA, fB, jr, wbar):
    """Exact d/dc2 of sum_n wbar[n] u^n_{jr} by forward-mode differentiation of
    the leapfrog with k = 2 - 2 c2 (dual numbers in rationals)."""
    u = [Fraction(0)] * nx
    u[0], u[-1] = Fraction(fA[0]), Fraction(fB[0])
    du = [Fraction(0)] * nx
    prev, dprev = list(u), list(du)
    k = 2 - 2 * c2
    total = wbar[0] * du[jr]
    for n in range(T):
        new = [Fraction(0)] * nx
        dnew = [Fraction(0)] * nx
        for j in range(1, nx - 1):
            new[j] = c2 * (u[j - 1] + u[j + 1]) + k * u[j] - prev[j]
            dnew[j] = ((u[j - 1] + u[j + 1]) - 2 * u[j]) + c2 * (du[j - 1] + du[j + 1]) + k * du[j] - dprev[j]
        new[0], new[-1] = Fraction(fA[n + 1]), Fraction(fB[n + 1])
        prev, u = u, new
        dprev, du = du, dnew
        total += wbar[n + 1] * du[jr]
    return total
