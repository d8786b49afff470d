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


def _ceil_frac(q):
    """Smallest integer >= the rational q."""
    q = Fraction(q)
    return -((-q.numerator) // q.denominator)


def rswr_paper(nx, T, c, c2, k, dx, fA, fB, N, ov, tau0=None, beta=Fraction(1, 10), record=None):
    """The paper's own RSWR loop in exact arithmetic (Sec. 2.3-2.6, Sec. 3).

    Each span starts from the combined (true) state pair at level n0:
      predict  every window is advanced over the predictive span with a zero
               input flux at each interior end (mirror ghost);
      select   at an overlap point x of windows i and i+1 the point span is the
               number of leading levels n0+1, n0+2, ... at which the two
               predictions are equal; a pair's span is the largest point span
               of its overlap, the global span the smallest pair span, bounded
               by the Waveform Time Span Theorem (largest whole number of
               steps below (ov - 1)/(2c), i.e. below Delta X_overlap / (2a))
               and by the predictive span itself, and at least one step;
      update   every window is solved again over the selected span, an input
               end taking the neighbour's predicted output flux
               g = (p[e+1] - p[e-1]) / (2 dx) as Neumann data
               (ghost = inner value -/+ 2 dx g);
      combine  a point takes the value of the leftmost window that holds it;
      redo     the next predictive span is ceil((1 + beta) * span) (beta = 0.1,
               Sec. 2.6), limited to ceil((1 + beta) max(tau0, cap)) + 1.
    c, c2, k, dx are the scheme's coefficients (rationals, or floats taken at
    their exact binary value).  Returns (u^T, u^{T-1}, spans).  When `record`
    is a list, (n0, steps, [span of each pair]) is appended for every span."""
    c, c2, k, dx = Fraction(c), Fraction(c2), Fraction(k), Fraction(dx)
    el, er = (ov + 1) // 2, ov // 2
    win = []
    for i in range(N):
        b0, b1 = i * nx // N, (i + 1) * nx // N
        win.append((max(b0 - el, 0), min(b1 - 1 + er, nx - 1)))
    cap = max(_ceil_frac(Fraction(ov - 1) / (2 * c)) - 1, 1)
    tau = tau0 if tau0 else ov
    tau_lim = _ceil_frac((1 + beta) * max(tau, cap)) + 1

    u = [Fraction(0)] * nx
    u[0], u[-1] = Fraction(fA[0]), Fraction(fB[0])
    prev = list(u)

    def solve(L, R, n0, steps, flux_left=None, flux_right=None):
        """Levels n0..n0+steps of window [L, R] as dicts j -> value; an
        interior end takes the ghost from the given flux per level (zero flux
        when None)."""
        cur = {j: u[j] for j in range(L, R + 1)}
        old = {j: prev[j] for j in range(L, R + 1)}
        levels = [cur]
        for s in range(steps):
            n = n0 + s
            new = {}
            for j in range(L, R + 1):
                if j == 0:
                    new[j] = Fraction(fA[n + 1])
                    continue
                if j == nx - 1:
                    new[j] = Fraction(fB[n + 1])
                    continue
                if j == L:
                    g = flux_left[s] if flux_left is not None else 0
                    west = cur[j + 1] - 2 * dx * g
                else:
                    west = cur[j - 1]
                if j == R:
                    g = flux_right[s] if flux_right is not None else 0
                    east = cur[j - 1] + 2 * dx * g
                else:
                    east = cur[j + 1]
                new[j] = c2 * (west + east) + k * cur[j] - old[j]
            old, cur = cur, new
            levels.append(cur)
        return levels

    spans = []
    n0 = 0
    while n0 < T:
        steps = min(tau, T - n0)
        pred = [solve(L, R, n0, steps) for (L, R) in win]
        pairs = []
        for i in range(N - 1):
            lo, hi = win[i + 1][0], win[i][1]  # the overlap of windows i and i+1
            pair = 0
            for x in range(lo, hi + 1):
                s = 1
                while s <= steps and pred[i][s][x] == pred[i + 1][s][x]:
                    s += 1
                pair = max(pair, s - 1)
            pairs.append(pair)
        if record is not None:
            record.append((n0, steps, pairs))
        span = max(1, min([steps, cap] + pairs))
        nu, nprev = [None] * nx, [None] * nx
        for i, (L, R) in enumerate(win):
            fl = fr = None
            if i > 0 and L > 0:
                p = pred[i - 1]
                fl = [(p[s][L + 1] - p[s][L - 1]) / (2 * dx) for s in range(span)]
            if i < N - 1 and R < nx - 1:
                p = pred[i + 1]
                fr = [(p[s][R + 1] - p[s][R - 1]) / (2 * dx) for s in range(span)]
            lv = solve(L, R, n0, span, fl, fr)
            for j in range(L, R + 1):
                if nu[j] is None:
                    nu[j], nprev[j] = lv[span][j], lv[span - 1][j]
        u, prev = nu, nprev
        spans.append(span)
        n0 += span
        tau = min(_ceil_frac((1 + beta) * span), tau_lim)
    return u, prev, spans
