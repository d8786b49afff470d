"""Pins of the CPU oracle against things other than itself.

Each test checks the oracle against a closed form, an exact rational brute
force, a conservation law, or a structural property that the mathematics or
the paper fixes, chosen so that a dropped term, a wrong sign, a wrong index or
a swapped operand in the oracle fails at least one of them.
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np
import pytest

from paper_2203_10477_gb300 import inputs
from tests import rational_ref as rr

CAN, INC = 0, 1


def bump(T, width=40):
    """A smooth boundary pulse that is exactly 0 at t = 0 (and after `width`)."""
    n = np.arange(T + 1)
    f = np.where(n < width, np.sin(np.pi * n / width) ** 2, 0.0)
    f[0] = 0.0
    return f


def dalembert_cfl1(nx, T, fA):
    """Leapfrog at Courant number 1 with u(1,t) = 0 reproduces d'Alembert's
    solution with image reflections exactly on the grid (M = nx - 1):
        u_j^n = sum_{m>=0} [F(n - 2mM - j) - F(n - 2(m+1)M + j)],
    F(s) = fA[s] for s >= 0 and 0 for s < 0 (fA[0] must be 0)."""
    M = nx - 1

    def F(s):
        return fA[s] if s >= 0 else 0.0

    u = np.zeros(nx)
    for j in range(nx):
        tot = 0.0
        m = 0
        while n_ok(T, m, M):
            tot += F(T - 2 * m * M - j) - F(T - 2 * (m + 1) * M + j)
            m += 1
        u[j] = tot
    return u


def n_ok(T, m, M):
    return T - 2 * m * M + M >= 0


# ----------------------------------------------------------------------------
# closed forms
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("form", [CAN, INC])
def test_cfl1_equals_dalembert_with_reflections(oracle_mod, form):
    nx, T = 101, 450  # four reflections off x = 1 and x = 0
    dt = 1.0 / (nx - 1)  # a = 1, c = 1 exactly
    fA = bump(T)
    assert fA[0] == 0.0
    out = oracle_mod.leapfrog(nx, T, 1.0, dt, fA, np.zeros(T + 1), form=form)
    assert out["coeffs"].c == 1.0
    ref = dalembert_cfl1(nx, T, fA)
    assert np.abs(ref).max() > 0.5
    np.testing.assert_allclose(out["u"], ref, rtol=0, atol=1e-13)
    # the previous level as well (canonical form stores it)
    if form == CAN:
        np.testing.assert_allclose(out["w"], dalembert_cfl1(nx, T - 1, fA), rtol=0, atol=1e-13)


def test_cfl1_receiver_trace_is_delayed_boundary(oracle_mod):
    """Before the first reflection the trace at j is fA delayed by j steps."""
    nx, T, j = 401, 300, 37
    dt = 1.0 / (nx - 1)
    fA = bump(T, 60)
    out = oracle_mod.leapfrog(nx, T, 1.0, dt, fA, np.zeros(T + 1), rec_j=[j])
    expect = np.concatenate([np.zeros(j), fA[: T + 1 - j]])
    np.testing.assert_allclose(out["rec"][0], expect, rtol=0, atol=1e-14)


def exact_continuous(x, t, f, L=1.0, a=1.0, terms=8):
    """d'Alembert with images for u(0,t) = f(t), u(L,t) = 0, zero initial data."""
    tot = np.zeros_like(x)
    for m in range(terms):
        tot += f(t - (x + 2 * m * L) / a) - f(t - (2 * (m + 1) * L - x) / a)
    return tot


def test_second_order_convergence_at_cfl_half(oracle_mod):
    def f(t):
        t = np.asarray(t, dtype=float)
        # a Gaussian pulse centred 6 sigma after t = 0 (f(0) ~ 2e-16: smooth start)
        return np.where(t > 0, np.exp(-(((t - 0.3) / 0.05) ** 2)), 0.0)

    t_end = 0.7
    errs = []
    for nx in (101, 201, 401, 801):
        dx = 1.0 / (nx - 1)
        dt = 0.5 * dx
        T = int(round(t_end / dt))
        fA = f(np.arange(T + 1) * dt)
        out = oracle_mod.leapfrog(nx, T, 1.0, dt, fA, np.zeros(T + 1))
        x = np.linspace(0, 1, nx)
        errs.append(np.abs(out["u"] - exact_continuous(x, T * dt, f)).max())
    ratios = [errs[i] / errs[i + 1] for i in range(len(errs) - 1)]
    assert all(3.6 < r < 4.4 for r in ratios[1:]), (errs, ratios)


# ----------------------------------------------------------------------------
# exact rational brute force
# ----------------------------------------------------------------------------

def _tiny_case(seed, nx=23, T=37):
    r = inputs.rng(seed)
    fA = np.round(r.standard_normal(T + 1) * 8) / 8  # dyadic samples: exact in binary
    fB = np.round(r.standard_normal(T + 1) * 8) / 8
    return nx, T, fA, fB


@pytest.mark.parametrize("seed", [1, 2, 3])
@pytest.mark.parametrize("form", [CAN, INC])
def test_oracle_within_rounding_of_exact_rationals(oracle_mod, seed, form):
    nx, T, fA, fB = _tiny_case(seed)
    dt = 0.6 / (nx - 1)
    cf = oracle_mod.coeffs(0.0, 1.0, 1.0, nx, dt)
    c2 = Fraction(cf.c2)
    k = Fraction(cf.k) if form == CAN else 2 - 2 * c2
    levels = rr.leapfrog(nx, T, c2, k, fA, fB)
    exact = np.array([float(v) for v in levels[-1]])
    out = oracle_mod.leapfrog(nx, T, 1.0, dt, fA, fB, form=form)
    scale = max(1.0, np.abs(exact).max())
    assert np.abs(out["u"] - exact).max() <= 1e-12 * scale
    # second state component
    if form == CAN:
        prev = np.array([float(v) for v in levels[-2]])
        assert np.abs(out["w"] - prev).max() <= 1e-12 * scale
    else:
        v = np.array([float(a - b) for a, b in zip(levels[-1], levels[-2])])
        assert np.abs(out["w"] - v).max() <= 1e-12 * scale


@pytest.mark.parametrize("N,ov", [(2, 4), (3, 6), (4, 5), (3, 8)])
def test_rswr_mask_exact_in_rationals_and_tight(N, ov):
    """Decomposition + Prediction Validation + Global Span theorems (Sec. 2.2,
    2.4, 3) on the discrete scheme: with S <= floor(ov/2) the combined RSWR
    state equals the monolithic state exactly; S = floor(ov/2) + 1 does not."""
    nx, T, fA, fB = _tiny_case(7 + N + ov, nx=31, T=29)
    c2 = Fraction(9, 25)
    k = 2 - 2 * c2
    mono = rr.leapfrog(nx, T, c2, k, fA, fB)
    S = ov // 2
    u, prev = rr.rswr_mask(nx, T, c2, k, fA, fB, N, ov, S)
    assert u == mono[-1] and prev == mono[-2]
    u_bad, _ = rr.rswr_mask(nx, T, c2, k, fA, fB, N, ov, S + 1)
    assert u_bad != mono[-1]


def test_tangent_linear_matches_oracle_adjoint_dc2(oracle_mod):
    """d/dc2 of a linear functional of the receiver trace: exact forward-mode
    differentiation in rationals vs the oracle's discrete adjoint."""
    nx, T, fA, fB = _tiny_case(11, nx=19, T=33)
    fB = np.zeros(T + 1)
    dt = 0.7 / (nx - 1)
    cf = oracle_mod.coeffs(0.0, 1.0, 1.0, nx, dt)
    r = inputs.rng(12)
    wbar = np.round(r.standard_normal(T + 1) * 4) / 4
    jr = 9
    exact = rr.tangent_dc2(nx, T, Fraction(cf.c2), fA, fB, jr, [Fraction(x) for x in wbar])
    g = oracle_mod.adjoint(nx, T, 1.0, dt, fA, fB, jr, wbar)
    assert abs(g["dc2"] - float(exact)) <= 1e-11 * max(1.0, g["abs_dc2"])


# ----------------------------------------------------------------------------
# structural properties
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("form", [CAN, INC])
def test_sine_mode_started_at_rest(oracle_mod, form):
    """sin(k pi x) is an eigenvector of the discrete Dirichlet Laplacian with
    eigenvalue -4 sin^2(k pi dx / 2)/dx^2, so from rest (u^{-1} = u^0) the
    leapfrog gives u^n = u^0 cos((n + 1/2) th) / cos(th/2) exactly, where
    cos th = 1 - 2 c^2 sin^2(k pi dx / 2)."""
    nx, T, c = 201, 333, 0.83
    dt = c / (nx - 1)
    x = np.linspace(0.0, 1.0, nx)
    for kk in (1, 5, 40):
        u0 = np.sin(kk * np.pi * x)
        u0[0] = u0[-1] = 0.0
        z = np.zeros(T + 1)
        out = oracle_mod.leapfrog(nx, T, 1.0, dt, z, z, q0=u0, form=form, rec_j=[37])
        th = 2.0 * np.arcsin(c * np.sin(kk * np.pi / (nx - 1) / 2))  # cos th = 1 - 2 c^2 sin^2(.)
        n = np.arange(T + 1)
        np.testing.assert_allclose(out["u"], u0 * np.cos((T + 0.5) * th) / np.cos(th / 2), rtol=0, atol=1e-12)
        np.testing.assert_allclose(out["rec"][0], u0[37] * np.cos((n + 0.5) * th) / np.cos(th / 2), rtol=0, atol=1e-12)


def test_discrete_energy_is_conserved(oracle_mod):
    """With u = 0 on both ends the leapfrog conserves
    E^{n+1/2} = ||u^{n+1} - u^n||^2 + c^2 <D u^{n+1}, D u^n>  (D = forward difference)."""
    nx = 257
    dt = 0.8 / (nx - 1)
    u0 = inputs.smooth_random_state(nx, seed=3)
    z = lambda T: np.zeros(T + 1)

    def energy(T):
        out = oracle_mod.leapfrog(nx, T, 1.0, dt, z(T), z(T), q0=u0, q1=u0)
        un, up = out["u"], out["w"]
        c2 = out["coeffs"].c2
        return np.sum((un - up) ** 2) + c2 * np.sum(np.diff(un) * np.diff(up))

    E = [energy(T) for T in (1, 17, 400, 1300)]
    assert E[0] > 1e-3
    np.testing.assert_allclose(E, E[0], rtol=1e-12)


def test_light_cone_and_causal_truncation(oracle_mod):
    """Zero initial data, quiet right end: u_j^n = 0 exactly for j > n, so a
    grid truncated to T + 2 points reproduces the full grid bit for bit."""
    nx, T = 3000, 700
    dt = 0.9 / (nx - 1)
    fA = inputs.gaussian_pulse(T, dt, sigma_steps=20)
    full = oracle_mod.leapfrog(nx, T, 1.0, dt, fA, np.zeros(T + 1), rec_j=[350])
    assert np.all(full["u"][T + 1:] == 0.0)
    assert full["u"][T] != 0.0
    n_run = oracle_mod.causal_extent(T, nx)
    cut = oracle_mod.leapfrog(nx, T, 1.0, dt, fA, np.zeros(T + 1), rec_j=[350], nx_run=n_run)
    assert np.array_equal(cut["u"], full["u"][:n_run])
    assert np.array_equal(cut["w"], full["w"][:n_run])
    assert np.array_equal(cut["rec"], full["rec"])


def test_forms_agree_in_fp64(oracle_mod):
    p = inputs.c1()
    a = oracle_mod.leapfrog(p.nx, p.T, p.a, p.dt, p.fA, p.fB, form=CAN)
    b = oracle_mod.leapfrog(p.nx, p.T, p.a, p.dt, p.fA, p.fB, form=INC)
    assert np.abs(a["u"] - b["u"]).max() <= 1e-12 * np.abs(a["u"]).max()
    assert np.abs(a["u"] - b["u"]).max() > 0  # they are different operation orders


def test_fp32_increment_form_within_1e5_of_fp64(oracle_mod):
    nx, T = 6000, 5000
    dt = 0.9 / (nx - 1)
    fA = inputs.gaussian_pulse(T, dt)
    ref = oracle_mod.leapfrog(nx, T, 1.0, dt, fA, np.zeros(T + 1))
    f32 = oracle_mod.leapfrog(nx, T, 1.0, dt, fA, np.zeros(T + 1), form=INC, prec="f32")
    err = np.abs(f32["u"].astype(np.float64) - ref["u"]).max() / np.abs(ref["u"]).max()
    assert err <= 1e-5, err


def test_t0_returns_initial_state(oracle_mod):
    nx = 40
    u0 = inputs.smooth_random_state(nx, seed=5)
    f = np.array([0.25])
    out = oracle_mod.leapfrog(nx, 0, 1.0, 0.5 / (nx - 1), f, f * 0, q0=u0)
    expect = u0.copy()
    expect[0], expect[-1] = 0.25, 0.0
    assert np.array_equal(out["u"], expect)
    assert np.array_equal(out["w"], expect)  # canonical: at rest, u^{-1} = u^0


# ----------------------------------------------------------------------------
# RSWR invariants on the oracle
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("form", [CAN, INC])
@pytest.mark.parametrize("nx,N,ov,T,S", [
    (1001, 2, 16, 300, None),
    (1001, 2, 16, 300, 5),
    (997, 7, 10, 211, None),
    (640, 10, 15, 173, None),
    (515, 1, 8, 97, None),
])
def test_rswr_mask_equals_monolithic_bitwise(oracle_mod, prec, form, nx, N, ov, T, S):
    dt = 0.7 / (nx - 1)
    fA = inputs.ramped_sine(T, dt, freq=20.0)
    fB = 0.3 * inputs.ramped_sine(T, dt, freq=11.0)
    q0 = inputs.smooth_random_state(nx, seed=nx)
    mono = oracle_mod.leapfrog(nx, T, 1.0, dt, fA, fB, form=form, prec=prec, q0=q0)
    rs = oracle_mod.rswr_mask(nx, T, 1.0, dt, fA, fB, N, ov, S=S, form=form, prec=prec, q0=q0)
    assert np.array_equal(rs["u"], mono["u"])
    assert np.array_equal(rs["w"], mono["w"])


def test_rswr_mask_too_long_span_differs(oracle_mod):
    nx, N, ov, T = 1001, 4, 16, 300
    dt = 0.7 / (nx - 1)
    q0 = inputs.smooth_random_state(nx, seed=9)
    z = np.zeros(T + 1)
    mono = oracle_mod.leapfrog(nx, T, 1.0, dt, z, z, q0=q0)
    bad = oracle_mod.rswr_mask(nx, T, 1.0, dt, z, z, N, ov, S=ov // 2 + 1, q0=q0)
    assert not np.array_equal(bad["u"], mono["u"])


def test_rswr_output_waveforms_equal_true_fluxes(oracle_mod):
    """Prediction Validation Theorem (Sec. 2.4): within the span the predicted
    boundary output waveforms are the true ones."""
    nx, N, ov, T = 801, 5, 12, 260
    dt = 0.8 / (nx - 1)
    q0 = inputs.smooth_random_state(nx, seed=4)
    fA = inputs.ramped_sine(T, dt, freq=9.0)
    z = np.zeros(T + 1)
    rs = oracle_mod.rswr_mask(nx, T, 1.0, dt, fA, z, N, ov, q0=q0)
    el, er = (ov + 1) // 2, ov // 2
    pts = []
    for i in range(N - 1):
        b1 = (i + 1) * nx // N
        pts += [b1 - el, b1 - 1 + er]
    mono = oracle_mod.leapfrog(nx, T, 1.0, dt, fA, z, q0=q0, flux_j=pts)
    assert np.array_equal(rs["traces"].reshape(-1, T + 1), mono["flux"])
    assert np.abs(mono["flux"]).max() > 1.0


@pytest.mark.parametrize("N,ov,cfl", [(2, 16, 0.5), (10, 16, 0.5), (4, 24, 0.9), (3, 9, 0.7)])
def test_rswr_paper_literal_matches_monolithic(oracle_mod, N, ov, cfl):
    nx, T = 1001, 600
    dt = cfl / (nx - 1)
    fA = inputs.ramped_sine(T, dt, freq=7.0)
    z = np.zeros(T + 1)
    mono = oracle_mod.leapfrog(nx, T, 1.0, dt, fA, z)
    pl = oracle_mod.rswr_paper(nx, T, 1.0, dt, fA, z, N, ov)
    scale = np.abs(mono["u"]).max()
    assert np.abs(pl["u"] - mono["u"]).max() <= 1e-12 * scale
    cap = math.ceil((ov - 1) / (2 * pl["coeffs"].c)) - 1
    assert pl["spans"].sum() == T
    assert pl["spans"].max() <= cap and pl["spans"].min() >= 1


# ----------------------------------------------------------------------------
# the paper-literal select and the beta rule (Sec. 2.4, Sec. 3, Sec. 2.6)
# ----------------------------------------------------------------------------

def delayed_pulse(T, delay, width=8):
    """A boundary pulse with dyadic samples (sin^2 rounded to 1/64), silent
    for the first `delay` steps."""
    m = np.arange(T + 1) - delay
    return np.where((m > 0) & (m < width), np.round(np.sin(np.pi * m / width) ** 2 * 64) / 64, 0.0)


# nx, N, ov, Courant number, T, pulse delay, first predictive span (0 = ov)
PAPER_SELECT_CASES = {
    "select binds below the cap": (33, 2, 8, 0.5, 60, 0, 0),
    "far below the cap": (40, 3, 8, 0.3, 70, 0, 0),
    "pairs differ": (41, 3, 10, 0.6, 80, 0, 0),
    "quiet start grows by beta, then binds": (41, 4, 8, 0.5, 60, 25, 2),
    "growth past the first pair's cap": (41, 3, 12, 0.5, 70, 20, 2),
    "the theorem cap binds": (29, 2, 6, 0.9, 50, 0, 0),
}


@pytest.mark.parametrize("name", list(PAPER_SELECT_CASES))
def test_paper_literal_select_equals_exact_restatement(oracle_mod, name):
    """The oracle's data-chosen spans are those of an exact-rational run of
    the paper's predict / select / update loop (tests/rational_ref.py), and
    with those spans the paper-literal method reproduces the monolithic
    solution exactly in rationals (Sec. 2.4: the selected span is valid)."""
    nx, N, ov, cfl, T, delay, tau0 = PAPER_SELECT_CASES[name]
    dt = cfl / (nx - 1)
    fA = delayed_pulse(T, delay)
    z = np.zeros(T + 1)
    cf = oracle_mod.coeffs(0.0, 1.0, 1.0, nx, dt)
    u, up, spans = rr.rswr_paper(nx, T, cf.c, cf.c2, cf.k, cf.dx, fA, z, N, ov, tau0=tau0 or None)
    mono = rr.leapfrog(nx, T, Fraction(cf.c2), Fraction(cf.k), fA, z)
    assert u == mono[-1] and up == mono[-2]
    got = oracle_mod.rswr_paper(nx, T, 1.0, dt, fA, z, N, ov, tau0=tau0)
    assert list(got["spans"]) == spans
    ex = np.array([float(v) for v in u])
    assert np.abs(got["u"] - ex).max() <= 1e-12 * np.abs(ex).max()


def test_paper_select_cases_cover_binding_growth_and_cap(oracle_mod):
    """The cases above are chosen so that each part of the select rule
    decides some span: the agreement test below the theorem cap, the minimum
    over several pairs, the beta growth from a small first span, the cap."""
    seen = {"below cap": False, "grows": False, "cap": False, "pair min": False}
    for nx, N, ov, cfl, T, delay, tau0 in PAPER_SELECT_CASES.values():
        dt = cfl / (nx - 1)
        cf = oracle_mod.coeffs(0.0, 1.0, 1.0, nx, dt)
        cap = math.ceil((ov - 1) / (2 * cf.c)) - 1
        spans = list(oracle_mod.rswr_paper(nx, T, 1.0, dt, delayed_pulse(T, delay), np.zeros(T + 1), N, ov,
                                           tau0=tau0)["spans"])
        full = spans[:-1]  # the last span may be cut by T
        seen["below cap"] |= any(s < cap for s in full)
        seen["cap"] |= cap in full
        seen["grows"] |= any(b > a for a, b in zip(full, full[1:]))
        rec = []
        rr.rswr_paper(nx, T, cf.c, cf.c2, cf.k, cf.dx, delayed_pulse(T, delay), np.zeros(T + 1), N, ov,
                      tau0=tau0 or None, record=rec)
        # a span decided by one pair while another pair would allow more
        seen["pair min"] |= any(min(p) < min(max(p), steps, cap) for _, steps, p in rec)
    assert all(seen.values()), seen


def test_paper_beta_rule_is_exact(oracle_mod):
    """Sec. 2.6: the next predictive span is (1 + beta) times the selected one
    (beta = 0.1), rounded up.  On a quiet grid the agreement never binds, so
    the spans are the predictive spans under the theorem cap: from a first
    span of 50 steps the next is ceil(55.0) = 55 (a floating-point 1.1 * 50
    rounds above 55 and would give 56), then the cap
    ceil((ov - 1)/(2c)) - 1 = ceil(59/1) - 1 = 58."""
    nx, N, ov, T = 121, 2, 60, 163
    dt = 0.5 / (nx - 1)
    z = np.zeros(T + 1)
    got = oracle_mod.rswr_paper(nx, T, 1.0, dt, z, z, N, ov, tau0=50)
    assert list(got["spans"]) == [50, 55, 58]


def test_paper_literal_cfl1_spans_from_the_cone(oracle_mod):
    """Hand-derived span sequence at Courant number 1.

    With c = 1 the leapfrog carries u^n_j = F(n - j) exactly (d'Alembert).
    Take the ramp F(s) = s/8 for s >= 1 entering at x = 0, N = 2, ov = 16 on
    nx = 65 (dx = 1/64: every value and flux is exact in binary), so the
    overlap is [L, R] = [24, 39] and the theorem cap is the largest integer
    below (ov - 1)/2, i.e. 7.  A zero-flux ghost at an interior end e first
    differs from the truth at the level after the front reaches e (level
    max(n0, e) + 1), and at c = 1 that error travels exactly one point per
    step with an unchanged leading value, so at overlap point x the
    predictions of a span starting at n0 first differ at level
        min(max(n0, R) + 1 + (R - x), max(n0, L) + 1 + (x - L)).
    The agreement at x is that level minus n0 + 1 (clipped to the span), the
    span is its maximum over x, capped by 7, and the first predictive span is
    3, so the spans grow by beta (3, 4, 5, 6, 7) and then stay at the cap.
    The final state is d'Alembert's F(T - j), bit for bit."""
    nx, N, ov, T, tau0 = 65, 2, 16, 60, 3
    dt = 1.0 / (nx - 1)
    F = lambda s: s / 8.0 if s >= 1 else 0.0
    fA = np.array([F(n) for n in range(T + 1)])
    z = np.zeros(T + 1)
    L, R, cap = 24, 39, 7
    expect, n0, tau = [], 0, tau0
    while n0 < T:
        steps = min(tau, T - n0)
        best = 0
        for x in range(L, R + 1):
            first = min(max(n0, R) + 1 + (R - x), max(n0, L) + 1 + (x - L))
            best = max(best, min(first - n0 - 1, steps))
        span = max(1, min(best, steps, cap))
        expect.append(span)
        n0 += span
        tau = -(-11 * span // 10)
    assert expect[:6] == [3, 4, 5, 6, 7, 7] and sum(expect) == T
    got = oracle_mod.rswr_paper(nx, T, 1.0, dt, fA, z, N, ov, tau0=tau0)
    assert got["coeffs"].c == 1.0
    assert list(got["spans"]) == expect
    assert np.array_equal(got["u"], np.array([F(T - j) for j in range(nx)]))


# ----------------------------------------------------------------------------
# adjoint
# ----------------------------------------------------------------------------

def _adj_case(nx=301, T=420, jr=120):
    dt = 0.9 / (nx - 1) / 1.3  # Courant number 0.9 at a = 1.3
    g = inputs.lowpass_noise(T, seed=21)
    return nx, T, dt, g, jr


def test_adjoint_dot_product(oracle_mod):
    nx, T, dt, g, jr = _adj_case()
    z = np.zeros(T + 1)
    r = inputs.rng(3)
    dgv = r.standard_normal(T + 1)
    w = r.standard_normal(T + 1)
    Jdg = oracle_mod.leapfrog(nx, T, 1.3, dt, dgv, z, rec_j=[jr])["rec"][0]
    JTw = oracle_mod.adjoint(nx, T, 1.3, dt, g, z, jr, w)["dg"]
    lhs, rhs = np.dot(Jdg, w), np.dot(dgv, JTw)
    assert abs(lhs - rhs) <= 1e-13 * max(abs(lhs), np.abs(Jdg * w).sum())


def test_adjoint_gradient_g_matches_central_difference(oracle_mod):
    nx, T, dt, g, jr = _adj_case()
    z = np.zeros(T + 1)
    target = oracle_mod.leapfrog(nx, T, 1.0, dt, g, z, rec_j=[jr])["rec"][0]
    res = oracle_mod.misfit_grad(nx, T, 1.3, dt, g, z, jr, target)
    d = inputs.rng(8).standard_normal(T + 1)
    for h in (1e-2, 1.0):  # the loss is quadratic in g: exact for any h
        lp = oracle_mod.misfit_grad(nx, T, 1.3, dt, g + h * d, z, jr, target)["loss"]
        lm = oracle_mod.misfit_grad(nx, T, 1.3, dt, g - h * d, z, jr, target)["loss"]
        fd = (lp - lm) / (2 * h)
        an = np.dot(res["dg"], d)
        assert abs(fd - an) <= 1e-8 * abs(an), (h, fd, an)


def test_adjoint_gradient_a_matches_central_difference(oracle_mod):
    """Central differences in a converge to the adjoint dL/da at O(h^2)."""
    nx, T, dt, g, jr = _adj_case()
    z = np.zeros(T + 1)
    target = oracle_mod.leapfrog(nx, T, 1.0, dt, g, z, rec_j=[jr])["rec"][0]
    a = 1.3
    res = oracle_mod.misfit_grad(nx, T, a, dt, g, z, jr, target)
    errs = []
    for rel in (1e-4, 1e-5, 1e-6):
        h = rel * a
        lp = oracle_mod.misfit_grad(nx, T, a + h, dt, g, z, jr, target)["loss"]
        lm = oracle_mod.misfit_grad(nx, T, a - h, dt, g, z, jr, target)["loss"]
        errs.append(abs((lp - lm) / (2 * h) - res["da"]) / abs(res["da"]))
    assert 80 < errs[0] / errs[1] < 120, errs  # second order in h
    assert errs[2] < 1e-8, errs


def test_adjoint_boundary_receiver_and_unreachable_receiver(oracle_mod):
    nx, T, dt, g, _ = _adj_case(T=100)
    z = np.zeros(T + 1)
    w = inputs.rng(2).standard_normal(T + 1)
    # receiver on the Dirichlet node: the trace is g itself, so dL/dg = wbar and dL/da = 0
    res = oracle_mod.adjoint(nx, T, 1.3, dt, g, z, 0, w)
    assert np.array_equal(res["dg"], w)
    assert res["dc2"] == 0.0
    # receiver beyond the reach of T steps: every gradient is exactly zero
    res = oracle_mod.adjoint(nx, T, 1.3, dt, g, z, T + 5, w)
    assert np.all(res["dg"] == 0.0) and res["dc2"] == 0.0


def test_adjoint_causal_truncation_is_exact(oracle_mod):
    nx, T, jr = 5000, 300, 140
    dt = 0.9 / (nx - 1) / 1.3
    g = inputs.lowpass_noise(T, seed=4)
    z = np.zeros(T + 1)
    w = inputs.rng(5).standard_normal(T + 1)
    full = oracle_mod.adjoint(nx, T, 1.3, dt, g, z, jr, w)
    cut = oracle_mod.adjoint(nx, T, 1.3, dt, g, z, jr, w, nx_run=oracle_mod.causal_extent(T, nx))
    assert np.array_equal(full["dg"], cut["dg"])
    assert full["dc2"] == cut["dc2"]


def test_source_driven_leapfrog_is_the_adjoint_sweep(oracle_mod):
    """The adjoint variables in reversed time are the leapfrog from rest with
    zero Dirichlet data and the source wbar[T+1-m] at j_r: its samples at j = 1
    times c2 are dL/dfA, equal to the oracle's discrete adjoint bit for bit."""
    nx, T, jr = 301, 420, 120
    dt = 0.9 / (nx - 1) / 1.3
    g = inputs.lowpass_noise(T, seed=21)
    z = np.zeros(T + 1)
    w = inputs.rng(3).standard_normal(T + 1)
    adj = oracle_mod.adjoint(nx, T, 1.3, dt, g, z, jr, w)
    src = np.concatenate([[0.0], w[::-1]])  # level m of the reversed run gets wbar[T+1-m]
    zz = np.zeros(T + 2)
    lam = oracle_mod.leapfrog(nx, T + 1, 1.3, dt, zz, zz, rec_j=[1], src_j=jr, src=src)
    c2 = adj["coeffs"].c2
    dg = np.array([c2 * lam["rec"][0][T - n] for n in range(T + 1)])
    assert np.array_equal(dg[:T], adj["dg"][:T])
    assert dg[T] == 0.0 and adj["dg"][T] == 0.0


# ----------------------------------------------------------------------------
# interior point sources (the paper's pulse sources, Sec. 4)
# ----------------------------------------------------------------------------

def lattice_light_cone(nx, T, sources):
    """Closed form of the leapfrog at Courant number 1 far from the boundaries:
    a unit impulse joining level m at point j0 is, at level n >= m, 1 at every j
    with |j - j0| <= n - m and j - j0 = n - m (mod 2), 0 elsewhere (the lattice
    d'Alembert solution: it spreads one cell per step in a checkerboard).  A
    source with samples s^m superposes s^m times that pattern."""
    u = np.zeros(nx)
    for j0, smp in sources:
        for m in range(1, T + 1):
            if smp[m] == 0:
                continue
            t = T - m
            for d in range(-t, t + 1, 2):
                u[j0 + d] += smp[m]
    return u


@pytest.mark.parametrize("form", [CAN, INC])
def test_sources_at_cfl1_form_lattice_light_cones(oracle_mod, form):
    nx, T = 301, 80
    dt = 1.0 / (nx - 1)  # Courant number 1
    r = np.random.default_rng(5)
    sources = []
    for j0 in (100, 150, 150, 201):  # two sources share a point
        smp = np.zeros(T + 1)
        smp[1:] = r.integers(-3, 4, size=T)
        sources.append((j0, smp))
    z = np.zeros(T + 1)
    out = oracle_mod.leapfrog(nx, T, 1.0, dt, z, z, form=form, src_j=[j for j, _ in sources],
                              src=np.stack([s for _, s in sources]))
    assert np.array_equal(out["u"], lattice_light_cone(nx, T, sources))


@pytest.mark.parametrize("N,ov", [(2, 4), (3, 6), (4, 5)])
def test_rswr_with_sources_exact_in_rationals_and_tight(N, ov):
    """With point sources inside windows, in halos and on core boundaries the
    combined RSWR state still equals the monolithic state exactly for
    S <= floor(ov/2) (the sources are local; the discrete domain of dependence
    is unchanged), and S = floor(ov/2) + 1 still breaks it."""
    nx, T, fA, fB = _tiny_case(40 + N + ov, nx=31, T=29)
    c2 = Fraction(9, 25)
    k = 2 - 2 * c2
    r = np.random.default_rng(N * 10 + ov)
    b1 = nx // N
    pts = sorted({2, b1 - 1, b1, b1 + 1, nx - 3})
    sources = [(j, np.concatenate([[0.0], np.round(r.standard_normal(T) * 4) / 4])) for j in pts]
    mono = rr.leapfrog(nx, T, c2, k, fA, fB, sources=sources)
    u, prev = rr.rswr_mask(nx, T, c2, k, fA, fB, N, ov, ov // 2, sources=sources)
    assert u == mono[-1] and prev == mono[-2]
    u_bad, _ = rr.rswr_mask(nx, T, c2, k, fA, fB, N, ov, ov // 2 + 1, sources=sources)
    assert u_bad != mono[-1]


@pytest.mark.parametrize("form", [CAN, INC])
def test_oracle_sources_within_rounding_of_exact_rationals(oracle_mod, form):
    nx, T, fA, fB = _tiny_case(17, nx=41, T=37)
    dt = 0.6 / (nx - 1)
    cf = oracle_mod.coeffs(0.0, 1.0, 1.0, nx, dt)
    c2 = Fraction(cf.c2)
    k = Fraction(cf.k) if form == CAN else 2 - 2 * c2
    r = np.random.default_rng(3)
    pts = [5, 20, 20, 33]
    smp = np.zeros((len(pts), T + 1))
    smp[:, 1:] = np.round(r.standard_normal((len(pts), T)) * 8) / 8
    levels = rr.leapfrog(nx, T, c2, k, fA, fB, sources=list(zip(pts, smp)))
    exact = np.array([float(v) for v in levels[-1]])
    out = oracle_mod.leapfrog(nx, T, 1.0, dt, fA, fB, form=form, src_j=pts, src=smp)
    assert np.abs(out["u"] - exact).max() <= 1e-12 * max(1.0, np.abs(exact).max())


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("form", [CAN, INC])
def test_rswr_mask_with_sources_equals_monolithic_bitwise(oracle_mod, prec, form):
    nx, N, ov, T = 1001, 10, 16, 300
    dt = 0.8 / (nx - 1)
    fA = inputs.ramped_sine(T, dt, freq=9.0)
    z = np.zeros(T + 1)
    pts = [50, 99, 100, 107, 450, 450, 951, 998]  # inside cores, on core edges, in halos, shared, near j = nx-1
    src = np.stack([inputs.gaussian_pulse(T, dt, sigma_steps=10 + 3 * i) * (1 + i) for i in range(len(pts))])
    mono = oracle_mod.leapfrog(nx, T, 1.0, dt, fA, z, form=form, prec=prec, src_j=pts, src=src)
    rs = oracle_mod.rswr_mask(nx, T, 1.0, dt, fA, z, N, ov, form=form, prec=prec, src_j=pts, src=src)
    assert np.abs(mono["u"]).max() > 0.1
    assert np.array_equal(rs["u"], mono["u"])
    assert np.array_equal(rs["w"], mono["w"])


# ----------------------------------------------------------------------------
# the threaded interior loop (the CPU timing baseline on all host cores)
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("form", [CAN, INC])
def test_threaded_leapfrog_equals_serial_bitwise(oracle_mod, form, prec):
    """The interior updates of one level are independent, so the threaded
    loop gives the serial result bit for bit (state, probes, sources)."""
    nx, T = 200_003, 40
    dt = 0.9 / (nx - 1)
    q0 = inputs.smooth_random_state(nx, seed=11)
    fA = inputs.ramped_sine(T, dt, freq=30.0)
    fB = inputs.ramped_sine(T, dt, freq=11.0)
    smp = np.stack([inputs.gaussian_pulse(T, dt, sigma_steps=4), -inputs.gaussian_pulse(T, dt, sigma_steps=6)])
    kw = dict(form=form, prec=prec, q0=q0, rec_j=[5, 100_000], flux_j=[77, 150_000], src_j=[1000, 123_456],
              src=smp)
    oracle_mod.set_threads(1)
    ser = oracle_mod.leapfrog(nx, T, 1.0, dt, fA, fB, **kw)
    oracle_mod.set_threads(4)
    try:
        par = oracle_mod.leapfrog(nx, T, 1.0, dt, fA, fB, **kw)
    finally:
        oracle_mod.set_threads(1)
    for key in ("u", "w", "rec", "flux"):
        assert np.array_equal(ser[key], par[key]), key
    assert np.abs(ser["u"]).max() > 0.1
