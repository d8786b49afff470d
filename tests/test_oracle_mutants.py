"""The oracle's pins catch plausible mistakes.

Each mutant is a copy of the oracle's C source with one planted mistake (a
flipped sign, a dropped term, an index or time level off by one, a wrong
coefficient), built on the CPU.  A set of small checks -- closed forms, exact
rational brute force, conservation, adjoint identities, RSWR invariants, the
same kinds of pins as tests/test_oracle_pins.py -- is run against the real
oracle (all must pass) and against every mutant (at least one must fail).
"""
from __future__ import annotations

import ctypes
import functools
import os
import shutil
import subprocess
import tempfile
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2203_10477_gb300 import inputs
from tests import rational_ref as rr

SRC = os.path.dirname(os.path.abspath(oracle.__file__))

# (file, original text, planted mistake), or (file, [(original, mistake), ...])
MUTANTS = {
    "canonical: sign of the centre term": ("leapfrog_body.h", "*u_new = FMA(c2, s, t);", "*u_new = FMA(c2, s, -t);"),
    "canonical: previous level added": ("leapfrog_body.h", "REAL t = FMA(k, uC, -w);", "REAL t = FMA(k, uC, w);"),
    "canonical: neighbour dropped": ("leapfrog_body.h", "REAL s = uL + uR;", "REAL s = uL + uL;"),
    "increment: Laplacian sign": ("leapfrog_body.h", "REAL lap = (uL - uC) + (uR - uC);",
                                  "REAL lap = (uL - uC) + (uR + uC);"),
    "increment: update sign": ("leapfrog_body.h", "*u_new = uC + v;", "*u_new = uC - v;"),
    "coefficient k": ("rswr_oracle.c", "*k = 2.0 - 2.0 * (*c2);", "*k = 2.0 - (*c2);"),
    "coefficient c2": ("rswr_oracle.c", "*c2 = cc * cc;", "*c2 = cc;"),
    "Dirichlet time level": ("leapfrog_body.h", "        un[0] = fA[n + 1];\n        wn[0] = NAME(dirichlet_w)(form, fA[n], fA[n + 1]);",
                             "        un[0] = fA[n];\n        wn[0] = NAME(dirichlet_w)(form, fA[n], fA[n + 1]);"),
    "rest state": ("leapfrog_body.h", "else w[j] = (form == 0) ? u[j] : (REAL)0;",
                   "else w[j] = (form == 0) ? (REAL)0 : u[j];"),
    "RSWR core write-back": ("leapfrog_body.h", "for (int64_t j = b0; j < b1; ++j) { nu[j] = pu[j]; nw[j] = pw[j]; }",
                             "for (int64_t j = b0; j + 1 < b1; ++j) { nu[j] = pu[j]; nw[j] = pw[j]; }"),
    "RSWR window too narrow": ("leapfrog_body.h", "int64_t el = (ov + 1) / 2, er = ov / 2;",
                               "int64_t el = (ov + 1) / 2 - 1, er = ov / 2;"),
    "flux difference": ("leapfrog_body.h", "flux[r * (T + 1) + n] = (u[j + 1] - u[j - 1]) * inv2dx;",
                        "flux[r * (T + 1) + n] = (u[j + 1] - u[j]) * inv2dx;"),
    "adjoint: boundary gradient index": ("rswr_oracle.c", "dg[n] = c2 * l1[1] + ((jr == 0) ? wbar[n] : 0.0);",
                                         "dg[n] = c2 * l1[2] + ((jr == 0) ? wbar[n] : 0.0);"),
    "adjoint: second level sign": ("rswr_oracle.c", "double v = fma(c2, left + right, fma(k, l1[j], -l2[j]));",
                                   "double v = fma(c2, left + right, fma(k, l1[j], l2[j]));"),
    "adjoint: dL/dc2 Laplacian": ("rswr_oracle.c", "double term = l1[j] * ((un_[j - 1] + un_[j + 1]) - 2.0 * un_[j]);",
                                  "double term = l1[j] * ((un_[j - 1] + un_[j + 1]) - un_[j]);"),
    "adjoint: source dropped": ("rswr_oracle.c", "if (j == jr) v = v + wbar[n];", "if (j == jr) v = v;"),
    # (the LEFT ghost cannot be caught: with the combination rule of Sec. 2.5 the
    # left neighbour's values win on the overlap, so errors from a subdomain's
    # left input boundary stay in the part that is discarded)
    "paper-literal: right ghost sign": ("rswr_oracle.c",
                                        "if (j == R) uR = gR ? pu[j - 1] + 2.0 * dx * gR[s] : pu[j - 1];",
                                        "if (j == R) uR = gR ? pu[j - 1] - 2.0 * dx * gR[s] : pu[j - 1];"),
    "paper-literal: combination": ("rswr_oracle.c", "int64_t from = (i == 0) ? L : win_right(i - 1, nx, N, er) + 1;",
                                   "int64_t from = (i == 0) ? L : win_right(i - 1, nx, N, er) + 2;"),
    "source: time level": ("leapfrog_body.h", "REAL s = src[q * (T + 1) + n + 1];", "REAL s = src[q * (T + 1) + n];"),
    "source: sign": ("leapfrog_body.h", "            un[j] = un[j] + s;", "            un[j] = un[j] - s;"),
    "source: increment not applied": ("leapfrog_body.h", "            un[j] = u_old[j] + wn[j];",
                                      "            un[j] = u_old[j];"),
    # (skipping only the two window end points cannot be caught: they are the
    # guessed input boundaries, whose values never reach the kept core)
    "source: only in the window's core": ("leapfrog_body.h",
                                          "if (src && nsrc > 0) NAME(add_sources)(form, nx, T, n, nsrc, src_j, src, L, R, pu, qu, qw);",
                                          "if (src && nsrc > 0) NAME(add_sources)(form, nx, T, n, nsrc, src_j, src, b0, b1 - 1, pu, qu, qw);"),
    # the paper-literal select (Sec. 2.4, Sec. 3) and predictive span (Sec. 2.6)
    "paper-literal: agreement ignored": ("rswr_oracle.c", "if (agree > best) best = agree;", "best = steps;"),
    "paper-literal: minimum over the overlap": ("rswr_oracle.c", [("int64_t best = 0;", "int64_t best = steps;"),
                                                                  ("if (agree > best) best = agree;",
                                                                   "if (agree < best) best = agree;")]),
    "paper-literal: maximum over the pairs": ("rswr_oracle.c", [("int64_t span = steps;", "int64_t span = 0;"),
                                                                ("if (best < span) span = best;",
                                                                 "if (best > span) span = best;")]),
    "paper-literal: agreement from level 0": ("rswr_oracle.c",
                                              "p1[(agree + 1) * nx + x] == p2[(agree + 1) * nx + x]",
                                              "p1[agree * nx + x] == p2[agree * nx + x]"),
    "paper-literal: beta dropped": ("rswr_oracle.c", "tau = (span * (1000 + beta_m) + 999) / 1000;", "tau = span;"),
    "paper-literal: beta product in floating point": ("rswr_oracle.c", "tau = (span * (1000 + beta_m) + 999) / 1000;",
                                                      "tau = (int64_t)ceil((1.0 + beta) * (double)span);"),
    "paper-literal: theorem cap one step longer": ("rswr_oracle.c", "int64_t cap = (int64_t)ceil(cap_real) - 1;",
                                                   "int64_t cap = (int64_t)ceil(cap_real);"),
}


def build_variant(tmp, name, mutation):
    d = os.path.join(tmp, name.replace(" ", "_").replace(":", "").replace("/", ""))
    os.makedirs(d)
    for f in ("rswr_oracle.c", "leapfrog_body.h"):
        shutil.copy(os.path.join(SRC, f), d)
    if mutation is not None:
        f, edits = mutation[0], mutation[1:]
        if len(edits) == 2:  # one (old, new) replacement
            edits = [tuple(edits)]
        else:  # a list of them
            edits = edits[0]
        p = os.path.join(d, f)
        text = open(p).read()
        for old, new in edits:
            assert text.count(old) >= 1, f"mutation anchor not found: {old}"
            text = text.replace(old, new, 1)
        open(p, "w").write(text)
    lib = os.path.join(d, "lib.so")
    subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-o", lib,
                    os.path.join(d, "rswr_oracle.c"), "-lm"], check=True, cwd=d)
    L = ctypes.CDLL(lib)
    oracle._declare(L)
    return L


# ---- the checks (small versions of the pins) -----------------------------

def chk_dalembert():
    nx, T = 41, 150
    fA = np.where(np.arange(T + 1) < 20, np.sin(np.pi * np.arange(T + 1) / 20) ** 2, 0.0)
    out = oracle.leapfrog(nx, T, 1.0, 1.0 / (nx - 1), fA, np.zeros(T + 1))["u"]
    M = nx - 1
    F = lambda s: fA[s] if s >= 0 else 0.0
    ref = [sum(F(T - 2 * m * M - j) - F(T - 2 * (m + 1) * M + j) for m in range(T // M + 2)) for j in range(nx)]
    return np.abs(out - np.array(ref)).max() < 1e-12


def chk_rational(form):
    r = inputs.rng(4)
    nx, T = 17, 23
    fA = np.round(r.standard_normal(T + 1) * 8) / 8
    fB = np.round(r.standard_normal(T + 1) * 8) / 8
    dt = 0.6 / (nx - 1)
    cf = oracle.coeffs(0.0, 1.0, 1.0, nx, dt)
    c2 = Fraction(0.36 if False else cf.c2)
    k = Fraction(cf.k) if form == 0 else 2 - 2 * c2
    lv = rr.leapfrog(nx, T, c2, k, fA, fB)
    out = oracle.leapfrog(nx, T, 1.0, dt, fA, fB, form=form)
    ex = np.array([float(v) for v in lv[-1]])
    ok = np.abs(out["u"] - ex).max() <= 1e-12 * max(1, np.abs(ex).max())
    # the exact value of c2 itself: c = a dt / dx
    ok &= abs(cf.c - 0.6) < 1e-14 and abs(cf.c2 - 0.36) < 1e-14 and abs(cf.k - 1.28) < 1e-14
    return bool(ok)


def chk_energy():
    nx = 65
    dt = 0.8 / (nx - 1)
    u0 = inputs.smooth_random_state(nx, seed=3)
    z = lambda T: np.zeros(T + 1)

    def E(T):
        o = oracle.leapfrog(nx, T, 1.0, dt, z(T), z(T), q0=u0)
        return np.sum((o["u"] - o["w"]) ** 2) + o["coeffs"].c2 * np.sum(np.diff(o["u"]) * np.diff(o["w"]))

    return abs(E(200) - E(1)) <= 1e-12 * abs(E(1))


def chk_rswr():
    nx, N, ov, T = 301, 4, 12, 90
    dt = 0.7 / (nx - 1)
    q0 = inputs.smooth_random_state(nx, seed=8)
    fA = inputs.ramped_sine(T, dt, freq=9.0)
    z = np.zeros(T + 1)
    m = oracle.leapfrog(nx, T, 1.0, dt, fA, z, q0=q0)
    s = oracle.rswr_mask(nx, T, 1.0, dt, fA, z, N, ov, q0=q0)
    ok = np.array_equal(m["u"], s["u"]) and np.array_equal(m["w"], s["w"])
    el, er = (ov + 1) // 2, ov // 2
    pts = []
    for i in range(N - 1):
        b1 = (i + 1) * nx // N
        pts += [b1 - el, b1 - 1 + er]
    fl = oracle.leapfrog(nx, T, 1.0, dt, fA, z, q0=q0, flux_j=pts)["flux"]
    # the central difference in physical units
    j = pts[0]
    u = oracle.leapfrog(nx, 5, 1.0, dt, fA[:6], z[:6], q0=q0)["u"]
    fl5 = oracle.leapfrog(nx, 5, 1.0, dt, fA[:6], z[:6], q0=q0, flux_j=[j])["flux"][0][5]
    ok &= abs(fl5 - (u[j + 1] - u[j - 1]) / (2.0 / (nx - 1))) <= 1e-9 * max(1.0, abs(fl5))
    return bool(ok and np.array_equal(s["traces"].reshape(-1, T + 1), fl))


def chk_mode():
    """A discrete Dirichlet sine mode started at rest: u^n = u^0 cos((n + 1/2) th) / cos(th/2),
    cos th = 1 - 2 c^2 sin^2(pi dx / 2) (pins the stencil and the rest-state start)."""
    nx, T = 129, 77
    c = 0.7
    dt = c / (nx - 1)
    x = np.linspace(0.0, 1.0, nx)
    u0 = np.sin(np.pi * x)
    u0[0] = u0[-1] = 0.0
    z = np.zeros(T + 1)
    th = 2.0 * np.arcsin(c * np.sin(np.pi / (nx - 1) / 2))
    ok = True
    for form in (0, 1):
        o = oracle.leapfrog(nx, T, 1.0, dt, z, z, q0=u0, form=form)
        ok &= np.abs(o["u"] - u0 * np.cos((T + 0.5) * th) / np.cos(th / 2)).max() < 1e-12
    return bool(ok)


def chk_paper():
    nx, N, ov, T = 401, 3, 16, 600
    dt = 0.9 / (nx - 1)
    fA = inputs.ramped_sine(T, dt, freq=7.0)
    z = np.zeros(T + 1)
    m = oracle.leapfrog(nx, T, 1.0, dt, fA, z)
    p = oracle.rswr_paper(nx, T, 1.0, dt, fA, z, N, ov)
    return np.abs(p["u"] - m["u"]).max() <= 1e-12 * np.abs(m["u"]).max()


def chk_adjoint():
    nx, T, jr = 61, 90, 20
    dt = 0.9 / (nx - 1) / 1.3
    z = np.zeros(T + 1)
    r = inputs.rng(3)
    g = inputs.lowpass_noise(T, seed=2)
    dgv, w = r.standard_normal(T + 1), r.standard_normal(T + 1)
    Jd = oracle.leapfrog(nx, T, 1.3, dt, dgv, z, rec_j=[jr])["rec"][0]
    res = oracle.adjoint(nx, T, 1.3, dt, g, z, jr, w)
    ok = abs(np.dot(Jd, w) - np.dot(dgv, res["dg"])) <= 1e-12 * np.abs(Jd * w).sum()
    exact = rr.tangent_dc2(nx, T, Fraction(res["coeffs"].c2), g, z, jr, [Fraction(x) for x in w])
    ok &= abs(res["dc2"] - float(exact)) <= 1e-10 * max(1.0, res["abs_dc2"])
    return bool(ok)


def chk_sources():
    """Point sources at Courant number 1 form lattice light cones (closed form),
    in both forms; serial RSWR with sources in halos equals the monolithic solve."""
    nx, T = 201, 40
    dt = 1.0 / (nx - 1)
    z = np.zeros(T + 1)
    r = inputs.rng(6)
    pts = [60, 100, 100, 141]  # the cones stay clear of both Dirichlet nodes
    smp = np.zeros((len(pts), T + 1))
    smp[:, 1:] = r.integers(-3, 4, size=(len(pts), T))
    ref = np.zeros(nx)
    for j0, sm in zip(pts, smp):
        for m in range(1, T + 1):
            for d in range(-(T - m), T - m + 1, 2):
                ref[j0 + d] += sm[m]
    ok = True
    for form in (0, 1):
        ok &= np.array_equal(oracle.leapfrog(nx, T, 1.0, dt, z, z, form=form, src_j=pts, src=smp)["u"], ref)
    nx, N, ov, T = 301, 4, 12, 90
    dt = 0.7 / (nx - 1)
    z = np.zeros(T + 1)
    pts = [70, 74, 76, 150]  # in the first interface's overlap and halos
    smp = np.stack([inputs.gaussian_pulse(T, dt, sigma_steps=8) * (i + 1) for i in range(len(pts))])
    for form in (0, 1):
        m = oracle.leapfrog(nx, T, 1.0, dt, z, z, form=form, src_j=pts, src=smp)
        s = oracle.rswr_mask(nx, T, 1.0, dt, z, z, N, ov, form=form, src_j=pts, src=smp)
        ok &= np.array_equal(m["u"], s["u"]) and np.array_equal(m["w"], s["w"])
    return bool(ok)


@functools.lru_cache(maxsize=None)
def _paper_select_expect(nx, N, ov, cfl, T, delay, tau0):
    """Spans of the exact-rational restatement of the paper's loop."""
    dt = cfl / (nx - 1)
    cf = oracle.coeffs(0.0, 1.0, 1.0, nx, dt)
    m = np.arange(T + 1) - delay
    fA = np.where((m > 0) & (m < 8), np.round(np.sin(np.pi * m / 8) ** 2 * 64) / 64, 0.0)
    return fA, rr.rswr_paper(nx, T, cf.c, cf.c2, cf.k, cf.dx, fA, np.zeros(T + 1), N, ov, tau0=tau0 or None)[2]


def chk_paper_select():
    """The paper-literal span sequence equals the exact-rational restatement
    (select below the cap, several pairs, beta growth, exact beta rounding)."""
    ok = True
    for case in [(33, 2, 8, 0.5, 60, 0, 0), (41, 3, 10, 0.6, 80, 0, 0), (41, 4, 8, 0.5, 60, 25, 2)]:
        nx, N, ov, cfl, T, delay, tau0 = case
        fA, spans = _paper_select_expect(*case)
        got = oracle.rswr_paper(nx, T, 1.0, cfl / (nx - 1), fA, np.zeros(T + 1), N, ov, tau0=tau0)
        ok &= list(got["spans"]) == spans
    z = np.zeros(164)
    ok &= list(oracle.rswr_paper(121, 163, 1.0, 0.5 / 120, z, z, 2, 60, tau0=50)["spans"]) == [50, 55, 58]
    return bool(ok)


CHECKS = {"paper-select": chk_paper_select, "sources": chk_sources, "dalembert": chk_dalembert, "mode": chk_mode, "rational-canonical": lambda: chk_rational(0),
          "rational-increment": lambda: chk_rational(1), "energy": chk_energy, "rswr": chk_rswr,
          "paper": chk_paper, "adjoint": chk_adjoint}


def run_checks(L):
    saved = oracle._lib
    oracle._lib = L
    try:
        res = {}
        for name, fn in CHECKS.items():
            try:
                res[name] = bool(fn())
            except Exception:
                res[name] = False
        return res
    finally:
        oracle._lib = saved


@pytest.fixture(scope="module")
def tmpdir_mod():
    d = tempfile.mkdtemp(prefix="oracle_mutants_")
    yield d
    shutil.rmtree(d, ignore_errors=True)


def test_unmutated_oracle_passes_every_check(tmpdir_mod):
    res = run_checks(build_variant(tmpdir_mod, "clean", None))
    assert all(res.values()), res


@pytest.mark.parametrize("name", list(MUTANTS))
def test_every_planted_mistake_is_caught(tmpdir_mod, name):
    res = run_checks(build_variant(tmpdir_mod, name, MUTANTS[name]))
    assert not all(res.values()), f"mutant '{name}' passed every check: {res}"
