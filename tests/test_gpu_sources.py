"""GPU parity of user point sources (the pulse sources of the paper's Sec. 4
experiments) against the CPU oracle.

A source adds its sample of level n+1 at its point when level n+1 is formed;
every RSWR window that holds the point applies it, halo included, so the
RSWR result equals the monolithic leapfrog with the sources bit for bit
(Sec. 2.4).  The placements below put sources on tile-core and window edges,
on neighbouring points held by one thread, twice on one point, next to the
Dirichlet nodes and on them (where they never apply).
"""
from __future__ import annotations

import numpy as np
import pytest

from paper_2203_10477_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CAN, INC = 1, 2
ORACLE_FORM = {CAN: 0, INC: 1}
F32, F64 = 0, 1
FORMS = [(F64, CAN), (F64, INC), (F32, INC), (F32, CAN)]


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_10477_gb300 import build, rswr

    build.build()
    return rswr


def host(t):
    return t.detach().cpu().numpy()


def prec(dtype):
    return "f64" if dtype == F64 else "f32"


def npdt(dtype):
    return np.float64 if dtype == F64 else np.float32


def assert_bitwise(a, b, what=""):
    a = np.asarray(a)
    b = np.asarray(b)
    assert a.shape == b.shape, (what, a.shape, b.shape)
    bad = np.flatnonzero(a != b)
    assert bad.size == 0, f"{what}: {bad.size} mismatches, first at {bad[:5]}: {a.ravel()[bad[:5]]} vs {b.ravel()[bad[:5]]}"


def edge_sources(nx, T, dt, info, seed=7):
    """Pulse sources at cell centres plus sources on the tiling's edges."""
    j, s = inputs.pulse_sources(nx, T, dt, K=10)
    core, H, W = info["core"], info["halo"], info["window"]
    extra = []
    for t in (1, 2, 3):
        c0 = t * core
        extra += [c0, c0 - 1, c0 - H, c0 + H - 1, c0 - H + W - 1, c0 + core - 1]
    extra += [5000, 5001, 5002, 5001, 1, nx - 2, 0, nx - 1, 5003 + 40]
    extra = [x for x in extra if 0 <= x < nx]
    r = inputs.rng(seed)
    es = 0.01 * r.standard_normal((len(extra), T + 1))
    return np.concatenate([j, np.asarray(extra, np.int64)]), np.concatenate([s, es])


def padded(samples, extra_cols, dtype):
    """Rows longer than T+1 (pitch > T+1): the trailing columns are never read."""
    K, L = samples.shape
    out = np.full((K, L + extra_cols), 1e30, npdt(dtype))
    out[:, :L] = samples
    return out


@pytest.mark.parametrize("dtype,form", FORMS)
@pytest.mark.parametrize("mode", [0, 1])
def test_sources_rswr_equals_oracle_bitwise(R, oracle_mod, dtype, form, mode):
    nx, N, ov, T = 20011, 10, 48, 600
    dt = 0.9 / (nx - 1)
    plan = R.Plan(0.0, 1.0, 1.0, nx, dt, N, ov, dtype=dtype, form=form)
    plan.set_mode(mode)
    j, s = edge_sources(nx, T, dt, plan.info())
    s = s.astype(npdt(dtype))
    plan.set_sources(j, padded(s, 5, dtype))
    q0 = inputs.smooth_random_state(nx, seed=5).astype(npdt(dtype))
    fA = inputs.ramped_sine(T, dt, freq=11.0)
    jr = 5001
    out = plan.run(fA, None, T, q0=q0, traces=True, j_r=jr)
    plan.check()
    ref = oracle_mod.leapfrog(nx, T, 1.0, dt, fA, np.zeros(T + 1), form=ORACLE_FORM[form], prec=prec(dtype),
                              q0=q0, rec_j=[jr], src_j=j, src=s)
    assert np.abs(ref["u"][4990:5010]).max() > 0
    assert_bitwise(host(out["u"]), ref["u"], "u")
    assert_bitwise(host(out["w"]), ref["w"], "w")
    assert_bitwise(host(out["recv"]), ref["rec"][0], "receiver")
    rs = oracle_mod.rswr_mask(nx, T, 1.0, dt, fA, np.zeros(T + 1), N, ov, form=ORACLE_FORM[form], prec=prec(dtype),
                              q0=q0, src_j=j, src=s)
    assert_bitwise(host(out["traces"]), rs["traces"], "traces")
    # without the sources the run differs (the sources did enter)
    plan.set_sources(None)
    bare = plan.run(fA, None, T, q0=q0)
    assert not np.array_equal(host(bare["u"]), ref["u"])


@pytest.mark.parametrize("dtype,form", FORMS)
def test_sources_monolithic_equals_oracle_bitwise(R, oracle_mod, dtype, form):
    nx, N, ov, T = 9001, 10, 32, 400
    dt = 0.8 / (nx - 1)
    plan = R.Plan(0.0, 1.0, 1.0, nx, dt, N, ov, dtype=dtype, form=form)
    j, s = edge_sources(nx, T, dt, plan.info())
    j = np.concatenate([j, [1023, 1024, 1025, 2047, 2048]])  # monolithic block edges
    s = np.concatenate([s, 0.02 * inputs.rng(9).standard_normal((5, T + 1))]).astype(npdt(dtype))
    plan.set_sources(j, s)
    out = plan.mono(None, None, T, j_r=1024)
    plan.check()
    ref = oracle_mod.leapfrog(nx, T, 1.0, dt, np.zeros(T + 1), np.zeros(T + 1), form=ORACLE_FORM[form],
                              prec=prec(dtype), rec_j=[1024], src_j=j, src=s)
    assert_bitwise(host(out["u"]), ref["u"], "mono u")
    assert_bitwise(host(out["w"]), ref["w"], "mono w")
    assert_bitwise(host(out["recv"]), ref["rec"][0], "mono receiver")
    run = plan.run(None, None, T, j_r=1024)
    assert_bitwise(host(run["u"]), host(out["u"]), "rswr vs mono")


@pytest.mark.parametrize("dtype,form", FORMS)
def test_sources_every_variant_and_span(R, oracle_mod, dtype, form):
    nx, N, ov, T = 30011, 10, 64, 230
    dt = 0.85 / (nx - 1)
    plan = R.Plan(0.0, 1.0, 1.0, nx, dt, N, ov, dtype=dtype, form=form)
    q0 = inputs.smooth_random_state(nx, seed=8).astype(npdt(dtype))
    vs = [v for v in R.variants() if v["dtype"] == dtype and v["form"] == form]
    refs = {}
    for v in vs:
        for S in (7, 16, ov // 2):
            if v["max_span"] and S > v["max_span"]:
                continue
            plan.set_span(S)
            plan.set_variant(v["variant"])
            # the edge placements follow each tiling
            j, s = edge_sources(nx, T, dt, plan.info(), seed=S)
            s = s.astype(npdt(dtype))
            key = (tuple(j), S)
            if key not in refs:
                refs[key] = oracle_mod.leapfrog(nx, T, 1.0, dt, np.zeros(T + 1), np.zeros(T + 1),
                                                form=ORACLE_FORM[form], prec=prec(dtype), q0=q0, src_j=j, src=s)
            ref = refs[key]
            plan.set_sources(j, s)
            for mode in (0, 1):
                plan.set_mode(mode)
                out = plan.run(None, None, T, q0=q0)
                plan.check()
                what = f"variant {v} S={S} mode={mode}"
                assert_bitwise(host(out["u"]), ref["u"], what)
                assert_bitwise(host(out["w"]), ref["w"], what)


@pytest.mark.parametrize("dtype,form", FORMS)
def test_sources_with_spans_longer_than_a_sample_chunk(R, oracle_mod, dtype, form):
    """64-step spans: a warp's source samples are reloaded inside the span."""
    nx, N, ov, T = 5003, 3, 128, 300
    dt = 0.9 / (nx - 1)
    plan = R.Plan(0.0, 1.0, 1.0, nx, dt, N, ov, dtype=dtype, form=form)
    plan.set_span(64)
    assert plan.info()["span_steps"] == 64
    j = np.array([1700, 2500, 2501, 3333], np.int64)
    s = (0.05 * inputs.rng(12).standard_normal((4, T + 1))).astype(npdt(dtype))
    plan.set_sources(j, s)
    out = plan.run(None, None, T, j_r=2500)
    plan.check()
    ref = oracle_mod.leapfrog(nx, T, 1.0, dt, np.zeros(T + 1), np.zeros(T + 1), form=ORACLE_FORM[form],
                              prec=prec(dtype), rec_j=[2500], src_j=j, src=s)
    assert_bitwise(host(out["u"]), ref["u"], "u")
    assert_bitwise(host(out["recv"]), ref["rec"][0], "receiver")


def test_sources_run_host_matches_device_run(R):
    nx, N, ov, T = 8001, 10, 32, 200
    dt = 0.9 / (nx - 1)
    plan = R.Plan(0.0, 1.0, 1.0, nx, dt, N, ov, dtype=F64)
    j, s = inputs.pulse_sources(nx, T, dt)
    plan.set_sources(j, s)
    d = plan.run(None, None, T, j_r=4000)
    h = plan.run_host(None, None, T, j_r=4000)
    assert_bitwise(h["u"].numpy(), host(d["u"]), "host u")
    assert_bitwise(h["recv"].numpy(), host(d["recv"]), "host receiver")


@pytest.mark.parametrize("dtype", [F32, F64])
def test_sources_in_a_batch(R, oracle_mod, dtype):
    T = 300
    probs = []
    for nx, a, cfl, N, ov in [(4001, 1.0, 0.9, 4, 32), (12007, 0.7, 0.8, 10, 48), (3001, 1.5, 0.6, 2, 16)]:
        probs.append(inputs.Problem(nx, a, inputs.dt_for_cfl(nx, a, cfl), T, N, ov, np.zeros(T + 1),
                                    np.zeros(T + 1)))
    b = R.Batch(probs, dtype=dtype)
    pidx = np.array([0, 0, 2, 1, 1, 1, 2], np.int32)
    jj = np.array([100, 101, 1500, 6000, 6000, 11000, 2999], np.int64)
    s = (0.05 * inputs.rng(21).standard_normal((len(jj), T + 1))).astype(npdt(dtype))
    b.set_sources(pidx, jj, s)
    out = b.run(None, None, T)
    b.check()
    u = host(out["u"])
    off = b.offsets
    for i, p in enumerate(probs):
        sel = np.flatnonzero(pidx == i)
        ref = oracle_mod.leapfrog(p.nx, T, p.a, p.dt, p.fA, p.fB, form=0 if dtype == F64 else 1,
                                  prec=prec(dtype), src_j=jj[sel], src=s[sel])
        assert_bitwise(u[off[i]:off[i + 1]], ref["u"], f"problem {i} u")


def test_source_errors(R):
    nx, T = 2001, 50
    dt = 0.9 / (nx - 1)
    plan = R.Plan(0.0, 1.0, 1.0, nx, dt, 2, 16, dtype=F64)
    with pytest.raises(R.RSWRError):
        plan.set_sources([nx], np.zeros((1, T + 1)))
    with pytest.raises(R.RSWRError):
        plan.set_sources([-1], np.zeros((1, T + 1)))
    plan.set_sources([1000], np.zeros((1, T + 1)))
    with pytest.raises(R.RSWRError):  # samples shorter than T+1 levels
        plan.run(None, None, T + 1)
    with pytest.raises(R.RSWRError):  # the adjoint runs without sources
        plan.adjoint(None, None, T, 500, np.ones(T + 1))
    plan.set_sources(None)
    plan.adjoint(None, None, T, 500, np.ones(T + 1))
    plan.check()
