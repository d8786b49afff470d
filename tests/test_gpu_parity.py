"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Bar: bit-exact in both precisions when the oracle runs the same operation
order (canonical FP64, increment FP32, and the other two combinations), and
|err|/max|u| <= 1e-5 for FP32 against the FP64 oracle.
"""
from __future__ import annotations

import numpy as np
import pytest

from paper_2203_10477_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CAN, INC = 1, 2          # library form codes
ORACLE_FORM = {CAN: 0, INC: 1}
F32, F64 = 0, 1


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


def assert_bitwise(a, b, what=""):
    a = np.asarray(a)
    b = np.asarray(b)
    assert a.shape == b.shape, (what, a.shape, b.shape)
    bad = np.flatnonzero(a != b)
    assert bad.size == 0, f"{what}: {bad.size} mismatches, first at {bad[:5]}: {a.ravel()[bad[:5]]} vs {b.ravel()[bad[:5]]}"


# ----------------------------------------------------------------------------
# config 1 (nx = 1001, N = 2, overlap 16, CFL 0.5, 2000 steps, FP64)
# ----------------------------------------------------------------------------

def test_c1_rswr_equals_oracle_bitwise(R, oracle_mod):
    p = inputs.c1()
    plan = R.Plan.from_problem(p, dtype=F64)
    info = plan.info()
    assert info["span_steps"] == 8
    jr = 500
    out = plan.run(p.fA, p.fB, p.T, traces=True, j_r=jr)
    plan.check()
    ref = oracle_mod.leapfrog(p.nx, p.T, p.a, p.dt, p.fA, p.fB, rec_j=[jr])
    assert np.abs(ref["u"]).max() > 0.5
    assert_bitwise(host(out["u"]), ref["u"], "u^T")
    assert_bitwise(host(out["w"]), ref["w"], "u^{T-1}")
    assert_bitwise(host(out["recv"]), ref["rec"][0], "receiver")
    rs = oracle_mod.rswr_mask(p.nx, p.T, p.a, p.dt, p.fA, p.fB, p.n_sub, p.overlap)
    assert_bitwise(host(out["traces"]), rs["traces"], "interface output waveforms")


def test_c1_coefficients_match_oracle(R, oracle_mod):
    p = inputs.c1()
    info = R.Plan.from_problem(p, dtype=F64).info()
    cf = oracle_mod.coeffs(p.xa, p.xb, p.a, p.nx, p.dt)
    assert info["c2"] == cf.c2 and info["k"] == cf.k and info["inv2dx"] == cf.inv2dx
    assert np.float32(info["c2f"]) == cf.c2f and np.float32(info["kf"]) == cf.kf


def test_c1_monolithic_equals_oracle_bitwise(R, oracle_mod):
    p = inputs.c1()
    plan = R.Plan.from_problem(p, dtype=F64)
    out = plan.mono(p.fA, p.fB, p.T, traces=True, j_r=123)
    ref = oracle_mod.leapfrog(p.nx, p.T, p.a, p.dt, p.fA, p.fB, rec_j=[123])
    assert_bitwise(host(out["u"]), ref["u"], "mono u")
    assert_bitwise(host(out["w"]), ref["w"], "mono w")
    assert_bitwise(host(out["recv"]), ref["rec"][0], "mono receiver")
    rs = oracle_mod.rswr_mask(p.nx, p.T, p.a, p.dt, p.fA, p.fB, p.n_sub, p.overlap)
    assert_bitwise(host(out["traces"]), rs["traces"], "mono traces")


# ----------------------------------------------------------------------------
# every dtype x form, several tilings, ragged tails, random initial data
# ----------------------------------------------------------------------------

CASES = [
    # nx, N, ov, T, cfl
    (1001, 2, 16, 300, 0.5),
    (9973, 7, 24, 257, 0.9),     # prime nx: ragged last tile
    (20000, 4, 64, 411, 0.9),    # several CTA tiles per subdomain
    (4099, 3, 10, 96, 0.7),      # odd overlap half: S = 5
    (517, 1, 8, 33, 1.0),        # one subdomain, Courant number exactly 1
]


@pytest.mark.parametrize("dtype,form", [(F64, CAN), (F64, INC), (F32, INC), (F32, CAN)])
@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("mode", [0, 1])
def test_random_state_bitwise(R, oracle_mod, dtype, form, case, mode):
    nx, N, ov, T, cfl = case
    dt = cfl / (nx - 1)
    fA = inputs.ramped_sine(T, dt, freq=13.0)
    fB = 0.5 * inputs.ramped_sine(T, dt, freq=7.0)
    q0 = inputs.smooth_random_state(nx, seed=nx + T)
    q1 = q0 * 0.999
    if form == INC:
        q1 = q0 - q1  # v^0 = u^0 - u^{-1}
    plan = R.Plan(0.0, 1.0, 1.0, nx, dt, N, ov, dtype=dtype, form=form)
    plan.set_mode(mode)
    jr = nx // 3
    out = plan.run(fA, fB, T, q0=q0, q1=q1, traces=N > 1, j_r=jr)
    plan.check()
    dt_ = np.float64 if dtype == F64 else np.float32
    ref = oracle_mod.leapfrog(nx, T, 1.0, dt, fA, fB, form=ORACLE_FORM[form], prec=prec(dtype),
                              q0=q0.astype(dt_), q1=q1.astype(dt_), rec_j=[jr])
    assert_bitwise(host(out["u"]), ref["u"], "u")
    assert_bitwise(host(out["w"]), ref["w"], "w")
    assert_bitwise(host(out["recv"]), ref["rec"][0], "receiver")
    if N > 1:
        rs = oracle_mod.rswr_mask(nx, T, 1.0, dt, fA, fB, N, ov, form=ORACLE_FORM[form], prec=prec(dtype),
                                  q0=q0.astype(dt_), q1=q1.astype(dt_))
        assert_bitwise(host(out["traces"]), rs["traces"], "traces")


@pytest.mark.parametrize("dtype,form", [(F64, CAN), (F32, INC), (F32, CAN), (F64, INC)])
def test_every_variant_and_span_gives_identical_bits(R, oracle_mod, dtype, form):
    nx, N, ov, T = 30011, 5, 48, 203
    dt = 0.85 / (nx - 1)
    fA = inputs.gaussian_pulse(T, dt, sigma_steps=15)
    q0 = inputs.smooth_random_state(nx, seed=3)
    dt_ = np.float64 if dtype == F64 else np.float32
    jr = 12345
    ref = oracle_mod.leapfrog(nx, T, 1.0, dt, fA, np.zeros(T + 1), form=ORACLE_FORM[form], prec=prec(dtype),
                              q0=q0.astype(dt_), rec_j=[jr])
    rs = oracle_mod.rswr_mask(nx, T, 1.0, dt, fA, np.zeros(T + 1), N, ov, form=ORACLE_FORM[form], prec=prec(dtype),
                              q0=q0.astype(dt_))
    plan = R.Plan(0.0, 1.0, 1.0, nx, dt, N, ov, dtype=dtype, form=form)
    vs = [v for v in R.variants() if v["dtype"] == dtype and v["form"] == form]
    assert len(vs) >= 1
    for v in vs:
        for S in (1, 7, 16, ov // 2):
            if v["max_span"] and S > v["max_span"]:
                continue
            plan.set_span(S)
            plan.set_variant(v["variant"])
            assert plan.info()["variant"] == v["variant"] and plan.info()["span_steps"] == S
            for mode in (0, 1):
                plan.set_mode(mode)
                out = plan.run(fA, None, T, q0=q0, traces=True, j_r=jr)
                plan.check()
                what = f"variant {v} S={S} mode={mode}"
                assert_bitwise(host(out["u"]), ref["u"], what)
                assert_bitwise(host(out["w"]), ref["w"], what)
                assert_bitwise(host(out["recv"]), ref["rec"][0], what + " receiver")
                assert_bitwise(host(out["traces"]), rs["traces"], what + " traces")


def test_span_limit_of_free_warp_windows(R):
    """A variant whose warp halo is shorter than the span is refused; set_span
    moves a plan off such a variant onto one that runs the span."""
    free = [v for v in R.variants() if v["max_span"] > 0]
    assert free, "no free-window variant registered"
    v = free[0]
    m = v["max_span"]
    nx = 40001
    plan = R.Plan(0.0, 1.0, 1.0, nx, 0.9 / (nx - 1), 4, 2 * m + 16, dtype=v["dtype"], form=v["form"])
    plan.set_span(m)
    plan.set_variant(v["variant"])
    assert plan.info()["variant"] == v["variant"]
    plan.set_span(m + 8)
    info = plan.info()
    assert info["span_steps"] == m + 8 and info["variant"] != v["variant"]
    other = R.variants()[info["variant"]]
    assert other["max_span"] == 0 or other["max_span"] >= m + 8
    with pytest.raises(R.RSWRError):
        plan.set_variant(v["variant"])
    assert plan.info()["variant"] == info["variant"]


@pytest.mark.parametrize("T", [0, 1, 5, 31, 32, 33])
def test_short_and_ragged_spans(R, oracle_mod, T):
    nx, N, ov = 3001, 3, 64
    dt = 0.9 / (nx - 1)
    fA = inputs.ramped_sine(T, dt, freq=50.0) + 0.25
    q0 = inputs.smooth_random_state(nx, seed=11)
    plan = R.Plan(0.0, 1.0, 1.0, nx, dt, N, ov, dtype=F64)
    out = plan.run(fA, None, T, q0=q0, traces=True, j_r=1500)
    ref = oracle_mod.leapfrog(nx, T, 1.0, dt, fA, np.zeros(T + 1), q0=q0, rec_j=[1500])
    assert_bitwise(host(out["u"]), ref["u"], "u")
    assert_bitwise(host(out["w"]), ref["w"], "w")
    assert_bitwise(host(out["recv"]), ref["rec"][0], "receiver")


@pytest.mark.parametrize("dtype,form", [(F64, CAN), (F64, INC), (F32, INC), (F32, CAN)])
def test_spans_longer_than_a_sample_chunk(R, oracle_mod, dtype, form):
    """Spans of 64 steps: the boundary samples a warp holds are reloaded inside
    the span (every 32 steps), at both Dirichlet ends."""
    nx, N, ov, T = 5003, 3, 128, 300
    dt = 0.9 / (nx - 1)
    fA = inputs.ramped_sine(T, dt, freq=40.0) + 0.3
    fB = 0.7 * inputs.ramped_sine(T, dt, freq=23.0) - 0.1
    plan = R.Plan(0.0, 1.0, 1.0, nx, dt, N, ov, dtype=dtype, form=form)
    plan.set_span(64)
    assert plan.info()["span_steps"] == 64
    out = plan.run(fA, fB, T, traces=True, j_r=4000)
    plan.check()
    ref = oracle_mod.leapfrog(nx, T, 1.0, dt, fA, fB, form=ORACLE_FORM[form], prec=prec(dtype), rec_j=[4000])
    assert_bitwise(host(out["u"]), ref["u"], "u")
    assert_bitwise(host(out["w"]), ref["w"], "w")
    assert_bitwise(host(out["recv"]), ref["rec"][0], "receiver")


def test_adjoint_source_with_long_spans(R, oracle_mod):
    """The adjoint source (cotangent) through the span kernel with 64-step spans."""
    nx, N, ov, T, jr = 3001, 2, 128, 700, 1500
    a = 1.0
    dt = 0.9 / (nx - 1)
    g = inputs.lowpass_noise(T, seed=31)
    w = inputs.rng(32).standard_normal(T + 1)
    plan = R.Plan(0.0, 1.0, a, nx, dt, N, ov, dtype=F64)
    plan.set_span(64)
    res = plan.adjoint(g, None, T, jr, w)
    plan.check()
    ref = oracle_mod.adjoint(nx, T, a, dt, g, np.zeros(T + 1), jr, w)
    assert_bitwise(host(res["grad_fA"]), ref["dg"], "grad_fA with 64-step spans")


def test_smallest_grids(R, oracle_mod):
    for nx, N, ov in ((3, 1, 2), (4, 2, 2), (9, 2, 4), (64, 4, 16)):
        T = 40
        dt = 0.8 / (nx - 1)
        fA = inputs.ramped_sine(T, dt, freq=3.0)
        plan = R.Plan(0.0, 1.0, 1.0, nx, dt, N, ov, dtype=F64)
        out = plan.run(fA, None, T)
        ref = oracle_mod.leapfrog(nx, T, 1.0, dt, fA, np.zeros(T + 1))
        assert_bitwise(host(out["u"]), ref["u"], f"nx={nx}")


def test_fp32_within_1e5_of_fp64_oracle(R, oracle_mod):
    nx, N, ov, T = 60001, 8, 64, 5000
    dt = 0.9 / (nx - 1)
    fA = inputs.gaussian_pulse(T, dt)
    plan = R.Plan(0.0, 1.0, 1.0, nx, dt, N, ov, dtype=F32)
    out = plan.run(fA, None, T)
    ref = oracle_mod.leapfrog(nx, T, 1.0, dt, fA, np.zeros(T + 1), nx_run=oracle_mod.causal_extent(T, nx))
    u = host(out["u"]).astype(np.float64)
    n = len(ref["u"])
    err = np.abs(u[:n] - ref["u"]).max() / np.abs(ref["u"]).max()
    assert err <= 1e-5, err
    assert np.all(u[n:] == 0.0)


def test_run_host_matches_device_run(R):
    p = inputs.c1()
    plan = R.Plan.from_problem(p, dtype=F64)
    dev = plan.run(p.fA, p.fB, p.T, traces=True, j_r=77)
    hst = plan.run_host(p.fA, p.fB, p.T, traces=True, j_r=77)
    assert_bitwise(hst["u"].numpy(), host(dev["u"]), "u")
    assert_bitwise(hst["traces"].numpy(), host(dev["traces"]), "traces")
    assert_bitwise(hst["recv"].numpy(), host(dev["recv"]), "recv")


def test_rswr_equals_monolithic_gpu(R):
    nx, N, ov, T = 100003, 16, 64, 700
    dt = 0.9 / (nx - 1)
    q0 = inputs.smooth_random_state(nx, seed=8)
    fA = inputs.gaussian_pulse(T, dt, sigma_steps=10)
    for dtype in (F64, F32):
        plan = R.Plan(0.0, 1.0, 1.0, nx, dt, N, ov, dtype=dtype)
        a = plan.run(fA, None, T, q0=q0, j_r=4)
        b = plan.mono(fA, None, T, q0=q0, j_r=4)
        assert_bitwise(host(a["u"]), host(b["u"]), "u")
        assert_bitwise(host(a["w"]), host(b["w"]), "w")
        assert_bitwise(host(a["recv"]), host(b["recv"]), "recv")


# ----------------------------------------------------------------------------
# batches of uneven problems
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("dtype", [F32, F64])
def test_batch_each_problem_equals_its_oracle(R, oracle_mod, dtype):
    r = inputs.rng(99)
    P, T = 23, 300
    probs = []
    for i in range(P):
        nx = int(r.integers(200, 40000))
        a = float(r.uniform(0.5, 2.0))
        dt = inputs.dt_for_cfl(nx, a, 0.8)
        probs.append(inputs.Problem(nx, a, dt, T, max(1, -(-nx // 2048)), 32, inputs.sine(T, dt, float(r.uniform(1, 20))),
                                    np.zeros(T + 1)))
    b = R.Batch(probs, dtype=dtype)
    fA = np.concatenate([p.fA for p in probs])
    jr = np.array([p.nx // 2 for p in probs])
    out = b.run(fA, None, T, j_r=jr)
    b.check()
    u = host(out["u"])
    w = host(out["w"])
    rec = host(out["recv"])
    off = b.offsets
    form = 0 if dtype == F64 else 1
    for i, p in enumerate(probs):
        ref = oracle_mod.leapfrog(p.nx, T, p.a, p.dt, p.fA, p.fB, form=form, prec=prec(dtype), rec_j=[p.nx // 2])
        assert_bitwise(u[off[i]:off[i + 1]], ref["u"], f"problem {i} u")
        assert_bitwise(w[off[i]:off[i + 1]], ref["w"], f"problem {i} w")
        assert_bitwise(rec[i], ref["rec"][0], f"problem {i} receiver")


# ----------------------------------------------------------------------------
# adjoint: gradient w.r.t. the boundary waveform
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("jr", [1, 7, 150, 299, 0])
def test_adjoint_grad_fA_fp64_bitwise(R, oracle_mod, jr):
    nx, N, ov, T = 301, 3, 16, 420
    a = 1.3
    dt = 0.9 / (nx - 1) / a
    g = inputs.lowpass_noise(T, seed=21)
    z = np.zeros(T + 1)
    w = inputs.rng(5).standard_normal(T + 1)
    plan = R.Plan(0.0, 1.0, a, nx, dt, N, ov, dtype=F64)
    res = plan.adjoint(g, None, T, jr, w)
    ref = oracle_mod.adjoint(nx, T, a, dt, g, z, jr, w)
    assert np.abs(ref["dg"]).max() > 0
    assert_bitwise(host(res["grad_fA"]), ref["dg"], "grad_fA")


@pytest.mark.parametrize("T", [300, 2000])
def test_adjoint_grad_fA_fp32_bitwise_vs_fp32_sweep(R, oracle_mod, T):
    """The FP32 adjoint is exactly the FP32 increment-form leapfrog with the
    adjoint source (oracle emulation), bit for bit."""
    nx, N, ov, jr = 3001, 4, 64, 1200
    a = 1.3
    dt = 0.9 / (nx - 1) / a
    w = inputs.rng(6).standard_normal(T + 1)
    plan = R.Plan(0.0, 1.0, a, nx, dt, N, ov, dtype=F32)
    got = host(plan.adjoint(None, None, T, jr, w)["grad_fA"])
    w32 = w.astype(np.float32)
    src = np.concatenate([[0.0], w32[::-1].astype(np.float64)])
    zz = np.zeros(T + 2)
    lam = oracle_mod.leapfrog(nx, T + 1, a, dt, zz, zz, form=1, prec="f32", rec_j=[1], src_j=jr, src=src)
    c2f = lam["coeffs"].c2f
    dg = np.array([np.float32(c2f) * np.float32(lam["rec"][0][T - n]) for n in range(T)], dtype=np.float32)
    assert_bitwise(got[:T], dg, "FP32 adjoint")
    assert got[T] == 0.0


def test_adjoint_grad_fA_fp32_close(R, oracle_mod):
    nx, N, ov, T = 3001, 4, 64, 2000
    a = 1.3
    dt = 0.9 / (nx - 1) / a
    g = inputs.lowpass_noise(T, seed=2)
    w = inputs.rng(6).standard_normal(T + 1)
    plan = R.Plan(0.0, 1.0, a, nx, dt, N, ov, dtype=F32)
    res = plan.adjoint(g, None, T, 1200, w)
    ref = oracle_mod.adjoint(nx, T, a, dt, g, np.zeros(T + 1), 1200, w)
    got = host(res["grad_fA"]).astype(np.float64)
    err = np.linalg.norm(got - ref["dg"]) / np.linalg.norm(ref["dg"])
    assert err <= 1e-4, err


def test_autograd_function_matches_oracle(R, oracle_mod):
    nx, N, ov, T = 501, 2, 32, 300
    a = 1.0
    dt = 0.9 / (nx - 1)
    g = torch.tensor(inputs.lowpass_noise(T, seed=4), dtype=torch.float64, device="cuda", requires_grad=True)
    at = torch.tensor([a], dtype=torch.float64, device="cuda", requires_grad=True)
    z = np.zeros(T + 1)
    target = torch.tensor(oracle_mod.leapfrog(nx, T, 0.9 * a, dt, host(g), z, rec_j=[200])["rec"][0],
                          dtype=torch.float64, device="cuda")
    plan = R.Plan(0.0, 1.0, a, nx, dt, N, ov, dtype=F64)
    fn = R.rswr_function()
    tr = fn.apply(g, at, plan, T, 200)
    loss = ((tr - target) ** 2).sum()
    loss.backward()
    ref = oracle_mod.misfit_grad(nx, T, a, dt, host(g), z, 200, host(target))
    assert abs(loss.item() - ref["loss"]) <= 1e-12 * ref["loss"]
    np.testing.assert_allclose(host(g.grad), ref["dg"], rtol=1e-12, atol=1e-14 * np.abs(ref["dg"]).max())
    assert abs(at.grad.item() - ref["da"]) <= 1e-12 * ref["abs_da"]


def test_autograd_function_with_right_boundary_waveform(R, oracle_mod):
    """A non-zero right Dirichlet waveform enters the forward run and dL/da;
    a right waveform that asks for a gradient is refused."""
    nx, N, ov, T, jr = 401, 3, 32, 500, 300
    a = 1.0
    dt = 0.9 / (nx - 1)
    g = torch.tensor(inputs.lowpass_noise(T, seed=8), dtype=torch.float64, device="cuda", requires_grad=True)
    fB_h = inputs.ramped_sine(T, dt, freq=6.0) * 0.7
    fB = torch.tensor(fB_h, dtype=torch.float64, device="cuda")
    at = torch.tensor([a], dtype=torch.float64, device="cuda", requires_grad=True)
    target = torch.tensor(oracle_mod.leapfrog(nx, T, 0.9 * a, dt, host(g), fB_h, rec_j=[jr])["rec"][0],
                          dtype=torch.float64, device="cuda")
    plan = R.Plan(0.0, 1.0, a, nx, dt, N, ov, dtype=F64)
    fn = R.rswr_function()
    tr = fn.apply(g, at, plan, T, jr, fB)
    loss = ((tr - target) ** 2).sum()
    loss.backward()
    ref = oracle_mod.misfit_grad(nx, T, a, dt, host(g), fB_h, jr, host(target))
    ref0 = oracle_mod.misfit_grad(nx, T, a, dt, host(g), np.zeros(T + 1), jr, host(target))
    assert abs(ref["da"] - ref0["da"]) > 1e-3 * ref["abs_da"]  # fB matters here
    assert abs(loss.item() - ref["loss"]) <= 1e-12 * ref["loss"]
    np.testing.assert_allclose(host(g.grad), ref["dg"], rtol=1e-12, atol=1e-14 * np.abs(ref["dg"]).max())
    assert abs(at.grad.item() - ref["da"]) <= 1e-12 * ref["abs_da"]
    with pytest.raises(ValueError):
        fn.apply(g, at, plan, T, jr, fB.clone().requires_grad_(True))


# ----------------------------------------------------------------------------
# adjoint: gradient w.r.t. the wave speed (checkpointed forward, in-SMEM recompute)
# ----------------------------------------------------------------------------

# spacing 0: automatic (every span state kept, one persistent adjoint launch);
# > 0: a checkpoint every `spacing` spans, segments recomputed, one launch per span
@pytest.mark.parametrize("spacing", [0, 7])
@pytest.mark.parametrize("nx,N,ov,T,jr", [
    (301, 3, 16, 420, 120),      # 53 spans of 8 steps (8 segments when spaced)
    (2001, 4, 64, 2003, 777),    # ragged last span
    (4099, 2, 10, 333, 2000),    # S = 5
    (301, 3, 16, 420, 0),        # receiver on the Dirichlet node: dL/da = 0
    (301, 3, 16, 50, 250),       # receiver out of reach: everything 0
])
def test_adjoint_grad_a_fp64(R, oracle_mod, nx, N, ov, T, jr, spacing):
    a = 1.3
    dt = 0.9 / (nx - 1) / a
    g = inputs.lowpass_noise(T, seed=21)
    z = np.zeros(T + 1)
    w = inputs.rng(5).standard_normal(T + 1)
    plan = R.Plan(0.0, 1.0, a, nx, dt, N, ov, dtype=F64)
    plan.set_checkpoint_spacing(spacing)
    res = plan.adjoint(g, None, T, jr, w, want_a=True)
    plan.check()
    ref = oracle_mod.adjoint(nx, T, a, dt, g, z, jr, w)
    assert_bitwise(host(res["grad_fA"]), ref["dg"], "grad_fA (checkpointed path)")
    da = res["grad_a"].item()
    assert abs(da - ref["da"]) <= 1e-12 * max(ref["abs_da"], 1e-300), (da, ref["da"], ref["abs_da"])
    if jr == 0 or jr > T + 1:
        assert da == 0.0


@pytest.mark.parametrize("spacing", [0, 11])
def test_adjoint_grad_a_fp32(R, oracle_mod, spacing):
    nx, N, ov, T, jr = 3001, 4, 64, 2000, 1200
    a = 1.3
    dt = 0.9 / (nx - 1) / a
    g = inputs.lowpass_noise(T, seed=2)
    w = inputs.rng(6).standard_normal(T + 1)
    plan = R.Plan(0.0, 1.0, a, nx, dt, N, ov, dtype=F32)
    plan.set_checkpoint_spacing(spacing)
    res = plan.adjoint(g, None, T, jr, w, want_a=True)
    ref = oracle_mod.adjoint(nx, T, a, dt, g, np.zeros(T + 1), jr, w)
    da = res["grad_a"].item()
    assert abs(da - ref["da"]) <= 1e-4 * ref["abs_da"], (da, ref["da"], ref["abs_da"])
    got = host(res["grad_fA"]).astype(np.float64)
    assert np.linalg.norm(got - ref["dg"]) <= 1e-4 * np.linalg.norm(ref["dg"])


@pytest.mark.parametrize("nx", [8001, 8192])
def test_persistent_adjoint_equals_per_span_adjoint(R, oracle_mod, nx):
    """FP32: the persistent adjoint sweep (every span state kept; free warp
    windows, the Laplacians in tensor memory) and the per-span launches of the
    checkpointed path (the warps of a tile exchange neighbours through shared
    memory, Laplacians in shared memory) update every adjoint point with the
    same operations on the same operands, so dL/dfA agrees bit for bit.  They
    tile the grid differently (cores of 896 and 992 points), so the per-thread
    FP32 sums of pairing terms meet in another order: dL/da is asserted to the
    rounding of a 128-term FP32 sum (128 * 2^-24 of the sum of |terms|, taken
    from the FP64 oracle).  250 spans of 16 steps (the last one ragged), 8 to
    10 tiles per span.  nx = 8192 puts the right node on a thread's last
    register (the persistent kernel's select patch), nx = 8001 on its first
    (the general patch)."""
    dtype = F32
    N, ov, T, jr = 8, 64, 4001, 2500
    a = 1.3
    dt = 0.9 / (nx - 1) / a
    g = inputs.lowpass_noise(T, seed=4)
    w = inputs.rng(9).standard_normal(T + 1)
    out = []
    for spacing in (0, 6):
        plan = R.Plan(0.0, 1.0, a, nx, dt, N, ov, dtype=dtype)
        plan.set_checkpoint_spacing(spacing)
        res = plan.adjoint(g, None, T, jr, w, want_a=True)
        plan.check()
        out.append((host(res["grad_fA"]), res["grad_a"].item()))
    assert np.abs(out[0][0]).max() > 0 and out[0][1] != 0.0
    assert_bitwise(out[0][0], out[1][0], "grad_fA, persistent vs per-span")
    ref = oracle_mod.adjoint(nx, T, a, dt, g, np.zeros(T + 1), jr, w)
    assert abs(out[0][1] - out[1][1]) <= 128 * 2.0 ** -24 * ref["abs_da"], (out[0][1], out[1][1], ref["abs_da"])


def test_batch_adjoint_with_grad_a_fp32(R, oracle_mod):
    """FP32 batch of uneven problems with dL/da (the persistent adjoint sweep
    with its tensor-memory store over several problems' tiles): every
    problem's dL/dfA is bit for bit the one a single-problem plan gives, and
    both gradients are within the FP32 tolerances of the FP64 oracle."""
    r = inputs.rng(27)
    T = 500
    probs, jrs = [], []
    for i in range(4):
        nx = int(r.integers(900, 7000))
        a = float(r.uniform(0.5, 2.0))
        dt = inputs.dt_for_cfl(nx, a, 0.8)
        probs.append(inputs.Problem(nx, a, dt, T, max(1, nx // 1024), 32, inputs.lowpass_noise(T, seed=40 + i),
                                    np.zeros(T + 1)))
        # well inside the reach of the boundary waveform (0.8 points per step),
        # so that every gradient is far above FP32's rounding
        jrs.append(int(r.integers(1, T // 3)))
    b = R.Batch(probs, dtype=F32)
    fA = np.concatenate([p.fA for p in probs])
    w = inputs.rng(28).standard_normal((len(probs), T + 1))
    res = b.adjoint(fA, None, T, jrs, w, want_a=True)
    b.check()
    gf = host(res["grad_fA"])
    ga = host(res["grad_a"])
    for i, p in enumerate(probs):
        plan = R.Plan(0.0, 1.0, p.a, p.nx, p.dt, p.n_sub, p.overlap, dtype=F32)
        single = plan.adjoint(p.fA, None, T, jrs[i], w[i], want_a=True)
        assert_bitwise(gf[i], host(single["grad_fA"]), f"problem {i} grad_fA, batch vs single plan")
        ref = oracle_mod.adjoint(p.nx, T, p.a, p.dt, p.fA, p.fB, jrs[i], w[i])
        got = gf[i].astype(np.float64)
        assert np.linalg.norm(got - ref["dg"]) <= 1e-4 * np.linalg.norm(ref["dg"]), i
        assert abs(ga[i] - ref["da"]) <= 1e-4 * ref["abs_da"], (i, ga[i], ref["da"])


@pytest.mark.parametrize("spacing", [0, 5])
def test_batch_adjoint_with_grad_a(R, oracle_mod, spacing):
    r = inputs.rng(17)
    T = 400
    probs, jrs = [], []
    for i in range(5):
        nx = int(r.integers(500, 6000))
        a = float(r.uniform(0.5, 2.0))
        dt = inputs.dt_for_cfl(nx, a, 0.8)
        probs.append(inputs.Problem(nx, a, dt, T, max(1, nx // 1024), 32, inputs.lowpass_noise(T, seed=i),
                                    np.zeros(T + 1)))
        jrs.append(int(r.integers(1, min(nx - 1, T))))
    b = R.Batch(probs, dtype=F64)
    b.set_checkpoint_spacing(spacing)
    fA = np.concatenate([p.fA for p in probs])
    w = inputs.rng(18).standard_normal((len(probs), T + 1))
    res = b.adjoint(fA, None, T, jrs, w, want_a=True)
    b.check()
    gf = host(res["grad_fA"])
    ga = host(res["grad_a"])
    for i, p in enumerate(probs):
        ref = oracle_mod.adjoint(p.nx, T, p.a, p.dt, p.fA, p.fB, jrs[i], w[i])
        assert_bitwise(gf[i], ref["dg"], f"problem {i} grad_fA")
        assert abs(ga[i] - ref["da"]) <= 1e-12 * ref["abs_da"], (i, ga[i], ref["da"])


def test_c4_full_size_adjoint(R, oracle_mod):
    """Config 4 (nx = 2^20, a = 1.3, CFL 0.9, 8192 steps, N = 256, overlap 64):
    as written its receiver (x = 0.7) is out of reach, so every gradient is
    exactly 0; the reachable variant j_r = 4000 is compared with the oracle on
    the causal prefix of the grid (exact: nothing moves beyond T + 2 points)."""
    p = inputs.c4()
    tgt = oracle_mod.leapfrog(p.nx, p.T, 1.0, p.dt, p.fA, p.fB, rec_j=[4000],
                              nx_run=oracle_mod.causal_extent(p.T, p.nx))["rec"][0]
    plan = R.Plan.from_problem(p, dtype=F64)
    # as written: unreachable receiver
    w0 = inputs.rng(1).standard_normal(p.T + 1)
    res0 = plan.adjoint(p.fA, None, p.T, p.meta["j_r"], w0, want_a=True)
    assert float(res0["grad_fA"].abs().max()) == 0.0 and res0["grad_a"].item() == 0.0
    # reachable variant with the misfit cotangent
    fw = plan.run(p.fA, None, p.T, j_r=4000)
    wbar = 2.0 * (host(fw["recv"]) - tgt)
    res = plan.adjoint(p.fA, None, p.T, 4000, wbar, want_a=True)
    plan.check()
    ref = oracle_mod.adjoint(p.nx, p.T, p.a, p.dt, p.fA, p.fB, 4000, wbar,
                             nx_run=oracle_mod.causal_extent(p.T, p.nx))
    assert np.abs(ref["dg"]).max() > 0
    assert_bitwise(host(res["grad_fA"]), ref["dg"], "c4 grad_fA")
    assert abs(res["grad_a"].item() - ref["da"]) <= 1e-12 * ref["abs_da"]


# ----------------------------------------------------------------------------
# bounded waits: a tile that never publishes makes its neighbours time out
# ----------------------------------------------------------------------------

def test_missing_flag_times_out_and_context_survives(R, oracle_mod):
    nx, N, ov, T = 50000, 4, 64, 400
    dt = 0.9 / (nx - 1)
    fA = inputs.gaussian_pulse(T, dt, sigma_steps=10)
    plan = R.Plan(0.0, 1.0, 1.0, nx, dt, N, ov, dtype=F64)
    assert plan.info()["ntiles"] >= 3
    plan.set_mode(R.MODE_PERSISTENT)
    plan.set_wait_limit(0.2)
    plan.inject_missing_flag(1, 3)
    plan.run(fA, None, T)
    with pytest.raises(R.RSWRError) as ei:
        plan.check()
    assert ei.value.status == 6
    # the context is still usable and a clean run is exact
    plan.inject_missing_flag(-1, 0)
    out = plan.run(fA, None, T)
    plan.check()
    ref = oracle_mod.leapfrog(nx, T, 1.0, dt, fA, np.zeros(T + 1), nx_run=oracle_mod.causal_extent(T, nx))
    assert_bitwise(host(out["u"])[: len(ref["u"])], ref["u"], "after timeout")


@pytest.mark.parametrize("dtype", [F64, F32])
def test_missing_flag_times_out_in_a_resident_variant(R, oracle_mod, dtype):
    """Resident tiles wait for their neighbours every span: a tile that stops
    publishing (host-injected) makes the neighbours' bounded waits expire, the
    run reports RSWR_ETIMEOUT, and a clean run afterwards is exact."""
    nx, N, ov, T = 50000, 4, 64, 400
    dt = 0.9 / (nx - 1)
    fA = inputs.gaussian_pulse(T, dt, sigma_steps=10)
    plan = R.Plan(0.0, 1.0, 1.0, nx, dt, N, ov, dtype=dtype)
    res = [v for v in R.variants() if v["dtype"] == dtype and v["form"] == plan.info()["form"] and v["resident"]]
    assert res, "no resident variant registered"
    plan.set_variant(res[0]["variant"])
    assert plan.info()["ntiles"] >= 3
    plan.set_wait_limit(0.2)
    plan.inject_missing_flag(1, 3)
    plan.run(fA, None, T)
    with pytest.raises(R.RSWRError) as ei:
        plan.check()
    assert ei.value.status == 6
    plan.inject_missing_flag(-1, 0)
    out = plan.run(fA, None, T)
    plan.check()
    form, prec_ = (0, "f64") if dtype == F64 else (1, "f32")
    ref = oracle_mod.leapfrog(nx, T, 1.0, dt, fA, np.zeros(T + 1), form=form, prec=prec_,
                              nx_run=oracle_mod.causal_extent(T, nx))
    assert_bitwise(host(out["u"])[: len(ref["u"])], ref["u"], "after timeout")


def test_resident_variant_refuses_a_grid_that_does_not_fit(R):
    """One CTA per tile for the whole run needs every tile on the GPU at once;
    a larger grid is refused before anything is launched."""
    nx = 1 << 24
    plan = R.Plan(0.0, 1.0, 1.0, nx, 0.9 / (nx - 1), 1024, 64, dtype=F32)
    res = [v for v in R.variants() if v["dtype"] == F32 and v["form"] == plan.info()["form"] and v["resident"]]
    plan.set_variant(res[0]["variant"])
    with pytest.raises(R.RSWRError) as ei:
        plan.run(np.zeros(11), None, 10)
    assert ei.value.status == 7  # RSWR_ENOTSUP


# ----------------------------------------------------------------------------
# CUDA graphs, autotuner
# ----------------------------------------------------------------------------

def test_graph_replay_and_direct_launch_agree(R, oracle_mod):
    nx, N, ov, T = 40009, 6, 48, 321
    dt = 0.9 / (nx - 1)
    fA = torch.tensor(inputs.gaussian_pulse(T, dt, sigma_steps=12), device="cuda", dtype=torch.float64)
    q0 = torch.tensor(inputs.smooth_random_state(nx, seed=2), device="cuda", dtype=torch.float64)
    out = (torch.empty(nx, dtype=torch.float64, device="cuda"), torch.empty(nx, dtype=torch.float64, device="cuda"))
    plan = R.Plan(0.0, 1.0, 1.0, nx, dt, N, ov, dtype=F64)
    ref = oracle_mod.leapfrog(nx, T, 1.0, dt, host(fA), np.zeros(T + 1), q0=host(q0))
    for mode in (0, 1):
        plan.set_mode(mode)
        for graph in (True, True, False, True):  # capture, replay, direct, capture again
            plan.set_graph(graph)
            out[0].fill_(7.0)
            plan.run(fA, None, T, q0=q0, out=out)
            plan.check()
            assert_bitwise(host(out[0]), ref["u"], f"mode {mode} graph {graph}")


def test_batch_autotune_then_exact(R, oracle_mod):
    r = inputs.rng(31)
    T = 257
    probs = []
    for i in range(9):
        nx = int(r.integers(3000, 60000))
        dt = inputs.dt_for_cfl(nx, 1.0, 0.8)
        probs.append(inputs.Problem(nx, 1.0, dt, T, max(1, nx // 2048), 32, inputs.sine(T, dt, 3.0 + i), np.zeros(T + 1)))
    b = R.Batch(probs, dtype=F32)
    v = b.autotune(48)
    info = b.info()
    assert info["variant"] == v and 1 <= info["span_steps"] <= 16
    out = b.run(np.concatenate([p.fA for p in probs]), None, T)
    b.check()
    u = host(out["u"])
    for i, p in enumerate(probs):
        ref = oracle_mod.leapfrog(p.nx, T, p.a, p.dt, p.fA, p.fB, form=1, prec="f32")
        assert_bitwise(u[b.offsets[i]:b.offsets[i + 1]], ref["u"], f"problem {i}")


# ----------------------------------------------------------------------------
# full-size workloads (sampled / causal-prefix parity)
# ----------------------------------------------------------------------------

def test_c2_full_size_both_precisions(R, oracle_mod):
    """nx = 2^24, N = 1024, overlap 64, CFL 0.9, 10^4 steps: the bench workload."""
    p = inputs.c2()
    n = oracle_mod.causal_extent(p.T, p.nx)
    ref64 = oracle_mod.leapfrog(p.nx, p.T, p.a, p.dt, p.fA, p.fB, rec_j=[5000], nx_run=n)
    ref32 = oracle_mod.leapfrog(p.nx, p.T, p.a, p.dt, p.fA, p.fB, rec_j=[5000], nx_run=n, form=1, prec="f32")
    for dtype, ref in ((F64, ref64), (F32, ref32)):
        plan = R.Plan.from_problem(p, dtype=dtype)
        out = plan.run(p.fA, p.fB, p.T, j_r=5000)
        plan.check()
        u = host(out["u"])
        assert_bitwise(u[:n], ref["u"], f"c2 dtype {dtype} causal prefix")
        assert np.all(u[n:] == 0.0)
        assert_bitwise(host(out["recv"]), ref["rec"][0], "c2 receiver")
        if dtype == F32:
            err = np.abs(u[:n].astype(np.float64) - ref64["u"]).max() / np.abs(ref64["u"]).max()
            assert err <= 1e-5, err


def host_map(fn, items):
    """fn over items on all host cores (the oracle's C calls release the GIL)."""
    import concurrent.futures as cf
    import os

    with cf.ThreadPoolExecutor(max_workers=os.cpu_count() or 1) as ex:
        return list(ex.map(fn, items))


def test_c3_full_size_batch(R, oracle_mod):
    """4096 independent problems (nx in [2^10, 2^18], a in [0.5, 2], CFL 0.8,
    4096 steps, N_p = ceil(nx/2048), overlap 32), one persistent launch, FP32:
    every problem within 1e-5 (relative to its max |u|) of the FP64 oracle on
    its causal prefix and exactly 0 beyond it; 24 sampled problems bit for bit
    against the oracle's FP32 twin of the same operation order."""
    probs = inputs.c3_problems()
    T = probs[0].T
    b = R.Batch(probs, dtype=F32)
    fA = np.concatenate([p.fA for p in probs])
    out = b.run(fA, None, T)
    b.check()
    u = host(out["u"])
    off = b.offsets
    n_of = lambda p: oracle_mod.causal_extent(T, p.nx)
    for i, p in enumerate(probs):
        assert np.all(u[off[i] + n_of(p):off[i + 1]] == 0.0), i

    def err64(i):
        p = probs[i]
        n = n_of(p)
        ref = oracle_mod.leapfrog(p.nx, T, p.a, p.dt, p.fA, p.fB, nx_run=n)["u"]
        return float(np.abs(u[off[i]:off[i] + n].astype(np.float64) - ref).max() / np.abs(ref).max())

    errs = np.array(host_map(err64, range(len(probs))))
    print(f"c3 FP32 vs FP64 oracle: max {errs.max():.2e}, median {np.median(errs):.2e} over {len(errs)} problems")
    assert errs.max() <= 1e-5, (int(errs.argmax()), errs.max())
    for i in inputs.rng(5).choice(len(probs), 24, replace=False):
        p = probs[i]
        n = n_of(p)
        ref = oracle_mod.leapfrog(p.nx, T, p.a, p.dt, p.fA, p.fB, form=1, prec="f32", nx_run=n)
        assert_bitwise(u[off[i]:off[i] + n], ref["u"], f"c3 problem {i}")


def test_c5_full_size(R, oracle_mod):
    """nx = 2^28 FP32, N = 8192, overlap 64, 2^15 steps (causal-prefix parity),
    then 512 uneven problems (nx in [2^12, 2^20]) with boundary-waveform
    gradients of a receiver misfit (two sampled problems against the oracle)."""
    p = inputs.c5_big()
    plan = R.Plan.from_problem(p, dtype=F32)
    out = plan.run(p.fA, p.fB, p.T, j_r=20000)
    plan.check()
    n = oracle_mod.causal_extent(p.T, p.nx)
    u = out["u"]
    assert float(u[n:].abs().max()) == 0.0
    ref = oracle_mod.leapfrog(p.nx, p.T, p.a, p.dt, p.fA, p.fB, rec_j=[20000], nx_run=n, form=1, prec="f32")
    assert_bitwise(host(u[:n]), ref["u"], "c5 causal prefix")
    assert_bitwise(host(out["recv"]), ref["rec"][0], "c5 receiver")
    # the FP32 run of 2^15 steps against the FP64 oracle
    ref64 = oracle_mod.leapfrog(p.nx, p.T, p.a, p.dt, p.fA, p.fB, nx_run=n)["u"]
    err = np.abs(host(u[:n]).astype(np.float64) - ref64).max() / np.abs(ref64).max()
    print(f"c5 grid FP32 vs FP64 oracle: {err:.2e}")
    assert err <= 1e-5, err
    del out, u, plan
    torch.cuda.empty_cache()

    probs = inputs.c5_uneven()
    T = probs[0].T
    jr = [q.meta["j_r"] for q in probs]
    b = R.Batch(probs, dtype=F32)
    fA = np.concatenate([q.fA for q in probs])
    # smooth cotangents (like a misfit residual of smooth traces) and white noise
    smooth = np.stack([inputs.lowpass_noise(T, seed=1000 + i) for i in range(len(probs))])
    rough = inputs.rng(77).standard_normal((len(probs), T + 1))
    # FP32 tolerance from the arithmetic: the leapfrog neither damps nor grows
    # a perturbation, so one FP32 rounding (2^-24 relative) per step adds up
    # to at most about T * 2^-24 over the T steps of the adjoint sweep
    # (1.95e-3 at T = 2^15; measured 1.2e-4 .. 5.6e-4 on these problems)
    tol_fp32 = T * 2.0 ** -24
    for w, tol in ((smooth, tol_fp32), (rough, tol_fp32)):
        g = b.adjoint(fA, None, T, jr, w)
        b.check()
        gf = host(g["grad_fA"])
        assert np.all(np.isfinite(gf))
        # eight problems spread over the sizes, plus two fixed ones
        order = np.argsort([q.nx for q in probs])
        pick = sorted(set([3, 200] + [int(order[k]) for k in np.linspace(0, len(probs) - 1, 8).round().astype(int)]))

        def gerr(i):
            q = probs[i]
            ref = oracle_mod.adjoint(q.nx, T, q.a, q.dt, q.fA, q.fB, jr[i], w[i],
                                     nx_run=oracle_mod.causal_extent(T, q.nx))
            return float(np.linalg.norm(gf[i].astype(np.float64) - ref["dg"]) / np.linalg.norm(ref["dg"]))

        for i, err in zip(pick, host_map(gerr, pick)):
            print(f"c5 problem {i} (nx {probs[i].nx}) FP32 grad_fA rel. 2-norm error {err:.2e} (tolerance {tol:g})")
            assert err <= tol, (i, err)


# ----------------------------------------------------------------------------
# the paper-literal RSWR (data-chosen spans, flux-exchange update)
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("form", [CAN, INC])
@pytest.mark.parametrize("nx,N,ov,cfl,T", [
    (1001, 2, 16, 0.5, 2000),     # config 1
    (1001, 10, 16, 0.5, 600),
    (1001, 4, 24, 0.9, 600),
    (1001, 3, 9, 0.7, 600),
    (20001, 16, 32, 0.9, 3000),
])
def test_paper_literal_equals_oracle_bitwise(R, oracle_mod, form, nx, N, ov, cfl, T):
    dt = cfl / (nx - 1)
    fA = inputs.ramped_sine(T, dt, freq=7.0)
    z = np.zeros(T + 1)
    plan = R.Plan(0.0, 1.0, 1.0, nx, dt, N, ov, dtype=F64, form=form)
    got = plan.run_paper(fA, None, T)
    ref = oracle_mod.rswr_paper(nx, T, 1.0, dt, fA, z, N, ov, form=ORACLE_FORM[form])
    assert np.array_equal(got["spans"], ref["spans"]), (got["spans"][:10], ref["spans"][:10])
    assert_bitwise(host(got["u"]), ref["u"], "paper-literal u")
    assert_bitwise(host(got["w"]), ref["w"], "paper-literal w")
    mono = oracle_mod.leapfrog(nx, T, 1.0, dt, fA, z, form=ORACLE_FORM[form])
    assert np.abs(host(got["u"]) - mono["u"]).max() <= 1e-12 * np.abs(mono["u"]).max()


# tiny grids on which the paper's select binds below the Theorem's cap (the
# oracle's span rule is pinned on the same geometries): nx, N, ov, Courant
# number, T; a dyadic boundary pulse
PAPER_BINDING_CASES = [(33, 2, 8, 0.5, 60), (40, 3, 8, 0.3, 70), (41, 3, 10, 0.6, 80), (29, 2, 6, 0.9, 50)]


@pytest.mark.parametrize("form", [CAN, INC])
@pytest.mark.parametrize("nx,N,ov,cfl,T", PAPER_BINDING_CASES)
def test_paper_literal_binding_select_bitwise(R, oracle_mod, form, nx, N, ov, cfl, T):
    """Spans chosen below the cap by the data: the device-side span choice
    needs several batches of queued spans (a batch is the fewest spans that
    could finish the run), and the span sequence and the state still equal
    the oracle's bit for bit."""
    dt = cfl / (nx - 1)
    m = np.arange(T + 1)
    fA = np.where((m > 0) & (m < 8), np.round(np.sin(np.pi * m / 8) ** 2 * 64) / 64, 0.0)
    z = np.zeros(T + 1)
    plan = R.Plan(0.0, 1.0, 1.0, nx, dt, N, ov, dtype=F64, form=form)
    got = plan.run_paper(fA, None, T)
    ref = oracle_mod.rswr_paper(nx, T, 1.0, dt, fA, z, N, ov, form=ORACLE_FORM[form])
    assert list(got["spans"]) == list(ref["spans"])
    assert sum(got["spans"]) == T
    assert_bitwise(host(got["u"]), ref["u"], "paper-literal u")
    assert_bitwise(host(got["w"]), ref["w"], "paper-literal w")


def test_paper_literal_binding_select_reached_below_the_cap(oracle_mod):
    """(CPU) the cases above do take spans below the Theorem's cap, so the
    device loop needs more than one batch on them."""
    below = 0
    for nx, N, ov, cfl, T in PAPER_BINDING_CASES:
        dt = cfl / (nx - 1)
        m = np.arange(T + 1)
        fA = np.where((m > 0) & (m < 8), np.round(np.sin(np.pi * m / 8) ** 2 * 64) / 64, 0.0)
        spans = oracle_mod.rswr_paper(nx, T, 1.0, dt, fA, np.zeros(T + 1), N, ov)["spans"]
        cap = int(np.ceil((ov - 1) / (2 * cfl))) - 1
        below += int(min(spans[:-1]) < cap) if len(spans) > 1 else 0
    assert below >= 3


def test_paper_literal_fp32_close_to_fp64(R, oracle_mod):
    nx, N, ov, T = 20001, 16, 32, 3000
    dt = 0.9 / (nx - 1)
    fA = inputs.gaussian_pulse(T, dt, sigma_steps=20)
    plan = R.Plan(0.0, 1.0, 1.0, nx, dt, N, ov, dtype=F32)
    got = plan.run_paper(fA, None, T)
    mono = oracle_mod.leapfrog(nx, T, 1.0, dt, fA, np.zeros(T + 1))
    err = np.abs(host(got["u"]).astype(np.float64) - mono["u"]).max() / np.abs(mono["u"]).max()
    assert err <= 1e-5, err
    assert got["spans"].sum() == T


@pytest.mark.parametrize("dtype,form", [(F64, CAN), (F32, INC), (F32, CAN), (F64, INC)])
@pytest.mark.parametrize("nx,N,ov,T,jr", [
    (20011, 1000, 8, 150, 10007),   # interfaces every 20 points: hundreds of probes per tile
    (8001, 20, 4, 200, 399),        # probes 3 apart next to the receiver: several per thread
])
def test_dense_interface_traces_every_variant(R, oracle_mod, dtype, form, nx, N, ov, T, jr):
    """Interface output waveforms where a tile or a thread holds many probes
    (the tile-list and the per-thread overflow recording paths), every variant."""
    dt = 0.9 / (nx - 1)
    fA = inputs.ramped_sine(T, dt, freq=60.0) + 0.2
    q0 = inputs.smooth_random_state(nx, seed=17)
    dt_ = np.float64 if dtype == F64 else np.float32
    ref = oracle_mod.leapfrog(nx, T, 1.0, dt, fA, np.zeros(T + 1), form=ORACLE_FORM[form], prec=prec(dtype),
                              q0=q0.astype(dt_), rec_j=[jr])
    rs = oracle_mod.rswr_mask(nx, T, 1.0, dt, fA, np.zeros(T + 1), N, ov, form=ORACLE_FORM[form], prec=prec(dtype),
                              q0=q0.astype(dt_))
    plan = R.Plan(0.0, 1.0, 1.0, nx, dt, N, ov, dtype=dtype, form=form)
    for v in [v for v in R.variants() if v["dtype"] == dtype and v["form"] == form]:
        plan.set_variant(v["variant"])
        for mode in (0, 1):
            plan.set_mode(mode)
            out = plan.run(fA, None, T, q0=q0, traces=True, j_r=jr)
            plan.check()
            what = f"variant {v['variant']} mode {mode}"
            assert_bitwise(host(out["u"]), ref["u"], what)
            assert_bitwise(host(out["recv"]), ref["rec"][0], what + " receiver")
            assert_bitwise(host(out["traces"]), rs["traces"], what + " traces")


def test_adjoint_matches_central_differences_of_the_gpu_forward(R):
    """The GPU gradients against central differences of GPU forward runs (FP64):
    along a random direction of f_A the loss is quadratic, so the difference is
    exact up to rounding; in a it is O(h^2)."""
    nx, N, ov, T, jr = 2001, 4, 64, 1500, 700
    a = 1.3
    dt = 0.9 / ((nx - 1) * a)
    g = inputs.lowpass_noise(T, seed=41)
    dirn = inputs.rng(42).standard_normal(T + 1)

    def trace(a_, fA):
        plan = R.Plan(0.0, 1.0, a_, nx, dt, N, ov, dtype=F64)
        out = plan.run(fA, None, T, j_r=jr)
        plan.check()
        return host(out["recv"])

    target = trace(1.0, g)

    def loss(a_, fA):
        r = trace(a_, fA) - target
        return float(np.dot(r, r))

    plan = R.Plan(0.0, 1.0, a, nx, dt, N, ov, dtype=F64)
    wbar = 2.0 * (trace(a, g) - target)
    res = plan.adjoint(g, None, T, jr, wbar, want_a=True)
    plan.check()
    gfa = host(res["grad_fA"])
    ga = float(host(res["grad_a"])[0])
    assert np.abs(gfa).max() > 0 and ga != 0.0
    h = 1e-3
    fd = (loss(a, g + h * dirn) - loss(a, g - h * dirn)) / (2 * h)
    assert abs(fd - np.dot(gfa, dirn)) <= 1e-8 * (abs(fd) + 1e-300)
    ha = 1e-6 * a  # the O(h^2) term is about 8e-9 relative here (7e-5 at 1e-4 a)
    fda = (loss(a + ha, g) - loss(a - ha, g)) / (2 * ha)
    assert abs(fda - ga) <= 1e-7 * abs(ga)


@pytest.mark.parametrize("dtype,form", [(F64, CAN), (F64, INC), (F32, INC), (F32, CAN)])
def test_resume_from_a_span_boundary_state(R, dtype, form):
    """Checkpoint / resume (Sec. 2.6: the span loop restarts from the combined
    state): a run of T1 steps followed by a run of T - T1 steps from its final
    state pair, with the boundary samples from level T1 on, equals one run of T
    steps bit for bit, at a span boundary and off one."""
    nx, N, ov, T = 6007, 6, 48, 400
    dt = 0.9 / (nx - 1)
    fA = inputs.ramped_sine(T, dt, freq=31.0) + 0.1
    fB = 0.4 * inputs.ramped_sine(T, dt, freq=17.0)
    q0 = inputs.smooth_random_state(nx, seed=23)
    plan = R.Plan(0.0, 1.0, 1.0, nx, dt, N, ov, dtype=dtype, form=form)
    full = plan.run(fA, fB, T, q0=q0)
    ref_u, ref_w = host(full["u"]), host(full["w"])
    S = plan.info()["span_steps"]
    for T1 in (5 * S, 5 * S + 3):
        a = plan.run(fA[:T1 + 1], fB[:T1 + 1], T1, q0=q0)
        b = plan.run(fA[T1:], fB[T1:], T - T1, q0=a["u"].clone(), q1=a["w"].clone())
        plan.check()
        assert_bitwise(host(b["u"]), ref_u, f"resumed at {T1}: u")
        assert_bitwise(host(b["w"]), ref_w, f"resumed at {T1}: w")


def test_c1_equals_the_stored_oracle_values(R):
    """The GPU run of the golden problem (the c1 grid with a polynomial boundary
    pulse) against the values stored in tests/golden/c1_fp64.txt (written from
    the oracle on another machine): final state, receiver and both interface
    waveforms, bit for bit, with no oracle run in the test."""
    import os
    import sys

    here = os.path.dirname(os.path.abspath(__file__))
    sys.path.insert(0, os.path.join(here, "golden"))
    import make_golden

    stored = make_golden.read(os.path.join(here, "golden", "c1_fp64.txt"))
    p = make_golden.problem()
    plan = R.Plan.from_problem(p, dtype=F64)
    out = plan.run(p.fA, p.fB, p.T, traces=True, j_r=make_golden.RECV_J)
    plan.check()
    u, rec, tr = host(out["u"]), host(out["recv"]), host(out["traces"])
    got = {"u_T": [(j, u[j]) for j in make_golden.U_POINTS],
           "recv": [(n, rec[n]) for n in make_golden.LEVELS],
           "trace_left": [(n, tr[0, 0, n]) for n in make_golden.LEVELS],
           "trace_right": [(n, tr[0, 1, n]) for n in make_golden.LEVELS]}
    for key, rows in got.items():
        assert [(i, float(v)) for i, v in rows] == stored[key], key


# ----------------------------------------------------------------------------
# a forward run kept for the gradient (rswr_run_keep)
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("dtype", [F64, F32])
@pytest.mark.parametrize("nx,N,ov,T,jr", [
    (301, 3, 16, 420, 120),      # 53 spans of 8 (FP64) / 27 of 16 (FP32)
    (2001, 4, 64, 2003, 777),    # ragged last span
    (301, 3, 16, 5, 2),          # one short span
    (301, 3, 16, 0, 2),          # no step
])
def test_run_keep_equals_run_and_the_adjoint_reuses_it(R, oracle_mod, dtype, nx, N, ov, T, jr):
    a = 1.3
    dt = 0.9 / (nx - 1) / a
    td = torch.float64 if dtype == F64 else torch.float32
    g = torch.tensor(inputs.lowpass_noise(T, seed=21), dtype=td, device="cuda")
    fB = torch.tensor(inputs.ramped_sine(T, dt, freq=3.0) * 0.3, dtype=td, device="cuda")
    w = torch.tensor(inputs.rng(5).standard_normal(T + 1), dtype=td, device="cuda")
    plan = R.Plan(0.0, 1.0, a, nx, dt, N, ov, dtype=dtype)
    ref = plan.run(g, fB, T, j_r=jr)
    ref = {k: ref[k].clone() for k in ("u", "w", "recv")}
    fresh = plan.adjoint(g, fB, T, jr, w, want_a=True)
    fresh = {k: fresh[k].clone() for k in ("grad_fA", "grad_a")}
    kept = plan.run_keep(g, fB, T, j_r=jr)
    for k in ("u", "w", "recv"):
        assert torch.equal(kept[k], ref[k]), f"rswr_run_keep {k} differs from rswr_run"
    for _ in range(2):  # the kept states serve more than one cotangent
        got = plan.adjoint(g, fB, T, jr, w, want_a=True)
        plan.check()
        assert torch.equal(got["grad_fA"], fresh["grad_fA"])
        assert torch.equal(got["grad_a"], fresh["grad_a"])
    if dtype == F64 and T > 0:
        o = oracle_mod.adjoint(nx, T, a, dt, host(g), host(fB), jr, host(w))
        assert_bitwise(host(got["grad_fA"]), o["dg"], "grad_fA after a kept run")
        assert abs(float(got["grad_a"][0]) - o["da"]) <= 1e-12 * o["abs_da"]


@pytest.mark.parametrize("dtype", [F32, F64])
def test_resident_checkpoint_sweep_equals_the_ticketed_one(R, oracle_mod, dtype):
    """A plan on a resident variant runs the adjoint's checkpoint sweep (every
    span state kept) as one resident launch that writes each span's core; the
    gradients, and a kept forward run (its state, receiver trace and the
    gradient that reuses it), equal those of a plan on the default variant
    bit for bit (the adjoint tiling is the same, so dL/da is summed in the
    same order).  63 spans, the last one ragged."""
    nx, N, ov, T, jr = 20001, 8, 64, 1001, 700
    a = 1.3
    dt = 0.9 / (nx - 1) / a
    g = inputs.lowpass_noise(T, seed=12)
    w = inputs.rng(13).standard_normal(T + 1)
    res_v = [v for v in R.variants() if v["dtype"] == dtype and v["resident"]]
    assert res_v
    ref_plan = R.Plan(0.0, 1.0, a, nx, dt, N, ov, dtype=dtype)
    ref = ref_plan.adjoint(g, None, T, jr, w, want_a=True)
    ref_keep = ref_plan.run_keep(g, None, T, j_r=jr)
    ref_after = ref_plan.adjoint(g, None, T, jr, w, want_a=True)
    ref_plan.check()
    assert float(ref["grad_fA"].abs().max()) > 0
    for v in res_v:
        plan = R.Plan(0.0, 1.0, a, nx, dt, N, ov, dtype=dtype)
        plan.set_span(min(32, v["max_span"] or 32))
        plan.set_variant(v["variant"])
        got = plan.adjoint(g, None, T, jr, w, want_a=True)
        plan.check()
        what = f"variant {v['variant']}"
        assert_bitwise(host(got["grad_fA"]), host(ref["grad_fA"]), what + " grad_fA")
        assert got["grad_a"].item() == ref["grad_a"].item(), what
        kept = plan.run_keep(g, None, T, j_r=jr)
        plan.check()
        for k in ("u", "w", "recv"):
            assert_bitwise(host(kept[k]), host(ref_keep[k]), f"{what} kept run {k}")
        after = plan.adjoint(g, None, T, jr, w, want_a=True)
        plan.check()
        assert_bitwise(host(after["grad_fA"]), host(ref_after["grad_fA"]), what + " grad_fA after keep")
        assert after["grad_a"].item() == ref_after["grad_a"].item(), what


def test_adjoint_after_run_keep_with_other_inputs_sweeps_again(R, oracle_mod):
    """Other boundary samples (another pointer) than the kept run's: the adjoint
    does its own forward sweep and matches the oracle for its own inputs."""
    nx, N, ov, T, jr, a = 301, 3, 16, 420, 120, 1.3
    dt = 0.9 / (nx - 1) / a
    g1 = torch.tensor(inputs.lowpass_noise(T, seed=1), dtype=torch.float64, device="cuda")
    g2 = torch.tensor(inputs.lowpass_noise(T, seed=2), dtype=torch.float64, device="cuda")
    w = torch.tensor(inputs.rng(5).standard_normal(T + 1), dtype=torch.float64, device="cuda")
    plan = R.Plan(0.0, 1.0, a, nx, dt, N, ov, dtype=F64)
    plan.run_keep(g1, None, T, j_r=jr)
    got = plan.adjoint(g2, None, T, jr, w, want_a=True)
    o = oracle_mod.adjoint(nx, T, a, dt, host(g2), np.zeros(T + 1), jr, host(w))
    assert abs(float(got["grad_a"][0]) - o["da"]) <= 1e-12 * o["abs_da"]
    # a changed span discards the kept states as well
    plan.run_keep(g1, None, T, j_r=jr)
    plan.set_span(4)
    got = plan.adjoint(g1, None, T, jr, w, want_a=True)
    o = oracle_mod.adjoint(nx, T, a, dt, host(g1), np.zeros(T + 1), jr, host(w))
    assert abs(float(got["grad_a"][0]) - o["da"]) <= 1e-12 * o["abs_da"]
    assert_bitwise(host(got["grad_fA"]), o["dg"], "grad_fA")
