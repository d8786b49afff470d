#!/usr/bin/env python3
"""RSWR benchmark: GLUP/s of the RSWR hot path on one GB300 (or N replicas).

Workload (one "step" = one whole RSWR run, every span of predict / select /
update): 1-D wave u_tt = u_xx on [0, 1], nx = 2**24 points, N = 1024
subdomains with a 64-point overlap (span S = 32), Courant number 0.9,
10**4 time steps, left boundary a Gaussian pulse (sigma = 50 dt, t0 = 4 sigma),
right boundary 0, zero initial data, interface output waveforms of all 1023
interfaces recorded.  GLUP/s counts useful interior updates: (nx - 2) * T per
step.

The headline line is the FP64 run (canonical form, bit-identical to the FP64
oracle); the same line carries the FP32 run (increment form), the monolithic
GPU leapfrog comparators, the span kernel's roofline, the end-to-end number
through the C ABI with host buffers, the CPU oracle baseline and the SM clocks
seen during the timed region.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun every rank runs its own replica of the workload (the problem is
not split across GPUs); the time is the maximum over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2203_10477_gb300 import inputs  # noqa: E402

METRIC = "GLUP/s and % stencil roofline, RSWR vs monolithic GPU leapfrog at FP64-matched error"
UNIT = "GLUP/s"
WORKLOAD = "1-D wave a=1, nx=2^24, N=1024 subdomains, overlap 64, CFL 0.9, 10^4 steps, Gaussian pulse"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
SM_MAX_MHZ = 2070.0
# streaming multiprocessors of the device; main() sets it from the device
# properties before any roofline is computed
SM_COUNT = None


def load_peaks() -> dict:
    try:
        with open(PEAKS_FILE) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "source": "measured"}
    except Exception:
        return {"hbm_gbs": 6800.0, "source": "fallback"}


NO_TRACES = False  # profiling case without interface traces (--no-traces)
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic_span_kernel_c2.md")
# the sources of the span kernels a run without point sources executes
KERNEL_SOURCES = ["span_kernel.cuh", "span_kernel.cu", "span_common.cuh", "rswr_device.cuh", "rswr_internal.h"]


def kernel_sha() -> str:
    import hashlib

    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2203_10477_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic(dtype: str, variant: int, span: int):
    """DRAM bytes per update of the span kernel from the committed ncu capture,
    when it was taken on these very kernel sources, variant and span."""
    try:
        sha = kernel_sha()
        for line in open(TRAFFIC_FILE):
            cells = [c.strip() for c in line.strip().strip("|").split("|")]
            if len(cells) >= 7 and cells[0] == dtype and cells[1].isdigit():
                if int(cells[1]) == variant and int(cells[2]) == span and cells[3] == sha:
                    return float(cells[6])
    except Exception:
        return None
    return None


# Arithmetic instructions per update of each measured path (the pipe that bounds it):
# forward span kernel: FP64 canonical 3 (add, 2 fma), FP32 increment 4 (2 sub, fma, add);
# dL/dfA alone: the adjoint variables through the same span kernel;
# dL/dfA and dL/da: checkpoint sweep (3 / 4) + adjoint kernel (recompute 3 / 4, Laplacian
# 1 / 0 (the increment form's second difference is the Laplacian), pairing 1, adjoint step 3 / 4).
# after a kept forward run (rswr_run_keep) the gradient skips the checkpoint sweep.
ADJ_OPS = {"f64": {"g": 3, "full": 3 + 3 + 1 + 1 + 3, "after_keep": 3 + 1 + 1 + 3},
           "f32": {"g": 4, "full": 4 + 4 + 0 + 1 + 4, "after_keep": 4 + 0 + 1 + 4}}


# FMA rates of the two pipes measured on this device by rswr_fma_probe (set in main)
MEASURED_ALU = {}


def alu_roofline(dtype: str, value: float, ops: int) -> dict:
    """ALU roofline of a path doing `ops` arithmetic instructions per update on the
    FP64 pipe (2 / clock / SM) or the FP32 pipe (128 lanes / clock / SM) at 2070 MHz,
    with the same bound from the pipe rate measured by the FMA probe beside it."""
    lanes = 2 if dtype == "f64" else 128
    peak = SM_COUNT * lanes * 2.07e9 / ops / 1e9
    out = {"bound": "alu", "unit": "GLUP/s", "peak": peak, "frac": value / peak,
           "ops_per_update": ops, "pipe": "fp64" if dtype == "f64" else "fp32",
           "peak_definition": f"{SM_COUNT} SMs x {lanes} {dtype.upper()} lanes/clk x 2070 MHz / {ops} instr per update"}
    m = MEASURED_ALU.get(dtype)
    if m:
        out["peak_measured"] = m["fma_per_s"] / ops / 1e9
        out["frac_of_measured"] = value / out["peak_measured"]
    return out


def span_roofline(dtype: str, value: float, ops: int, info: dict) -> dict:
    """The binding roofline of a span-kernel run: the lower of the ALU bound
    (alu_roofline) and the HBM bound at the span kernel's algorithmic bytes per
    update, w (2 W + 2 core) / (core S) (both levels of every window in, both
    levels of its core out, once per span of S steps)."""
    w = 8 if dtype == "f64" else 4
    W, core, S = info["window"], info["core"], info["span_steps"]
    bpu = w * (2 * W + 2 * core) / (core * S)
    hbm = load_peaks()["hbm_gbs"]
    alu = alu_roofline(dtype, value, ops)
    hbm_peak = hbm / bpu
    out = dict(alu, alu_peak=alu["peak"], hbm_peak=hbm_peak, algorithmic_bytes_per_update=bpu)
    if hbm_peak < alu["peak"]:
        out.update(bound="hbm", peak=hbm_peak, frac=value / hbm_peak)
    return out


def measure_alu(torch, dev) -> dict:
    """FMA throughput of the FP64 and FP32 pipes on `dev` (rswr_fma_probe),
    with the SM clocks sampled while the probe ran."""
    from paper_2203_10477_gb300 import rswr

    clocks = ClockSampler(gpu_uuid(torch, dev))
    clocks.start()
    time.sleep(0.3)
    res = {name: rswr.fma_rate(dt, device=dev) for name, dt in (("f64", rswr.F64), ("f32", rswr.F32),
                                                                ("f32x2", 2), ("f32x2_add", 3))}
    clk = clocks.stop()
    mhz = clk["sm_mhz"] if clk else SM_MAX_MHZ
    for r in res.values():
        r["per_sm_per_clock"] = r["fma_per_s"] / (r["sms"] * mhz * 1e6)
    res["clocks"] = clk
    return res


def alu_peaks(sm_mhz: float) -> dict:
    """Arithmetic-pipe-bound LUP rates of the span kernel's fast path.

    FP64 canonical form: 3 FP64-pipe instructions per update (DADD, 2 DFMA);
    GB300 issues 2 FP64 instructions per clock per SM (its 1.25 TFLOP/s FP64
    rating at 2.07 GHz on 152 SMs).  FP32 increment form: 4 FP32-pipe
    instructions per update (3 FADD, 1 FFMA) at 128 lanes per clock per SM."""
    f = sm_mhz * 1e6
    return {"f64": SM_COUNT * 2 * f / 3 / 1e9, "f32": SM_COUNT * 128 * f / 4 / 1e9}


# ----------------------------------------------------------------------------
# clocks during the timed region
# ----------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None
        self.path = None

    def other_processes(self):
        """Compute processes on this GPU other than this one (a shared GPU skews timing)."""
        try:
            out = subprocess.run(["nvidia-smi", "-i", self.gpu_id, "--query-compute-apps=pid,used_memory",
                                  "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=10).stdout
        except Exception:
            return None
        pids = []
        for line in out.splitlines():
            parts = [q.strip() for q in line.split(",")]
            if parts and parts[0].isdigit() and int(parts[0]) != os.getpid():
                pids.append(int(parts[0]))
        return pids

    def start(self):
        self.others = set(self.other_processes() or [])
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", self.gpu_id, f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.others |= set(self.other_processes() or [])
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                rows.append((float(parts[0]), float(parts[1]), parts[3:]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        sm = [r[0] for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for name, val in zip(names, r[2][1:]):
                if val.strip().lower() == "active":
                    reasons.add(name)
        loaded = [s for s in sm if s > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": sorted(reasons), "samples": len(rows),
                "other_gpu_processes": sorted(self.others)}


# ----------------------------------------------------------------------------
# the reference arm and the CPU baseline: the oracle on the host cores
# ----------------------------------------------------------------------------

def host_cores() -> int:
    """Host cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def oracle_sample(p, steps: int, threads: int = 1) -> float:
    """Seconds for `steps` leapfrog steps of the CPU oracle over the full grid
    on `threads` host threads (the result is the same bit for bit)."""
    import oracle

    oracle.set_threads(threads)
    try:
        t0 = time.perf_counter()
        oracle.leapfrog(p.nx, steps, p.a, p.dt, p.fA[: steps + 1], p.fB[: steps + 1])
        return time.perf_counter() - t0
    finally:
        oracle.set_threads(1)


def cpu_baseline(p, budget_s: float = 10.0) -> dict:
    """The oracle's monolithic leapfrog on all host cores (the reported value)
    and on one core, each on a sample of about `budget_s` seconds."""
    import oracle

    oracle.build()
    res = {}
    for cores in (host_cores(), 1):
        oracle_sample(p, 2, cores)  # start the threads
        # each call allocates and first-touches its arrays: calibrate on enough
        # steps that this start-up cost is a small part
        t64 = oracle_sample(p, 64, cores)
        steps = int(max(64, min(p.T, budget_s / max(t64 / 64, 1e-9))))
        secs = oracle_sample(p, steps, cores)
        res[cores] = ((p.nx - 2) * steps / secs / 1e9, steps, secs)
    n = host_cores()
    v, steps, secs = res[n]
    v1, steps1, secs1 = res[1]
    return {"value": v, "unit": UNIT, "cores": n, "kind": "oracle",
            "sample": f"FP64 canonical oracle leapfrog (plain C, OpenMP over the points of a level, {n} threads), "
                      f"full nx=2^24 grid, {steps} of the 10^4 steps, {secs:.1f} s",
            "single_core": {"value": v1, "unit": UNIT, "cores": 1,
                            "sample": f"the same on one thread, {steps1} steps, {secs1:.1f} s"}}


def run_reference(args, rank: int, world: int) -> None:
    if rank != 0:
        return
    p = inputs.c2()
    import oracle

    oracle.build()
    cores = host_cores()
    oracle_sample(p, 2, cores)  # start the threads
    t64 = oracle_sample(p, 64, cores)
    steps_per = int(max(64, min(p.T, 4.0 / max(t64 / 64, 1e-9))))  # about 4 s of CPU work per step
    for _ in range(args.warmup):
        oracle_sample(p, steps_per, cores)
    times = [oracle_sample(p, steps_per, cores) for _ in range(args.steps)]
    total = sum(times)
    lups = (p.nx - 2) * steps_per * args.steps
    value = lups / total / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
        "config": {"workload": WORKLOAD, "nx": p.nx, "n_sub": p.n_sub, "overlap": p.overlap, "cfl": 0.9,
                   "T": p.T, "sample_steps_per_step": steps_per},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"each step: FP64 oracle leapfrog (OpenMP, {cores} threads) over the full "
                                   f"nx=2^24 grid for {steps_per} of the 10^4 time steps"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------
# the checker leg: FP32 results against the FP64 oracle (outside timed regions)
# ----------------------------------------------------------------------------

def host_map(fn, items):
    """fn over items on the host cores (the oracle's C calls release the GIL)."""
    import concurrent.futures as cf

    import oracle

    oracle.build()
    oracle.set_threads(1)
    with cf.ThreadPoolExecutor(max_workers=host_cores()) as ex:
        return list(ex.map(fn, items))


def rel_max(u, ref) -> float:
    """max |u - ref| / max |ref| in FP64."""
    u = np.asarray(u, np.float64)
    ref = np.asarray(ref, np.float64)
    scale = float(np.abs(ref).max())
    return float(np.abs(u - ref).max()) / scale if scale > 0 else float(np.abs(u).max())


def prefix_ref(p, T=None):
    """The FP64 oracle on the causal prefix of a zero-data run with a quiet
    right end: level T vanishes beyond j = T + 1, so the grid truncated to
    T + 2 points gives the full grid's values there."""
    import oracle

    T = p.T if T is None else T
    m = oracle.causal_extent(T, p.nx)
    return m, oracle.leapfrog(p.nx, T, p.a, p.dt, p.fA[: T + 1], p.fB[: T + 1], nx_run=m)["u"]


def state_error(u_dev, p) -> dict:
    """FP32 final state (device) of one problem against the FP64 oracle on its
    causal prefix; the FP32 state beyond the prefix must be exactly 0."""
    m, ref = prefix_ref(p)
    u = u_dev[:m].double().cpu().numpy()
    tail = int((u_dev[m:] != 0).sum()) if m < p.nx else 0
    return {"err_vs_fp64": rel_max(u, ref), "prefix_points": m, "nonzero_beyond_prefix": tail}


def batch_state_error(out_dev, offsets, probs, idx=None) -> dict:
    """state_error over the problems `idx` (all by default) of a packed batch output."""
    idx = list(range(len(probs))) if idx is None else list(idx)
    refs = host_map(lambda i: prefix_ref(probs[i]), idx)
    errs, tail = [], 0
    for i, (m, ref) in zip(idx, refs):
        o0, o1 = int(offsets[i]), int(offsets[i + 1])
        u = out_dev[o0:o0 + m].double().cpu().numpy()
        errs.append(rel_max(u, ref))
        if o0 + m < o1:
            tail += int((out_dev[o0 + m:o1] != 0).sum())
    return {"err_vs_fp64": max(errs), "err_vs_fp64_median": float(np.median(errs)), "problems_checked": len(idx),
            "problems_above_1e-5": int(sum(e > 1e-5 for e in errs)), "nonzero_beyond_prefix": tail}


def pulse10_error(u_dev, p, j, s) -> dict:
    """FP32 final state of the pulse-source run against the FP64 oracle.  Each
    source's disturbance stays within T points of it (zero data and quiet
    ends), and the sources are far apart, so the oracle runs each source on the
    2T + 5 points around it (same coefficients, zero ends); every other point
    must be exactly 0."""
    import oracle

    T = p.T
    m = 2 * T + 5
    z = np.zeros(T + 1)

    def one(q):
        lo = int(j[q]) - T - 2
        assert lo >= 1 and lo + m <= p.nx - 1
        return lo, oracle.leapfrog(p.nx, T, p.a, p.dt, z, z, nx_run=m, src_j=[T + 2], src=s[q:q + 1])["u"]

    refs = host_map(one, range(len(j)))
    covered = np.zeros(p.nx, bool)
    err_num, scale = 0.0, 0.0
    for lo, ref in refs:
        u = u_dev[lo:lo + m].double().cpu().numpy()
        err_num = max(err_num, float(np.abs(u - ref).max()))
        scale = max(scale, float(np.abs(ref).max()))
        covered[lo:lo + m] = True
    mask = torch_from_numpy_like(covered, u_dev)
    tail = int((u_dev[~mask] != 0).sum())
    return {"err_vs_fp64": err_num / scale, "nonzero_outside_cones": tail, "sources_checked": len(refs)}


def torch_from_numpy_like(a, like):
    import torch

    return torch.from_numpy(a).to(like.device)


def grad_error(g32, ga32, p, j_r, wbar, want_a=True, nx_run=None) -> dict:
    """FP32 gradients against the FP64 oracle's discrete adjoint (same inputs
    in FP64): relative 2-norm error of dL/dfA, relative error of dL/da."""
    import oracle

    m = nx_run or oracle.causal_extent(p.T, p.nx)
    ref = oracle.adjoint(p.nx, p.T, p.a, p.dt, p.fA, p.fB, j_r, np.asarray(wbar, np.float64), nx_run=m)
    g = np.asarray(g32, np.float64)
    out = {"grad_fA_err_vs_fp64": float(np.linalg.norm(g - ref["dg"]) / np.linalg.norm(ref["dg"]))}
    if want_a:
        out["grad_a_err_vs_fp64"] = abs(float(ga32) - ref["da"]) / abs(ref["da"])
        out["grad_a_err_vs_fp64_of_sum_abs_terms"] = abs(float(ga32) - ref["da"]) / ref["abs_da"]
    out["_ref"] = ref
    return out


# ----------------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------------

def gpu_uuid(torch, dev) -> str:
    try:
        u = torch.cuda.get_device_properties(dev).uuid
        s = str(u)
        return s if s.startswith("GPU-") else "GPU-" + s
    except Exception:
        return str(dev.index or 0)


class RunBench:
    """Device buffers and timing events for repeated whole RSWR runs of one plan."""

    def __init__(self, torch, plan, p):
        from paper_2203_10477_gb300 import rswr

        self.torch, self.plan, self.p = torch, plan, p
        td = torch.float64 if plan.dtype == rswr.F64 else torch.float32
        self.fA = torch.as_tensor(p.fA, device="cuda").to(td)
        self.fB = torch.as_tensor(p.fB, device="cuda").to(td)
        self.out = (torch.empty(p.nx, dtype=td, device="cuda"), torch.empty(p.nx, dtype=td, device="cuda"))
        self.k0 = torch.cuda.Event(enable_timing=True)
        self.k1 = torch.cuda.Event(enable_timing=True)
        # torch creates the CUDA events on first record: create them before the
        # library is given their handles
        self.k0.record()
        self.k1.record()
        torch.cuda.synchronize()

    def warmup(self, n):
        for _ in range(n):
            self.plan.run(self.fA, self.fB, self.p.T, traces=True, out=self.out)
        self.torch.cuda.synchronize()
        self.plan.check()

    def timed(self, steps, flush):
        """Per-step (whole run ms, span-kernel ms), each on the launching stream."""
        torch = self.torch
        stream = torch.cuda.current_stream()
        self.plan.set_kernel_events(self.k0, self.k1)
        run_ms, ker_ms = [], []
        for _ in range(steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            self.plan.run(self.fA, self.fB, self.p.T, traces=True, out=self.out)
            e1.record(stream)
            e1.synchronize()
            run_ms.append(e0.elapsed_time(e1))
            ker_ms.append(self.k0.elapsed_time(self.k1))
        self.plan.set_kernel_events(None, None)
        self.plan.check()
        return run_ms, ker_ms


def mono_runs(torch, plan, p, steps, flush):
    stream = torch.cuda.current_stream()
    from paper_2203_10477_gb300 import rswr

    fA = torch.as_tensor(p.fA, device="cuda").to(torch.float64 if plan.dtype == rswr.F64 else torch.float32)
    out = (torch.empty(p.nx, dtype=fA.dtype, device="cuda"), torch.empty(p.nx, dtype=fA.dtype, device="cuda"))
    plan.mono(fA, None, p.T, out=out)  # warm-up
    ms = []
    for _ in range(steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        plan.mono(fA, None, p.T, out=out)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    return ms


def e2e_run(torch, plan, p, steps):
    """rswr_run_host: pinned host waveforms in, final state pair + traces out."""
    from paper_2203_10477_gb300 import rswr

    td = torch.float64 if plan.dtype == rswr.F64 else torch.float32
    es = 8 if plan.dtype == rswr.F64 else 4
    fA = torch.as_tensor(p.fA).to(td).pin_memory()
    fB = torch.as_tensor(p.fB).to(td).pin_memory()
    out = (torch.empty(p.nx, dtype=td).pin_memory(), torch.empty(p.nx, dtype=td).pin_memory())
    plan.run_host(fA, fB, p.T, out=out)  # warm-up
    stream = torch.cuda.current_stream()
    ms = []
    for _ in range(steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        plan.run_host(fA, fB, p.T, out=out)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    h2d = 2 * (p.T + 1) * es
    d2h = 2 * p.nx * es
    return ms, h2d, d2h


def profile_case(which: str, variant=None, span=None, full=False, log2_nx=22) -> None:
    """The bench workload (full = True) or its small version for detailed
    captures: nx = 2^log2_nx (default 2^22), subdomains of the bench's length of
    16384 points (so the same share of tiles carries interface probes) and 1280 steps
    (40 spans of 32, so the fill and drain of the span pipeline are a small
    part); four state arrays of 32 MiB (FP64) / 16 MiB (FP32), so DRAM counters
    still see traffic beyond L2.  Runs the workload twice (the first run warms
    up).  adj64 / adj32: the c4 gradient workload (dL/dfA and dL/da)."""
    import dataclasses

    import torch

    from paper_2203_10477_gb300 import build, rswr

    build.build()
    if which == "c3":
        # the batched workload's first 1024 problems for 256 steps (16 spans of
        # 16), FP32, in the bench's configuration (variant, one launch per span)
        probs = inputs.c3_problems(P=1024, T=256)
        b = rswr.Batch(probs, dtype=rswr.F32)
        if variant is not None:
            b.set_variant(variant)
        b.set_mode(1)
        fA = torch.as_tensor(np.concatenate([q.fA for q in probs]), device="cuda").to(torch.float32)
        for _ in range(2):
            b.run(fA, None, probs[0].T)
        torch.cuda.synchronize()
        b.check()
        print(json.dumps({"profile_case": which, "problems": len(probs), "T": probs[0].T, "info": b.info()}))
        return
    if which == "g32":
        # the c4 FP32 boundary gradient (the adjoint variables through the span
        # kernel, source at j_r = 4000, probe at j = 1), 2^log2_nx points and
        # 1024 steps, in the given variant; run twice
        p = inputs.c4(T=1024, nx=1 << log2_nx, j_r=4000)
        plan = rswr.Plan.from_problem(p, dtype=rswr.F32)
        if variant is not None:
            plan.set_span(span or 32)
            plan.set_variant(variant)
        fA = torch.as_tensor(p.fA, device="cuda").float()
        w = torch.as_tensor(inputs.lowpass_noise(p.T, seed=4), device="cuda").float()
        for _ in range(2):
            plan.adjoint(fA, None, p.T, 4000, w, want_a=False)
        torch.cuda.synchronize()
        plan.check()
        print(json.dumps({"profile_case": which, "nx": p.nx, "T": p.T, "info": plan.info()}))
        return
    if which in ("paper64", "paper32"):
        # the paper-literal run on the c2 grid, 2000 steps (once to warm, once to capture)
        p = inputs.c2(T=2000)
        dtype = rswr.F64 if which == "paper64" else rswr.F32
        td = torch.float64 if dtype == rswr.F64 else torch.float32
        plan = rswr.Plan.from_problem(p, dtype=dtype)
        if span is not None:
            plan.set_span(span)
        if variant is not None:
            plan.set_variant(variant)
        fA = torch.as_tensor(p.fA, device="cuda").to(td)
        for _ in range(2):
            r = plan.run_paper(fA, None, p.T)
        torch.cuda.synchronize()
        plan.check()
        print(json.dumps({"profile_case": which, "nx": p.nx, "T": p.T, "spans": len(r["spans"]), "info": plan.info()}))
        return
    if which in ("adj64", "adj32"):
        # the c4 gradient workload (dL/dfA and dL/da), run twice; a smaller grid
        # (log2_nx < 20) scales the steps with it
        if log2_nx >= 20:
            p = inputs.c4(j_r=4000)
        else:
            sh = 20 - log2_nx
            p = inputs.c4(T=8192 >> sh, nx=1 << log2_nx, j_r=4000 >> sh)
        dtype = rswr.F64 if which == "adj64" else rswr.F32
        td = torch.float64 if dtype == rswr.F64 else torch.float32
        plan = rswr.Plan.from_problem(p, dtype=dtype)
        if span is not None:
            plan.set_span(span)
        if variant is not None:
            plan.set_variant(variant)  # e.g. the resident variant the bench's autotuner picks on c4
        fA = torch.as_tensor(p.fA, device="cuda").to(td)
        w = torch.as_tensor(inputs.lowpass_noise(p.T, seed=4), device="cuda").to(td)
        for _ in range(2):
            plan.adjoint(fA, None, p.T, p.meta["j_r"], w, want_a=True)
        torch.cuda.synchronize()
        plan.check()
        print(json.dumps({"profile_case": which, "nx": p.nx, "T": p.T, "info": plan.info()}))
        return
    if full:
        p = inputs.c2()
    else:
        p = inputs.c2(T=1280, nx=1 << log2_nx)
        p = dataclasses.replace(p, n_sub=max(1, p.nx // 16384))
    plan = rswr.Plan.from_problem(p, dtype=rswr.F64 if which == "f64" else rswr.F32)
    if span is not None:
        plan.set_span(span)
    if variant is not None:
        plan.set_variant(variant)
    for _ in range(2):
        plan.run(p.fA, p.fB, p.T, traces=not NO_TRACES)
    torch.cuda.synchronize()
    plan.check()
    print(json.dumps({"profile_case": which, "nx": p.nx, "T": p.T, "traces": not NO_TRACES, "info": plan.info()}))


# ----------------------------------------------------------------------------
# extra measurements: batched (c3), adjoint (c4), large grid (c5)
# ----------------------------------------------------------------------------

def _time(torch, fn, reps):
    stream = torch.cuda.current_stream()
    ms = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    return ms


def bench_batched(torch, rank, world, dist, dev):
    """4096 independent problems (nx in [2^10, 2^18], CFL 0.8, 4096 steps,
    overlap 32), FP32, one persistent launch per run; problems sharded across
    ranks by size."""
    from paper_2203_10477_gb300 import rswr
    from paper_2203_10477_gb300.shard import max_over_ranks, shard_problems, sum_over_ranks

    probs = inputs.c3_problems()
    T = probs[0].T
    mine = [probs[i] for i in shard_problems([p.nx for p in probs], rank, world)]
    b = rswr.Batch(mine, dtype=rswr.F32, device=dev)
    b.autotune(64)
    fA = torch.as_tensor(np.concatenate([p.fA for p in mine]), device=dev).to(torch.float32)
    n = int(b.offsets[-1])
    out = (torch.empty(n, dtype=torch.float32, device=dev), torch.empty(n, dtype=torch.float32, device=dev))
    run = lambda: b.run(fA, None, T, out=out)
    run()
    ms = _time(torch, run, 2)
    b.check()
    lups = float(sum((p.nx - 2) * T for p in mine))
    t = max_over_ranks([sum(ms) / len(ms) / 1e3], dist, dev)[0]
    tot = sum_over_ranks([lups], dist, dev)[0]
    info = b.info()
    # checker leg: every problem of this rank against the FP64 oracle on its causal prefix
    err = batch_state_error(out[0], b.offsets, mine)
    return {"workload": "4096 problems, nx U[2^10,2^18], a U[0.5,2], CFL 0.8, 4096 steps, overlap 32, FP32",
            "value": tot / t / 1e9, "unit": UNIT, "ms_per_run": 1e3 * t, "lups_per_run": tot,
            "variant": info["variant"], "span_steps": info["span_steps"], "mode": info["mode"],
            "sharding": f"{world} rank(s), whole problems per rank",
            "roofline": span_roofline("f32", tot / t / 1e9 / world, 4, info),
            "error_vs_fp64_oracle": dict(err, note="max over every problem of this rank, causal prefix "
                                                    "j <= T + 1 (or the whole grid when shorter)")}


def bench_adjoint(torch, dev):
    """c4 gradients (nx = 2^20, a = 1.3, CFL 0.9, 8192 steps, N = 256, overlap
    64; receiver j_r = 4000): dL/dfA and dL/da with checkpoints and in-kernel
    recompute.  GLUP/s counts the forward problem's updates per gradient."""
    from paper_2203_10477_gb300 import rswr

    p = inputs.c4(j_r=4000)
    res = {}
    w = torch.as_tensor(inputs.lowpass_noise(p.T, seed=4), device=dev)
    for name, dtype in (("f64", rswr.F64), ("f32", rswr.F32)):
        plan = rswr.Plan.from_problem(p, dtype=dtype, device=dev)
        # variant, mode and span of the sweeps through the span kernel, timed on
        # 16 spans (a few spans would mostly time the start of a launch)
        plan.autotune(512)
        td = torch.float64 if dtype == rswr.F64 else torch.float32
        fA = torch.as_tensor(p.fA, device=dev).to(td)
        wt = w.to(td)
        last = {}

        def full():
            last["r"] = plan.adjoint(fA, None, p.T, 4000, wt, want_a=True)

        gonly = lambda: plan.adjoint(fA, None, p.T, 4000, wt, want_a=False)
        fwd_keep = lambda: plan.run_keep(fA, None, p.T, j_r=4000)
        full()
        gonly()
        ms_full = _time(torch, full, 2)
        ms_g = _time(torch, gonly, 2)
        # the training pattern: a forward run that keeps its span states, then the gradient
        ms_keep, ms_after = [], []
        for _ in range(2):
            ms_keep += _time(torch, fwd_keep, 1)
            ms_after += _time(torch, full, 1)
        plan.check()
        lups = (p.nx - 2) * p.T
        v_full = lups / (min(ms_full) / 1e3) / 1e9
        v_g = lups / (min(ms_g) / 1e3) / 1e9
        res[name] = {"grad_fA_and_a": {"value": v_full, "ms": min(ms_full),
                                       "roofline": alu_roofline(name, v_full, ADJ_OPS[name]["full"])},
                     "grad_fA_only": {"value": v_g, "ms": min(ms_g),
                                      "roofline": alu_roofline(name, v_g, ADJ_OPS[name]["g"])}}
        v_after = lups / (min(ms_after) / 1e3) / 1e9
        v_pair = lups / ((min(ms_keep) + min(ms_after)) / 1e3) / 1e9
        res[name]["grad_fA_and_a_after_kept_forward"] = {
            "value": v_after, "ms": min(ms_after), "roofline": alu_roofline(name, v_after, ADJ_OPS[name]["after_keep"]),
            "kept_forward_ms": min(ms_keep), "forward_and_gradient_value": v_pair,
            "note": "rswr_run_keep (forward, span states kept) then rswr_adjoint with dL/da, which skips its "
                    "checkpoint sweep; value counts the gradient call alone"}
        # checker leg: the gradients of the last timed run against the FP64 oracle's adjoint
        g = last["r"]["grad_fA"].double().cpu().numpy()
        ga = float(last["r"]["grad_a"][0])
        chk = grad_error(g, ga, p, 4000, inputs.lowpass_noise(p.T, seed=4))
        ref = chk.pop("_ref")
        if name == "f64":
            chk = {"grad_fA_bitwise_equal_to_oracle": bool(np.array_equal(g, ref["dg"])),
                   "grad_a_err_of_sum_abs_terms": chk["grad_a_err_vs_fp64_of_sum_abs_terms"]}
        res[name]["check"] = chk
        res[name]["variant"] = plan.info()["variant"]
        res[name]["mode"] = plan.info()["mode"]
        res[name]["span_steps"] = plan.info()["span_steps"]
    res["unit"] = UNIT
    res["workload"] = "c4: nx=2^20, a=1.3, CFL 0.9, 8192 steps, N=256, overlap 64, receiver j_r=4000"
    return res


def bench_large(torch, dev):
    """c5 grid: nx = 2^28 FP32, N = 8192, overlap 64, 2^15 steps (8.8e12 updates)."""
    from paper_2203_10477_gb300 import rswr

    p = inputs.c5_big()
    plan = rswr.Plan.from_problem(p, dtype=rswr.F32, device=dev)
    plan.autotune(64)
    fA = torch.as_tensor(p.fA, device=dev).to(torch.float32)
    out = (torch.empty(p.nx, dtype=torch.float32, device=dev), torch.empty(p.nx, dtype=torch.float32, device=dev))
    run = lambda: plan.run(fA, None, p.T, out=out)
    run()
    ms = _time(torch, run, 1)
    plan.check()
    lups = (p.nx - 2) * p.T
    info = plan.info()
    err = state_error(out[0], p)  # checker leg, outside the timed region
    del out
    v = lups / (ms[0] / 1e3) / 1e9
    return {"workload": "c5: nx=2^28 FP32, N=8192, overlap 64, 2^15 steps", "value": v,
            "unit": UNIT, "ms_per_run": ms[0], "variant": info["variant"], "span_steps": info["span_steps"],
            "roofline": span_roofline("f32", v, 4, info),
            "error_vs_fp64_oracle": dict(err, note="causal prefix j <= T + 1")}


def bench_c5_batch(torch, rank, world, dist, dev):
    """c5, second part: 512 uneven problems (nx in [2^12, 2^20], a in [0.5, 2],
    CFL 0.9, overlap 64, 2^15 steps) in one persistent launch, FP32: the forward
    run and the adjoint sweep that gives every problem's boundary-waveform
    gradient for a smooth receiver cotangent.  Problems sharded across ranks."""
    from paper_2203_10477_gb300 import rswr
    from paper_2203_10477_gb300.shard import max_over_ranks, shard_problems, sum_over_ranks

    probs = inputs.c5_uneven()
    T = probs[0].T
    idx = shard_problems([q.nx for q in probs], rank, world)
    mine = [probs[i] for i in idx]
    b = rswr.Batch(mine, dtype=rswr.F32, device=dev)
    b.autotune(64)
    fA = torch.as_tensor(np.concatenate([q.fA for q in mine]), device=dev).to(torch.float32)
    n = int(b.offsets[-1])
    out = (torch.empty(n, dtype=torch.float32, device=dev), torch.empty(n, dtype=torch.float32, device=dev))
    run = lambda: b.run(fA, None, T, out=out)
    run()
    ms_f = _time(torch, run, 1)[0]
    b.check()
    jr = [q.meta["j_r"] for q in mine]
    w64 = [inputs.lowpass_noise(T, seed=1000 + i) for i in idx]
    wbar = torch.as_tensor(np.stack(w64), device=dev).to(torch.float32)
    last = {}

    def adj():
        last["r"] = b.adjoint(fA, None, T, jr, wbar)

    adj()
    ms_a = _time(torch, adj, 1)[0]
    b.check()
    info = b.info()
    lups = float(sum((q.nx - 2) * T for q in mine))
    t_f, t_a = max_over_ranks([ms_f / 1e3, ms_a / 1e3], dist, dev)
    tot = sum_over_ranks([lups], dist, dev)[0]
    # checker leg: a spread sample of the problems (by size) against the FP64 oracle
    order = sorted(range(len(mine)), key=lambda i: mine[i].nx)
    fwd_idx = [order[k] for k in np.linspace(0, len(order) - 1, min(16, len(order))).round().astype(int)]
    err_f = batch_state_error(out[0], b.offsets, mine, sorted(set(fwd_idx)))
    adj_idx = sorted(set(order[k] for k in np.linspace(0, len(order) - 1, min(4, len(order))).round().astype(int)))
    g = last["r"]["grad_fA"]
    errs = host_map(lambda i: grad_error(g[i].double().cpu().numpy(), None, mine[i], jr[i], w64[i],
                                         want_a=False)["grad_fA_err_vs_fp64"], adj_idx)
    del out, wbar, last
    return {"workload": "c5: 512 uneven problems, nx U[2^12,2^20], a U[0.5,2], CFL 0.9, overlap 64, 2^15 steps, FP32",
            "unit": UNIT, "lups_per_run": tot,
            "forward": {"value": tot / t_f / 1e9, "ms_per_run": t_f * 1e3,
                        "roofline": span_roofline("f32", tot / t_f / 1e9, 4, info),
                        "error_vs_fp64_oracle": dict(err_f, note="16 problems spread over the sizes, causal prefix")},
            "adjoint_grad_fA": {"value": tot / t_a / 1e9, "ms_per_run": t_a * 1e3,
                                "roofline": span_roofline("f32", tot / t_a / 1e9, 4, info),
                                "error_vs_fp64_oracle": {"grad_fA_err_vs_fp64": max(errs),
                                                         "per_problem": errs, "problems_checked": len(adj_idx),
                                                         "norm": "relative 2-norm"}},
            "variant": info["variant"], "span_steps": info["span_steps"], "mode": info["mode"],
            "sharding": f"{world} rank(s), whole problems per rank"}


def bench_paper_literal(torch, dev, T=2000):
    """The paper-literal RSWR (data-chosen spans, flux-exchange update) on the
    c2 grid (nx = 2^24, N = 1024, overlap 64, CFL 0.9) for 2000 steps."""
    from paper_2203_10477_gb300 import rswr

    p = inputs.c2(T=T)
    res = {"workload": "c2 grid, 2000 steps, paper-literal select/update", "unit": UNIT}
    for name, dtype in (("f64", rswr.F64), ("f32", rswr.F32)):
        plan = rswr.Plan.from_problem(p, dtype=dtype, device=dev)
        plan.autotune(64)  # the span kernel that advances the grid each span
        td = torch.float64 if dtype == rswr.F64 else torch.float32
        fA = torch.as_tensor(p.fA, device=dev).to(td)
        out = (torch.empty(p.nx, dtype=td, device=dev), torch.empty(p.nx, dtype=td, device=dev))
        plan.run_paper(fA, None, 64, out=out)
        t0 = time.perf_counter()
        r = plan.run_paper(fA, None, p.T, out=out)
        secs = time.perf_counter() - t0
        v = (p.nx - 2) * p.T / secs / 1e9
        # the pipe bound of the updates themselves: the select predictions and the
        # zone re-solves add under 2 % to them on this grid (2 x 1023 interfaces x
        # about 40 points next to the input boundaries per span)
        res[name] = {"value": v, "seconds": secs, "spans": int(len(r["spans"])),
                     "mean_span": float(np.mean(r["spans"])),
                     "roofline": alu_roofline(name, v, 3 if name == "f64" else 4)}
        m, ref = prefix_ref(p)
        u = out[0][:m].double().cpu().numpy()
        if name == "f64":
            res[name]["err_vs_monolithic_oracle"] = rel_max(u, ref)
        else:
            res[name]["error_vs_fp64_oracle"] = {"err_vs_fp64": rel_max(u, ref), "note": "causal prefix"}
    return res


def bench_pulse10(torch, dev, T=10_000):
    """The N = 10 pulse-source experiment (Sec. 4) on a 2^24-point grid: N = 10
    subdomains, overlap 64, CFL 0.9, zero Dirichlet data, ten Gaussian pulse
    sources at the centres of ten equal cells (inputs.pulse_experiment).  RSWR
    (FP64 canonical, FP32 increment) against the monolithic solve with the same
    sources; the two final states are compared bit for bit on the device."""
    from paper_2203_10477_gb300 import rswr

    p, j, s = inputs.pulse_experiment(nx=1 << 24, T=T)
    res = {"workload": "pulse10: nx=2^24, N=10 subdomains, overlap 64, CFL 0.9, 10^4 steps, 10 pulse sources",
           "unit": UNIT, "sources": [int(x) for x in j]}
    lups = (p.nx - 2) * p.T
    for name, dtype, ops in (("f64", rswr.F64, 3), ("f32", rswr.F32, 4)):
        plan = rswr.Plan.from_problem(p, dtype=dtype, device=dev)
        td = torch.float64 if dtype == rswr.F64 else torch.float32
        plan.autotune(64)
        plan.set_sources(j, torch.as_tensor(s, device=dev).to(td))
        out = (torch.empty(p.nx, dtype=td, device=dev), torch.empty(p.nx, dtype=td, device=dev))
        ref = (torch.empty(p.nx, dtype=td, device=dev), torch.empty(p.nx, dtype=td, device=dev))
        run = lambda: plan.run(None, None, p.T, out=out)
        mono = lambda: plan.mono(None, None, p.T, out=ref)
        run()
        ms = min(_time(torch, run, 2))
        mono()
        ms_mono = min(_time(torch, mono, 1))
        plan.check()
        v = lups / (ms / 1e3) / 1e9
        info = plan.info()
        res[name] = {"value": v, "ms_per_run": ms, "monolithic": lups / (ms_mono / 1e3) / 1e9,
                     "monolithic_ms": ms_mono, "bitwise_equal_to_monolithic": bool(torch.equal(out[0], ref[0])
                                                                                   and torch.equal(out[1], ref[1])),
                     "max_abs_u": float(out[0].abs().max()), "variant": info["variant"],
                     "span_steps": info["span_steps"], "roofline": span_roofline(name, v, ops, info)}
        if name == "f32":
            res[name]["error_vs_fp64_oracle"] = pulse10_error(out[0], p, j, s)
        del out, ref
    return res


def bench_split_step(torch, sp, p, flush, dist):
    """One whole c2 run split over the ranks (SplitPlan), the waveforms already
    on the device; seconds between two barriers, with a device
    synchronisation on both sides."""
    fA = torch.as_tensor(p.fA).to(device=sp.device, dtype=sp.tdtype)
    fB = torch.as_tensor(p.fB).to(device=sp.device, dtype=sp.tdtype)
    flush.zero_()
    torch.cuda.synchronize()
    dist.barrier()
    t0 = time.perf_counter()
    res = sp.run(fA, fB, p.T)
    torch.cuda.synchronize()
    dist.barrier()
    return time.perf_counter() - t0, res


def main_split(args, torch, rank, world, dist, dev):
    """--gpus N > 1: the c2 problem split over the N ranks (paper Sec. 3
    subdomains in a row; a halo exchange between neighbouring ranks every 128
    steps, i.e. every 4 spans of 32), the whole job's GLUP/s at a fixed total
    work (strong scaling).  The sharded batch extras run beside it."""
    from paper_2203_10477_gb300 import rswr
    from paper_2203_10477_gb300.shard import max_over_ranks
    from paper_2203_10477_gb300.split import SplitPlan

    p = inputs.c2()
    lups = (p.nx - 2) * p.T
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    res = {}
    for name, dtype in (("f64", rswr.F64), ("f32", rswr.F32)):
        sp = SplitPlan.from_problem(p, rank, world, dist, dtype=dtype, halo=128, device=dev)
        for _ in range(args.warmup):
            bench_split_step(torch, sp, p, flush, dist)
        clocks = ClockSampler(gpu_uuid(torch, dev)) if name == "f64" else None
        if clocks:
            clocks.start()
            time.sleep(0.3)
        secs = []
        for _ in range(args.steps):
            t, out = bench_split_step(torch, sp, p, flush, dist)
            secs.append(t)
        clk = clocks.stop() if clocks else None
        t = max_over_ranks([sum(secs)], dist, dev)[0]
        # checker leg: the gathered final state against the FP64 oracle on the causal prefix
        u = sp.gather(out["u"])
        chk = None
        if rank == 0:
            m, ref = prefix_ref(p)
            uu = u[:m].double().cpu().numpy()
            chk = ({"bitwise_equal_to_oracle": bool(np.array_equal(uu, ref))} if name == "f64"
                   else {"err_vs_fp64": rel_max(uu, ref)})
            chk["nonzero_beyond_prefix"] = int((u[m:] != 0).sum())
        res[name] = {"value": lups * args.steps / t / 1e9, "ms_per_step": 1e3 * t / args.steps, "check": chk,
                     "exchanged_bytes_per_step": sp.exchanged_bytes / (args.steps + args.warmup), "clocks": clk}
        # end to end: host waveforms in, the owned state out, every step
        if name == "f64":
            e2e = []
            for _ in range(max(1, min(args.steps, 3))):
                torch.cuda.synchronize()
                dist.barrier()
                t0 = time.perf_counter()
                o = sp.run(p.fA, p.fB, p.T)
                o["u"].cpu()
                o["w"].cpu()
                dist.barrier()
                e2e.append(time.perf_counter() - t0)
            t_e2e = max_over_ranks([sum(e2e) / len(e2e)], dist, dev)[0]
            res["e2e"] = {"value": lups / t_e2e / 1e9, "unit": UNIT, "h2d_bytes_per_step": 2 * (p.T + 1) * 8,
                          "d2h_bytes_per_step": 2 * (sp.blk.c1 - sp.blk.c0) * 8,
                          "path": "SplitPlan.run from host waveforms, owned state pair copied to the host"}
        del sp
        torch.cuda.empty_cache()
    v64 = res["f64"]["value"]
    line = {
        "metric": METRIC, "value": v64, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": res["f64"]["ms_per_step"], "higher_is_better": True, "scaling": "strong",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "nx": p.nx, "n_sub": p.n_sub, "overlap": p.overlap, "cfl": 0.9, "T": p.T,
                   "lups_per_step": lups, "parallelism": f"one problem split over {world} ranks: contiguous blocks "
                   f"of subdomains, halo of 128 points exchanged between neighbouring ranks every 128 steps (NCCL)",
                   "l2": "flushed between steps (256 MiB write); state > L2"},
        "pct_stencil_roofline": 100.0 * v64 / world / (load_peaks()["hbm_gbs"] / 24.0),
        "roofline": {"bound": "alu", "kernel": "span_kernel<double, canonical> (all ranks)",
                     "achieved": v64 / world, "peak": alu_roofline("f64", 1.0, 3)["peak"], "unit": "GLUP/s",
                     "frac": v64 / world / alu_roofline("f64", 1.0, 3)["peak"], "traffic": None,
                     "note": "per GPU from the whole-step time (barrier to barrier), not kernel events"},
        "check_vs_oracle": res["f64"]["check"],
        "f32": res["f32"],
        "e2e": res["e2e"],
        "gpu_launches": 2 * -(-p.T // 128) * args.steps,
        "gpu_launches_detail": "per rank and timed FP64 run: one set_boundary_kernel and one persistent span "
                               "kernel per round of 128 steps",
        "clocks": res["f64"]["clocks"],
    }
    if not args.no_extras:
        line["batched"] = bench_batched(torch, rank, world, dist, dev)
        torch.cuda.empty_cache()
        line["large_batch"] = bench_c5_batch(torch, rank, world, dist, dev)
    if rank == 0:
        print(json.dumps(line), flush=True)
    dist.barrier()
    dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mono", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the batched / adjoint / large-grid measurements")
    ap.add_argument("--profile-case", choices=["f64", "f32", "adj64", "adj32", "g32", "c3", "paper64", "paper32"],
                    default=None,
                    help="run a small profiling case twice and exit (for ncu): f64/f32 nx=2^22, 1280 steps; "
                         "adj64/adj32 the c4 gradient; c3 the first 1024 batched problems, 256 steps; "
                         "paper64/paper32 the paper-literal run on the c2 grid, 2000 steps")
    ap.add_argument("--variant", type=int, default=None, help="kernel variant of the profiling case")
    ap.add_argument("--profile-log2-nx", type=int, default=None,
                    help="grid of the profiling case: 2^N points (default 22; 24 = the bench grid; "
                         "adj64/adj32: default 20 = the c4 grid)")
    ap.add_argument("--span", type=int, default=None, help="steps per span of the profiling case")
    ap.add_argument("--full", action="store_true", help="profiling case at the bench's full size")
    ap.add_argument("--no-traces", action="store_true", help="profiling case without the interface traces")
    ap.add_argument("--peaks", action="store_true",
                    help="measure the FP64 / FP32 pipe rates with the library's FMA probe kernel and exit")
    args = ap.parse_args()

    if args.profile_case:
        global NO_TRACES
        NO_TRACES = args.no_traces
        lg = args.profile_log2_nx
        if lg is None:
            lg = 20 if args.profile_case in ("adj64", "adj32", "g32") else 22
        profile_case(args.profile_case, args.variant, args.span, args.full, lg)
        return

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch

    global SM_COUNT
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    SM_COUNT = torch.cuda.get_device_properties(dev).multi_processor_count
    if args.peaks:
        from paper_2203_10477_gb300 import build

        build.build()
        m = measure_alu(torch, dev)
        print(json.dumps({"peaks": "FMA throughput of the FP64 and FP32 pipes (rswr_fma_probe)", "sms": SM_COUNT,
                          "f64_fma_per_s": m["f64"]["fma_per_s"], "f32_fma_per_s": m["f32"]["fma_per_s"],
                          "f64_per_sm_per_clock": m["f64"]["per_sm_per_clock"],
                          "f32_per_sm_per_clock": m["f32"]["per_sm_per_clock"],
                          "f32x2_lanes_per_sm_per_clock": m["f32x2"]["per_sm_per_clock"],
                          "f32x2_add_lanes_per_sm_per_clock": m["f32x2_add"]["per_sm_per_clock"],
                          "f64_glups_at_3_instr": m["f64"]["fma_per_s"] / 3 / 1e9,
                          "f32_glups_at_4_instr": m["f32"]["fma_per_s"] / 4 / 1e9,
                          "detail": m}), flush=True)
        return
    dist = None
    if world > 1:
        import torch.distributed as dist_

        dist_.init_process_group("nccl", device_id=dev)
        dist = dist_

    from paper_2203_10477_gb300 import build, rswr

    build.build()
    if world > 1:
        main_split(args, torch, rank, world, dist, dev)
        return
    alu_measured = measure_alu(torch, dev)
    MEASURED_ALU.update({k: alu_measured[k] for k in ("f64", "f32")})
    p = inputs.c2()
    lups = (p.nx - 2) * p.T
    peaks = load_peaks()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # 256 MiB > 129 MB L2

    plan64 = rswr.Plan.from_problem(p, dtype=rswr.F64, device=dev)
    plan32 = rswr.Plan.from_problem(p, dtype=rswr.F32, device=dev)
    v64 = plan64.autotune(3 * 32)
    v32 = plan32.autotune(3 * 32)
    info64, info32 = plan64.info(), plan32.info()

    b64, b32 = RunBench(torch, plan64, p), RunBench(torch, plan32, p)
    b64.warmup(args.warmup)
    b32.warmup(args.warmup)

    clocks = ClockSampler(gpu_uuid(torch, dev))
    clocks.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    run64, ker64 = b64.timed(args.steps, flush)
    run32, ker32 = b32.timed(args.steps, flush)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()

    # checker leg (outside the timed region): the last timed runs against the
    # FP64 oracle on the causal prefix j <= T + 1
    m_pre, ref_pre = prefix_ref(p)
    u64 = b64.out[0][:m_pre].cpu().numpy()
    check64 = {"bitwise_equal_to_oracle": bool(np.array_equal(u64, ref_pre)),
               "nonzero_beyond_prefix": int((b64.out[0][m_pre:] != 0).sum()), "prefix_points": m_pre}
    err32 = state_error(b32.out[0], p)

    from paper_2203_10477_gb300.shard import max_over_ranks

    t64, t32 = max_over_ranks([sum(run64) / 1e3, sum(run32) / 1e3], dist, dev)
    n = world
    value64 = n * lups * args.steps / t64 / 1e9
    value32 = n * lups * args.steps / t32 / 1e9

    mono = {}
    if not args.no_mono:
        for name, dtype in (("f64", rswr.F64), ("f32", rswr.F32)):
            pl = plan64 if dtype == rswr.F64 else plan32
            ms = mono_runs(torch, pl, p, 1, flush)
            mono[name] = {"value": lups / (sum(ms) / 1e3) / 1e9, "unit": UNIT, "ms_per_step": sum(ms) / len(ms),
                          "form": "canonical" if dtype == rswr.F64 else "increment"}

    e2e_ms, h2d, d2h = e2e_run(torch, plan64, p, max(1, min(args.steps, 3)))
    e2e_value = lups / (sum(e2e_ms) / len(e2e_ms) / 1e3) / 1e9

    sm_mhz = clk["sm_mhz"] if clk else SM_MAX_MHZ
    alu_max = alu_peaks(SM_MAX_MHZ)
    alu_run = alu_peaks(sm_mhz)
    r_hbm = {"f64": peaks["hbm_gbs"] / 24.0, "f32": peaks["hbm_gbs"] / 12.0}

    # span kernel (the dominant kernel): achieved LUP rate over its own launches
    k64 = lups / (statistics.mean(ker64) / 1e3) / 1e9
    k32 = lups / (statistics.mean(ker32) / 1e3) / 1e9
    # algorithmic bytes per LUP of RSWR with the subdomain geometry:
    # w * (2 (core + ov) + 2 core) / (core * S), core = nx / N
    core_sub = p.nx / p.n_sub
    bpl = lambda w, S: w * (2 * (core_sub + p.overlap) + 2 * core_sub) / (core_sub * S)

    line = {
        "metric": METRIC,
        "value": value64,
        "unit": UNIT,
        "n_gpus": n,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": 1e3 * t64 / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "nx": p.nx, "n_sub": p.n_sub, "overlap": p.overlap, "cfl": 0.9,
                   "T": p.T, "span_steps": info64["span_steps"], "lups_per_step": lups,
                   "traces": "all 1023 interfaces x 2 output waveforms per level",
                   "l2": "flushed between steps (256 MiB write); state > L2",
                   "variant_f64": {k: info64[k] for k in ("variant", "points_per_thread", "threads_per_cta",
                                                            "window", "core", "mode", "span_steps")},
                   "variant_f32": {k: info32[k] for k in ("variant", "points_per_thread", "threads_per_cta",
                                                            "window", "core", "mode", "span_steps")},
                   "replicas": "one independent replica per GPU" if n > 1 else None},
        "pct_stencil_roofline": 100.0 * value64 / n / r_hbm["f64"],
        "stencil_roofline": {"f64_glups": r_hbm["f64"], "f32_glups": r_hbm["f32"],
                             "definition": "HBM-bound untiled leapfrog: measured copy GB/s / (3 w) bytes per LUP",
                             "hbm_gbs": peaks["hbm_gbs"], "source": peaks["source"]},
        "roofline": {"bound": "alu", "kernel": "span_kernel<double, canonical>",
                     "achieved": k64, "peak": alu_max["f64"], "unit": "GLUP/s",
                     "frac": k64 / alu_max["f64"], "frac_at_run_clock": k64 / alu_run["f64"],
                     "traffic": (lambda b: None if b is None else b * lups)(
                         measured_traffic("f64", info64["variant"], info64["span_steps"])),
                     "traffic_source": "profiles/traffic_span_kernel_c2.md (bytes/update x updates per launch)",
                     "algorithmic_bytes_per_lup": bpl(8, info64["span_steps"]),
                     "achieved_gbs": k64 * bpl(8, info64["span_steps"]),
                     "peak_definition": f"{SM_COUNT} SMs x 2 FP64 instr/clk x 2070 MHz / 3 FP64 instr per LUP",
                     "peak_measured": alu_measured["f64"]["fma_per_s"] / 3 / 1e9,
                     "frac_of_measured": k64 / (alu_measured["f64"]["fma_per_s"] / 3 / 1e9),
                     "peak_measured_definition": "rswr_fma_probe FP64 FMA/s / 3 FP64 instr per LUP"},
        "check_vs_oracle": check64,
        "f32": {"value": value32, "unit": UNIT, "ms_per_step": 1e3 * t32 / args.steps, "form": "increment",
                "pct_stencil_roofline": 100.0 * value32 / n / r_hbm["f32"],
                "error_vs_fp64_oracle": dict(err32, note="max |u32 - u64| / max |u64| of the last timed run "
                                                         "on the causal prefix j <= T + 1"),
                "roofline": {"bound": "alu", "kernel": "span_kernel<float, increment>", "achieved": k32,
                             "peak": alu_max["f32"], "unit": "GLUP/s", "frac": k32 / alu_max["f32"],
                             "frac_at_run_clock": k32 / alu_run["f32"],
                             "traffic": (lambda b: None if b is None else b * lups)(
                                 measured_traffic("f32", info32["variant"], info32["span_steps"])),
                             "algorithmic_bytes_per_lup": bpl(4, info32["span_steps"]),
                             "achieved_gbs": k32 * bpl(4, info32["span_steps"]),
                             "peak_definition": f"{SM_COUNT} SMs x 128 FP32 lanes x 2070 MHz / 4 FP32 instr per LUP",
                             "peak_measured": alu_measured["f32"]["fma_per_s"] / 4 / 1e9,
                             "frac_of_measured": k32 / (alu_measured["f32"]["fma_per_s"] / 4 / 1e9)}},
        "alu_measured": {k: {kk: alu_measured[k][kk] for kk in ("fma_per_s", "per_sm_per_clock", "ms")}
                         for k in ("f64", "f32")},
        "monolithic": mono,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "path": "rswr_run_host (C ABI, pinned host buffers, copies inside the timed region)"},
        "gpu_launches": 3 * 2 * args.steps,
        "gpu_launches_detail": "per timed run: set_boundary_kernel + span_kernel (persistent: one launch for all "
                               "313 spans) + probe_final_kernel; FP64 and FP32 runs",
        "clocks": clk,
    }
    if not args.no_extras:
        del b64, b32
        torch.cuda.empty_cache()
        line["batched"] = bench_batched(torch, rank, world, dist, dev)
        torch.cuda.empty_cache()
        line["adjoint"] = bench_adjoint(torch, dev)
        torch.cuda.empty_cache()
        line["large_grid"] = bench_large(torch, dev)
        torch.cuda.empty_cache()
        line["large_batch"] = bench_c5_batch(torch, rank, world, dist, dev)
        torch.cuda.empty_cache()
        line["paper_literal"] = bench_paper_literal(torch, dev)
        torch.cuda.empty_cache()
        line["pulse10"] = bench_pulse10(torch, dev)
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(p)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
