#!/usr/bin/env python
"""Benchmark: node-updates/s of the local RBF-SL step on one GB300 (mixed and FP64).

Workload (one "step" = one SL step of Algorithm 1: RK4 departure points, k-NN stencils,
FP64 saddle-point weights, gather-dot W.q over all tracers): N = 40,962 Fibonacci nodes
(1e-3 rad jitter), stencils of n = 84 nearest nodes of each departure point, PHS r^9,
spherical harmonics to degree 4, reversing deformational flow psi = 2.4 y^2 cos(pi t) over
600 steps (T_f = 1), 32 tracers (one field of two Gaussian hills + 31 smooth random fields). Mixed
precision = FP64 solves, FP32 stage increments in the tracer, weights and fields as FP32 pairs
with the W.q sum in pair arithmetic.

The L2 cache (129 MB) is flushed between timed steps by writing a 256 MB buffer, so every
step starts cold. Prints one JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "node-updates/s per SL step, mixed vs FP64 at equal l2 err; p50/p99 solve latency"
UNIT = "node-updates/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--accuracy-steps", type=int, default=600,
                    help="steps of the full-trajectory accuracy runs (0 = skip)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the 64-problem batched measurement")
    ap.add_argument("--no-served", action="store_true", help="skip the served (Poisson arrivals) measurement")
    ap.add_argument("--served-requests", type=int, default=128, help="requests of the served leg")
    ap.add_argument("--served-steps", type=int, nargs=2, default=[50, 120], metavar=("MIN", "MAX"),
                    help="steps per served request, drawn uniformly from [MIN, MAX]")
    ap.add_argument("--case", default=None, choices=["weights", "gather", "knn", "trace", "center", "wq", "tceval",
                                                  "cardinal", "served", "batched"],
                    help="run one kernel of the workload on --nq points (for profilers); no JSON")
    ap.add_argument("--nq", type=int, default=3040)
    ap.add_argument("--repeat", type=int, default=3)
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def job_seconds(local_seconds, world, device="cuda"):
    """Wall time of the job's timed region: the maximum over the ranks of each rank's time
    (one all-reduce; NCCL on the GPUs, gloo on the host)."""
    if world <= 1:
        return float(local_seconds)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(local_seconds)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank, world, seconds):
    """Whole-job rate: the units every rank processed (replicas: world x one rank's) per
    second of the job's wall time."""
    return world * units_per_rank / seconds


def workload():
    from paper_1804_01609_gb300 import inputs
    return inputs.config_local_deformation()


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- helpers
def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


# FP64 ALU peak of a GB300: 152 SMs x 2 FP64 FMA/clk/SM x 2 flop x 2.07 GHz = 1.26 TFLOP/s
# (NVIDIA's 1.25 TFLOP/s FP64 figure for the part; the clock is the maximum SM clock).
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


# DRAM bytes (read + write) of one full-size launch of the DIRECT weights kernel, from one ncu
# capture (dram__bytes_read.sum + dram__bytes_write.sum) of the kernel version this file ships
# with; None when no capture of that version exists.
WEIGHTS_DRAM_BYTES = 15.802624e6 + 512


def weights_flops(m):
    """Algorithmic work of one m x m saddle-point solve with one right-hand side, the per-unit
    figure of the roofline: (2/3) m^3 + 2 m^2 FP64 flops (Gaussian elimination's count)."""
    return 2.0 / 3.0 * m ** 3 + 2.0 * m ** 2


def weights_kernel_flops(m):
    """FP64 flops the L D L^T kernel itself performs for that solve: (1/3) m^3 for the
    factorisation (m^3 / 6 FMAs), 2 m^2 for the forward and back substitutions."""
    return 1.0 / 3.0 * m ** 3 + 2.0 * m ** 2


def make_ctx(w, precision, stream, rbfsl, mode=None):
    ctx = rbfsl.Context(0, stream=stream)
    ctx.set_nodes(w.X)
    ctx.set_velocity(w.vel_kind, w.vel_params)
    ctx.set_method(rbfsl.LOCAL, rbfsl.DIRECT if mode is None else mode)
    ctx.set_stencil_size(w.n)
    ctx.set_sh_degree(w.ell)
    ctx.set_kernel(rbfsl.PHS, w.power)
    ctx.set_precision(precision)
    ctx.set_dt(w.dt)
    ctx.set_time(0.0)
    ctx.set_tracers(w.q0())  # FP64 field; the mixed step keeps it as FP32 pairs
    return ctx


def timed_steps(ctx, K, W, stream, flush, torch):
    for _ in range(W):
        ctx.step(1)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    for i in range(K):
        with torch.cuda.stream(stream):
            flush.fill_(float(i))
        ev[i][0].record(stream)
        ctx.step(1)
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    return np.array([a.elapsed_time(b) for a, b in ev])


def time_op(fn, K, stream, flush, torch):
    fn()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    for i in range(K):
        with torch.cuda.stream(stream):
            flush.fill_(float(i))
        ev[i][0].record(stream)
        fn()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    return float(np.mean([a.elapsed_time(b) for a, b in ev]))


def accuracy_run(w, precision, steps, stream, rbfsl, mode=None):
    ctx = make_ctx(w, precision, stream, rbfsl, mode)
    ctx.step(steps)
    q = ctx.get_q(dtype=np.float64)
    st = ctx.get_stats()
    ctx.close()
    return q, st


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def rel_linf(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def cpu_baseline(w, budget_s=10.0, single_budget_s=5.0):
    """The FP64 oracle as it stands, on this host's cores, over a bounded sample: departure
    points of one step for all nodes, then brute-force k-NN + GEPP weights + gather for the
    first S nodes, with S sized to ~budget_s of work; timed on all cores and on one core."""
    import oracle
    oracle.build()
    X = w.X
    q = w.q0()
    Xi = oracle.trace_rk4(X, w.vel_kind, w.vel_params, w.dt, w.dt)

    def timed(budget):
        S = 64
        t0 = time.perf_counter()
        oracle.local_apply(X, Xi[:S], q, w.n, w.ell, oracle.PHS, float(w.power))
        dt0 = time.perf_counter() - t0
        S = int(min(w.N, max(64, S * budget / max(dt0, 1e-3))))
        t0 = time.perf_counter()
        oracle.local_apply(X, Xi[:S], q, w.n, w.ell, oracle.PHS, float(w.power))
        return S, time.perf_counter() - t0

    oracle.set_threads(0)
    S, el = timed(budget_s)
    cores = oracle.num_threads()
    oracle.set_threads(1)
    S1, el1 = timed(single_budget_s)
    oracle.set_threads(0)
    return {"value": S / el, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{S} of {w.N} node-updates of one SL step (brute-force k-NN, GEPP, "
                      f"gather of {w.T} tracers; FP64 C + OpenMP); {el:.1f} s",
            "single_thread": {"value": S1 / el1, "unit": UNIT, "cores": 1,
                              "sample": f"{S1} node-updates of the same step, one thread; {el1:.1f} s"}}


# ----------------------------------------------------------------------------- W.q roofline
def morton_order(X, bits=10):
    """Node permutation along a 3-D Morton (Z-order) curve of the coordinates."""
    q = np.clip(((X + 1.0) * 0.5 * (1 << bits)).astype(np.int64), 0, (1 << bits) - 1)
    code = np.zeros(len(X), dtype=np.int64)
    for b in range(bits):
        for a in range(3):
            code |= ((q[:, a] >> b) & 1) << (3 * b + a)
    return np.argsort(code, kind="stable")


def pairs_of(a):
    """FP64 array -> FP32 pairs (hi, lo) in a trailing axis of 2, as the mixed step stores q."""
    hi = a.astype(np.float32)
    return np.ascontiguousarray(np.stack([hi, (a - hi.astype(np.float64)).astype(np.float32)], axis=-1))


def pairs_of_t(t):
    import torch
    hi = t.to(torch.float32)
    return torch.stack([hi, (t - hi.to(torch.float64)).to(torch.float32)], dim=-1).contiguous()


def bench_wq_hbm(rbfsl, torch, stream, flush, K=10):
    """The gather-dot W.q alone at a size where it is HBM-bound: N = 655,362 Morton-ordered
    Fibonacci nodes, n = 84 nearest-node stencils, T = 16 tracers; FP32 (difference form), FP64
    and FP32 pairs (the mixed step's storage and arithmetic). Algorithmic bytes per launch:
    N n (w + index) + 2 N T (read and write one row of q)."""
    from paper_1804_01609_gb300 import inputs
    N, n, T = 655362, 84, 16
    X = inputs.nodes(N, 1804 * 100 + 6)
    X = np.ascontiguousarray(X[morton_order(X)])
    x = torch.as_tensor(X, device="cuda")
    ix = rbfsl.rbfsl_knn_index_create(x, n, stream=stream)
    I = torch.empty((N, n), dtype=torch.int32, device="cuda")
    rbfsl.rbfsl_knn_query(ix, x, n, I, stream=stream)
    ix.close()
    g = torch.Generator(device="cuda").manual_seed(7)
    out = {}
    for name, dt, es in (("f32", torch.float32, 4), ("f64", torch.float64, 8), ("f32x2", None, 8)):
        with torch.cuda.stream(stream):
            W = torch.rand((N, n), generator=g, device="cuda", dtype=torch.float64)
            W = W / W.sum(1, keepdim=True)
            q = torch.rand((N, T), generator=g, device="cuda", dtype=torch.float64)
            if dt is None:  # FP32 pairs (the mixed-precision storage)
                W, q = pairs_of_t(W), pairs_of_t(q)
            else:
                W, q = W.to(dt), q.to(dt)
            qo = torch.empty_like(q)
        ms = time_op(lambda: rbfsl.rbfsl_gather_dot(I, W, q, qo, stream=stream, pairs=dt is None), K, stream,
                     flush, torch)
        by = N * n * (es + 4) + 2 * N * T * es
        out[name] = {"ms_per_launch": ms, "algorithmic_bytes": by, "achieved_gbs": by / (ms * 1e-3) / 1e9}
    return out


# ----------------------------------------------------------------------------- global RBF
def json_safe(o):
    """The JSON line must be strict JSON: non-finite floats (a diverged run) become null."""
    if isinstance(o, dict):
        return {k: json_safe(v) for k, v in o.items()}
    if isinstance(o, (list, tuple)):
        return [json_safe(v) for v in o]
    if isinstance(o, (float, np.floating)):
        return float(o) if np.isfinite(o) else None
    if isinstance(o, np.integer):
        return int(o)
    return o


def finite_or_none(v):
    v = float(v)
    return v if np.isfinite(v) else None


def global_ctx(rbfsl, w, prec, stream, eps=None, form=None, evaluation=None):
    ctx = rbfsl.Context(0, stream=stream)
    ctx.set_nodes(w.X)
    ctx.set_velocity(w.vel_kind, w.vel_params)
    ctx.set_method(rbfsl.GLOBAL)
    ctx.set_kernel(rbfsl.GAUSS, w.eps if eps is None else eps)
    ctx.set_precision(prec)
    if form is not None:
        ctx.set_global_form(form)
    if evaluation is not None:
        ctx.set_global_eval(evaluation)
    ctx.set_dt(w.dt)
    ctx.set_tracers(w.q0())
    return ctx


def bench_global_cardinal(rbfsl, torch, stream, flush, K=5, accuracy_eps=(6.0, 9.0, 24.0)):
    """The global workload (N = 10,242, 64 tracers, steady tilted rotation) in cardinal form:
    E = Phi(Xi, X) A_X^-1 formed once (FP64 LU, then 2 N^3 flops of triangular solves), each step
    q <- E q: 2 N^2 T = 13.4 GFLOP in FP64, or the same terms in FP32-pair arithmetic (~12 FP32
    operations each, 8.1e10 per step). Peaks derived from GB300's unit counts at 2,070 MHz:
    FP64 2 DFMA/clk/SM = 1.26 TFLOP/s; FP32 128 lanes/clk/SM = 40.3 T operations/s. Errors after
    one revolution (200 steps) against the exact solution for several eps."""
    from paper_1804_01609_gb300 import inputs
    w = inputs.config_global_rotation()
    N, T = w.N, w.T
    terms = float(N) * N * T
    peaks = {"fp64": 152 * 2 * 2 * 2.07e9, "mixed": 152 * 128 * 2.07e9}
    work = {"fp64": 2.0 * terms, "mixed": 12.0 * terms}
    out = {"eps": w.eps, "form": "cardinal"}
    for prec, name in ((rbfsl.FP64, "fp64"), (rbfsl.MIXED, "mixed")):
        ctx = global_ctx(rbfsl, w, prec, stream, form=rbfsl.GLOBAL_CARDINAL)
        t0 = time.perf_counter()
        ctx.step(1)
        torch.cuda.synchronize()
        setup = time.perf_counter() - t0
        ms = timed_steps(ctx, K, 1, stream, flush, torch)
        ctx.close()
        rate = work[name] / (float(ms.mean()) * 1e-3)
        out[name] = {"value": N / (float(ms.mean()) / 1e3), "ms_per_step": float(ms.mean()),
                     "setup_and_first_step_s": setup,
                     ("tflops" if name == "fp64" else "fp32_tops"): rate / 1e12,
                     "frac_of_derived_peak": rate / peaks[name]}
    q0 = w.q0()
    acc = []
    for eps in accuracy_eps:
        row = {"eps": eps}
        qs = {}
        for prec, name in ((rbfsl.FP64, "fp64"), (rbfsl.MIXED, "mixed")):
            ctx = global_ctx(rbfsl, w, prec, stream, eps, form=rbfsl.GLOBAL_CARDINAL)
            ctx.step(w.steps)
            qs[name] = ctx.get_q()
            ctx.close()
            ok = bool(np.isfinite(qs[name]).all())
            row[name + "_l2_vs_exact"] = finite_or_none(rel_l2(qs[name], q0)) if ok else None
        if row["fp64_l2_vs_exact"] is not None and row["mixed_l2_vs_exact"] is not None:
            row["mixed_over_fp64"] = row["mixed_l2_vs_exact"] / row["fp64_l2_vs_exact"]
            row["mixed_l2_vs_fp64"] = finite_or_none(rel_l2(qs["mixed"], qs["fp64"]))
        acc.append(row)
    out["accuracy_after_200_steps"] = acc
    return out


def bench_global(rbfsl, torch, stream, flush, K=3, accuracy_eps=(6.0, 9.0, 24.0)):
    """Global Gaussian RBF, N = 10,242, 64 smooth tracers, tilted rotation: one-time FP64 LU,
    then per step an FP64 solve and the evaluation at the departure points: FP64; mixed with
    split TF32 on the tensor cores (the default); mixed with FP64 kernel values and FP32-pair
    sums. Step times at the workload's eps = 6; errors after one revolution (200 steps)
    against the exact solution (the initial field) for several eps: at eps = 6 the
    interpolation matrix is numerically singular (smallest LU pivot ~1e-15) and the FP64
    iteration itself diverges (the oracle's too); eps = 9 is accurate in FP64; eps = 24 is well
    conditioned. A diverged run is reported as null."""
    from paper_1804_01609_gb300 import inputs
    w = inputs.config_global_rotation()
    out = {"eps": w.eps}
    variants = ((rbfsl.FP64, "fp64", None), (rbfsl.MIXED, "mixed", rbfsl.GLOBAL_EVAL_TC),
                (rbfsl.MIXED, "mixed_fp32_pairs", rbfsl.GLOBAL_EVAL_PAIRS))
    for prec, name, ev in variants:
        ctx = global_ctx(rbfsl, w, prec, stream, evaluation=ev)
        t0 = time.perf_counter()
        ctx.step(1)
        torch.cuda.synchronize()
        setup = time.perf_counter() - t0
        ms = timed_steps(ctx, K, 1, stream, flush, torch)
        ctx.close()
        out[name] = {"value": w.N / (float(ms.mean()) / 1e3), "ms_per_step": float(ms.mean()),
                     "setup_and_first_step_s": setup}
    q0 = w.q0()
    acc = []
    for eps in accuracy_eps:
        row = {"eps": eps}
        qs = {}
        for prec, name, ev in variants:
            ctx = global_ctx(rbfsl, w, prec, stream, eps, evaluation=ev)
            ctx.step(w.steps)
            qs[name] = ctx.get_q()
            ctx.close()
            ok = bool(np.isfinite(qs[name]).all())
            row[name + "_l2_vs_exact"] = finite_or_none(rel_l2(qs[name], q0)) if ok else None
        for name in ("mixed", "mixed_fp32_pairs"):
            if row["fp64_l2_vs_exact"] is not None and row[name + "_l2_vs_exact"] is not None:
                row[name + "_over_fp64"] = row[name + "_l2_vs_exact"] / row["fp64_l2_vs_exact"]
                row[name + "_l2_vs_fp64"] = finite_or_none(rel_l2(qs[name], qs["fp64"]))
        acc.append(row)
    out["accuracy_after_200_steps"] = acc
    return out


def bench_global_eval(rbfsl, torch, stream, flush, K=10):
    """The global evaluation alone at the global workload's size (N = Nq = 10,242 departure
    points of one step, 64 tracers, Gaussian eps = 6): tensor cores (split TF32, the mixed
    step's kernel), FP32 CUDA cores and FP64. Algorithmic work 2 N Nq T flop plus N Nq kernel
    values; the split-TF32 product executes four TF32 MMA products per useful one."""
    from paper_1804_01609_gb300 import inputs
    w = inputs.config_global_rotation()
    N, T = w.N, w.T
    x = torch.as_tensor(w.X, device="cuda")
    xi = torch.empty_like(x)
    rbfsl.rbfsl_trace_rk4(x, w.vel_kind, w.vel_params, w.dt, w.dt, rbfsl.FP64, xi, stream=stream)
    with torch.cuda.stream(stream):
        g = torch.Generator(device="cuda").manual_seed(11)
        C = torch.randn((N, T), generator=g, device="cuda", dtype=torch.float64)
        C32 = C.float()
        o_tc = torch.empty((N, T), dtype=torch.float32, device="cuda")
        o32 = torch.empty_like(o_tc)
        o64 = torch.empty((N, T), dtype=torch.float64, device="cuda")
    ws = rbfsl.rbfsl_global_eval_tc(xi, x, rbfsl.GAUSS, w.eps, C, o_tc, stream=stream)
    t_tc = time_op(lambda: rbfsl.rbfsl_global_eval_tc(xi, x, rbfsl.GAUSS, w.eps, C, o_tc, workspace=ws,
                                                      stream=stream), K, stream, flush, torch)
    t32 = time_op(lambda: rbfsl.rbfsl_global_eval(xi, x, rbfsl.GAUSS, w.eps, C32, o32, stream=stream), K,
                  stream, flush, torch)
    t64 = time_op(lambda: rbfsl.rbfsl_global_eval(xi, x, rbfsl.GAUSS, w.eps, C, o64, stream=stream), 3,
                  stream, flush, torch)
    with torch.cuda.stream(stream):
        o_pr = torch.empty((N, T, 2), dtype=torch.float32, device="cuda")
    ws_pr = rbfsl.rbfsl_global_eval_pairs(xi, x, rbfsl.GAUSS, w.eps, C, o_pr, stream=stream)
    t_pr = time_op(lambda: rbfsl.rbfsl_global_eval_pairs(xi, x, rbfsl.GAUSS, w.eps, C, o_pr, workspace=ws_pr,
                                                         stream=stream), K, stream, flush, torch)
    torch.cuda.synchronize()
    scale = float(o64.abs().max())
    flop = 2.0 * N * N * T
    return {"N": N, "Nq": N, "T": T,
            "tensor_cores": {"kernel": "global_eval_tc_kernel (+ tc_prepare, tc_reduce_kernel)",
                             "us": 1e3 * t_tc, "useful_tflops": flop / (t_tc * 1e-3) / 1e12,
                             "tf32_mma_tflops": 4 * flop / (t_tc * 1e-3) / 1e12,
                             "max_err_vs_fp64_rel_to_max": float((o_tc.double() - o64).abs().max()) / scale},
            "fp32_cuda_cores": {"us": 1e3 * t32, "useful_tflops": flop / (t32 * 1e-3) / 1e12,
                                "max_err_vs_fp64_rel_to_max": float((o32.double() - o64).abs().max()) / scale},
            "fp64": {"us": 1e3 * t64, "useful_tflops": flop / (t64 * 1e-3) / 1e12},
            "fp32_pairs": {"kernel": "phi_pairs_kernel + cardinal_apply_pair_kernel (FP64 kernel values, pair sums)",
                           "us": 1e3 * t_pr, "useful_tflops": flop / (t_pr * 1e-3) / 1e12,
                           "max_err_vs_fp64_rel_to_max": float(((o_pr[..., 0].double() + o_pr[..., 1].double())
                                                                - o64).abs().max()) / scale}}


# ----------------------------------------------------------------------------- paper cases
def bench_paper_cases(rbfsl, torch, stream, Ns=(2562, 10242, 40962, 92162)):
    """The paper's test cases (Sec. 4) on Fibonacci nodes in FP64 with Fehlberg's RK5 tracer,
    with the error measures of Sec. 4 against the exact solution (the initial field): solid-body
    rotation of the cosine
    bell (alpha = pi/2, one revolution, dt = pi/10) and the deformational flow of two cosine
    bells and of two Gaussian bells (T = 5, dt = 1/10). Local centre stencils n = 31 and 84
    (ell and the PHS power by the paper's rules) over N, with the order p of err ~ N^(-p/2)
    fitted without the smallest N as in the paper; RBF-PU (~84 nodes per patch, ell = 3, r^7)
    on the rotation; the global IMQ interpolant (eps = 5; the paper does not print its eps) in
    cardinal form on the rotation at N = 10,242, FP64 and mixed. Seconds are wall time of the
    steps (set-up excluded, as the paper's cost comparison)."""
    from paper_1804_01609_gb300 import diagnostics, inputs

    def run(w, method, mode=None, precision=rbfsl.FP64, eps=None, a=2.5):
        ctx = rbfsl.Context(0, stream=stream)
        ctx.set_nodes(w.X)
        ctx.set_velocity(w.vel_kind, w.vel_params)
        ctx.set_precision(precision)
        ctx.set_integrator(rbfsl.RK5)  # the paper's choice for its experiments (Sec. 3.2)
        if method == "global":
            ctx.set_method(rbfsl.GLOBAL)
            ctx.set_kernel(rbfsl.IMQ, eps)
            ctx.set_global_form(rbfsl.GLOBAL_CARDINAL)
        else:
            ctx.set_method(rbfsl.LOCAL if method == "local" else rbfsl.PU, mode or rbfsl.DIRECT)
            ctx.set_stencil_size(w.n)
            ctx.set_sh_degree(w.ell)
            ctx.set_kernel(rbfsl.PHS, w.power)
            if method == "pu":
                ctx.set_pu(inputs.fibonacci_nodes(int(np.ceil(a * w.N / w.n))))
        ctx.set_dt(w.dt)
        ctx.set_tracers(w.q0())
        ctx.step(1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.step(w.steps - 1)
        torch.cuda.synchronize()
        secs = time.perf_counter() - t0
        q = ctx.get_q()[:, 0]
        st = ctx.get_stats()
        ctx.close()
        m = diagnostics.error_measures(q, w.q0()[:, 0])
        m.update({"N": w.N, "steps_s": secs * w.steps / max(w.steps - 1, 1)})
        if method == "pu":
            # departure points in no patch (the patches must cover the sphere, Sec. 2.3):
            # their values are NaN and flagged, so the error measures are then undefined
            m["uncovered_points"] = int(st.uncovered_points)
        return m

    def sweep(mk, method, mode, ns, Nlist):
        res = {}
        for n in ns:
            rows = [run(mk(N, n), method, mode) for N in Nlist]
            res[f"n{n}"] = {"rows": rows,
                            "order_l2": diagnostics.convergence_order(Nlist[1:], [r["l2"] for r in rows[1:]]),
                            "order_linf": diagnostics.convergence_order(Nlist[1:], [r["linf"] for r in rows[1:]])}
        return res

    out = {"node_sets": "Fibonacci + 1e-3 rad jitter", "precision": "fp64", "tracer": "rk5"}
    sbr = lambda N, n: inputs.config_sbr(N, n=n)
    out["sbr_cosine_bell"] = {"local_center": sweep(sbr, "local", rbfsl.CENTER, (31, 84), Ns)}
    pu = lambda N, n: inputs.config_sbr(N, method="pu", n=n, ell=3, power=7)
    out["sbr_cosine_bell"]["pu"] = sweep(pu, "pu", None, (84,), Ns[1:])
    wg = inputs.config_sbr(10242, method="global")
    out["sbr_cosine_bell"]["global_imq_eps5_cardinal"] = {
        "fp64": run(wg, "global", eps=5.0), "mixed": run(wg, "global", precision=rbfsl.MIXED, eps=5.0)}
    for ic in ("cosine", "gaussian"):
        mk = lambda N, n, ic=ic: inputs.config_nl(N, ic=ic, n=n)
        out[f"nl_{ic}_bells"] = {"local_center": sweep(mk, "local", rbfsl.CENTER, (31, 84), Ns)}

    # error measures against the stencil / patch size n at N = 40,962 (the paper's dissipation
    # and dispersion plots), local centre stencils and RBF-PU (overlap a = 2.5)
    nsw = {}
    for case, mk in (("sbr_cosine_bell", lambda n, meth: inputs.config_sbr(
                          40962, method=meth, n=n, **({"ell": 3, "power": 7} if meth == "pu" and n >= 49 else {}))),
                     ("nl_cosine_bells", lambda n, meth: inputs.config_nl(40962, ic="cosine", method=meth, n=n))):
        nsw[case] = {meth: [dict(run(mk(n, meth), meth, rbfsl.CENTER if meth == "local" else None), n=n)
                            for n in (17, 31, 49, 84)] for meth in ("local", "pu")}
    out["n_sweep_N40962"] = nsw

    # RBF-PU against the nodes per patch n and the overlap a (Eqs. rad_patches, num_patches:
    # R = 2 sqrt(n / N) fixed by n, M = ceil(a N / n) patches): error and step time, rotation
    # of the cosine bell at N = 40,962
    ovl = []
    for n in (31, 49, 84):
        for a in (1.5, 2.5, 3.5, 5.0):
            w = inputs.config_sbr(40962, method="pu", n=n, **({"ell": 3, "power": 7} if n >= 49 else {}))
            ovl.append(dict(run(w, "pu", a=a), n=n, a=a, patches=int(np.ceil(a * w.N / n))))
    out["pu_n_a_sweep_N40962"] = ovl

    # ten revolutions of the cosine bell with dt = pi/20 (the paper's mass-conservation run):
    # mass error and l2 error after each revolution, N = 40,962, n = 49
    def revolutions(method):
        w = inputs.config_sbr(40962, method=method, n=49, steps=40, revolutions=10)
        ctx = rbfsl.Context(0, stream=stream)
        ctx.set_nodes(w.X)
        ctx.set_velocity(w.vel_kind, w.vel_params)
        ctx.set_integrator(rbfsl.RK5)
        ctx.set_method(rbfsl.LOCAL if method == "local" else rbfsl.PU,
                       rbfsl.CENTER if method == "local" else rbfsl.DIRECT)
        ctx.set_stencil_size(w.n)
        ctx.set_sh_degree(w.ell)
        ctx.set_kernel(rbfsl.PHS, w.power)
        if method == "pu":
            ctx.set_pu(inputs.fibonacci_nodes(int(np.ceil(2.5 * w.N / w.n))))
        ctx.set_dt(w.dt)
        ctx.set_tracers(w.q0())
        q0 = w.q0()[:, 0]
        rows = []
        for rev in range(1, 11):
            ctx.step(40)
            m = diagnostics.error_measures(ctx.get_q()[:, 0], q0)
            rows.append({"revolution": rev, "l2": m["l2"], "mass": m["mass"]})
        ctx.close()
        return {"rows": rows, "l2_growth_10_over_1": rows[-1]["l2"] / rows[0]["l2"]}
    out["sbr_ten_revolutions_N40962_n49"] = {"local": revolutions("local"), "pu": revolutions("pu")}
    return out


# ----------------------------------------------------------------------------- batched
def bench_batched(rbfsl, torch, stream, steps=10, seq_steps=3, P=64, Ns=(2562, 10242, 40962, 163842),
                  precisions=("mixed", "fp64")):
    """P independent local problems (N from Ns, (n, ell) from {(31,2), (55,3), (84,4)} with
    r^(2 ell + 1), 1-16 tracers, own rotation or deformation), direct stencils, one persistent
    fused kernel per step under a CUDA graph, in the given precisions; against the same problems
    stepped one after another through single-problem contexts (mixed); per-problem relative l2
    of the mixed result against the FP64 one."""
    from paper_1804_01609_gb300 import inputs
    specs = inputs.batched_problems(P, Ns=Ns)
    probs = []
    for sp in specs:
        X = inputs.nodes(sp["N"], sp["seed"])
        rng = np.random.default_rng(sp["seed"])
        fns = [inputs.plane_wave_field(rng, 8.0) for _ in range(sp["T"])]
        probs.append((sp, X, np.stack([f(X) for f in fns], axis=1)))
    nodes = sum(sp["N"] for sp, _, _ in probs)
    out = {"problems": len(probs), "nodes": nodes, "steps": steps}
    finals = {}
    for prec, name in ((rbfsl.MIXED, "mixed"), (rbfsl.FP64, "fp64")):
        if name not in precisions:
            continue
        b = rbfsl.Batch(0, stream=stream)
        ids = [b.add(X, q0, sp["n"], sp["ell"], sp["power"], sp["vel_kind"], sp["vel_params"], 1.0 / 100,
                     mode=rbfsl.DIRECT, precision=prec) for sp, X, q0 in probs]
        choices = b.autotune()
        b.step(1)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        finals[name] = [b.get_q(i) for i in ids]
        b.close()
        out[name] = {"value": nodes / (ms / 1e3), "ms_per_step": ms, "tile_shapes": [list(c) for c in choices]}
    # the same problems one after another through contexts (mixed), seq_steps steps each
    seq_ms = 0.0
    for sp, X, q0 in probs:
        ctx = rbfsl.Context(0, stream=stream)
        ctx.set_nodes(X)
        ctx.set_velocity(sp["vel_kind"], sp["vel_params"])
        ctx.set_method(rbfsl.LOCAL, rbfsl.DIRECT)
        ctx.set_stencil_size(sp["n"])
        ctx.set_sh_degree(sp["ell"])
        ctx.set_kernel(rbfsl.PHS, sp["power"])
        ctx.set_precision(rbfsl.MIXED)
        ctx.set_dt(1.0 / 100)
        ctx.set_tracers(q0)
        ctx.step(1)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.step(seq_steps)
        e1.record(stream)
        torch.cuda.synchronize()
        seq_ms += e0.elapsed_time(e1) / seq_steps
        ctx.close()
    out["sequential_contexts_mixed"] = {"ms_per_step": seq_ms, "value": nodes / (seq_ms / 1e3),
                                        "steps_timed_per_problem": seq_steps}
    out["batched_over_sequential"] = seq_ms / out["mixed"]["ms_per_step"]
    if "fp64" in finals:
        d = [rel_l2(a, b) for a, b in zip(finals["mixed"], finals["fp64"])]
        out["accuracy_mixed_vs_fp64"] = {"steps": steps + 1, "rel_l2_max": float(max(d)),
                                         "rel_l2_median": float(np.median(d))}
    return out


# ----------------------------------------------------------------------------- served
def served_requests(R, rate, Ns, steps, seed, rbfsl):
    """R transport solves with Poisson arrival times (mean `rate`/s): half local (centre
    stencils, (n, ell) from {(31,2),(55,3),(84,4)}, r^(2 ell + 1)) and half RBF-PU (~100 nodes per
    patch, ell = 3, r^7, Wendland weights, a = 2.5), N drawn from Ns, 1-16 smooth tracers, steps
    drawn from [steps[0], steps[1]], each its own tilted rotation over one period. Returns
    (arrival time, request, exact-solution function)."""
    from paper_1804_01609_gb300 import inputs
    rng = np.random.default_rng(seed)
    reqs = []
    t = 0.0
    for k in range(R):
        t += rng.exponential(1.0 / rate)
        N = int(rng.choice(Ns))
        T = int(rng.integers(1, 17))
        S = int(rng.integers(steps[0], steps[1] + 1))
        X = inputs.nodes(N, seed * 100 + k)
        fns = [inputs.plane_wave_field(rng, 8.0) for _ in range(T)]
        q0 = np.stack([f(X) for f in fns], axis=1)
        vp = inputs.rigid_rotation_params(inputs.random_unit_vectors(1, rng)[0], 1.0)
        if k % 2 == 0:
            n, ell = [(31, 2), (55, 3), (84, 4)][int(rng.integers(0, 3))]
            r = dict(X=X, q0=q0, n=n, ell=ell, power=2 * ell + 1, vel_kind=0, vel_params=vp, dt=1.0 / S,
                     steps=S, method=rbfsl.LOCAL, mode=rbfsl.CENTER, centers=None)
        else:
            n = 100
            r = dict(X=X, q0=q0, n=n, ell=3, power=7, vel_kind=0, vel_params=vp, dt=1.0 / S, steps=S,
                     method=rbfsl.PU, mode=rbfsl.DIRECT, centers=inputs.fibonacci_nodes(int(np.ceil(2.5 * N / n))))
        reqs.append((t, r, fns))
    return reqs


def serve_once(rbfsl, reqs, precision, budget=150 * 10 ** 9, slots=64):
    import threading
    srv = rbfsl.Server(0, budget_bytes=budget, max_slots=slots)
    tickets = []

    def submitter():
        t0 = time.perf_counter()
        for ta, r, _ in reqs:
            d = ta - (time.perf_counter() - t0)
            if d > 0:
                time.sleep(d)
            tickets.append(srv.submit(r["X"], r["q0"], r["n"], r["ell"], r["power"], r["vel_kind"],
                                      r["vel_params"], r["dt"], r["steps"], method=r["method"],
                                      mode=r["mode"], precision=precision, centers=r["centers"]))

    th = threading.Thread(target=submitter)
    th.start()
    th.join()
    srv.wait_idle(3600)
    res = [srv.result(tk, raise_on_failure=False) for tk in tickets]
    info = srv.info()
    srv.close()
    return res, info


def bench_served(rbfsl, R=128, rate=200.0, Ns=(642, 2562, 10242, 40962, 163842, 655362), steps=(50, 120),
                 seed=1804 * 100 + 5):
    """The served workload (requests as in served_requests, device-memory budget 150 GB, 64
    slots), once in mixed precision and once in FP64 on the same requests. Reports per precision
    the achieved node-updates/s, p50/p99 latency (submission to result), the offered load (node
    updates of all requests over their arrival span) and the admission peak; per request the
    relative l2 of the mixed result against the FP64 one and both errors against the exact
    solution (one full rotation: the initial field); the FP64 results of the smallest requests
    against the oracle's run of the same solve."""
    reqs = served_requests(R, rate, Ns, steps, seed, rbfsl)
    arrivals = [t for t, _, _ in reqs]
    work = sum(r["X"].shape[0] * r["steps"] for _, r, _ in reqs)
    offered = work / max(arrivals[-1] - arrivals[0], 1e-9)
    out = {"requests": R, "arrival_rate_per_s": rate, "N": list(Ns), "steps": list(steps),
           "node_updates": int(work), "offered_node_updates_per_s": offered}
    results, stats_of = {}, {}
    for prec, name in ((rbfsl.MIXED, "mixed"), (rbfsl.FP64, "fp64")):
        res, info = serve_once(rbfsl, reqs, prec)
        stats = [st for _, st in res]
        results[name] = [q for q, _ in res]
        stats_of[name] = stats
        lat = np.array([st.finish_s - st.submit_s for st in stats])
        span = max(st.finish_s for st in stats) - min(st.submit_s for st in stats)
        nu = sum(st.node_updates for st in stats)
        out[name] = {"value": nu / span, "wall_s": span, "latency_p50_s": float(np.percentile(lat, 50)),
                     "latency_p99_s": float(np.percentile(lat, 99)),
                     "failed": int(sum(st.status != 0 for st in stats)),
                     "requests_with_failed_points": int(sum(st.failed_points > 0 for st in stats)),
                     "errors": sorted({st.message.decode() for st in stats if st.status != 0})[:3],
                     "peak_bytes": int(info.peak_bytes), "budget_bytes": int(info.budget_bytes),
                     "ticks": int(info.ticks)}
    ratios, d, bad = [], [], []
    for k, ((_, r, fns), qm, q64) in enumerate(zip(reqs, results["mixed"], results["fp64"])):
        desc = {"request": k, "method": "local" if r["method"] == rbfsl.LOCAL else "pu", "N": r["X"].shape[0],
                "n": r["n"], "ell": r["ell"], "steps": r["steps"], "T": r["q0"].shape[1],
                "failed_points": {nm: int(stats_of[nm][k].failed_points) for nm in ("mixed", "fp64")}}
        fin = {nm: q is not None and bool(np.isfinite(q).all()) for nm, q in (("mixed", qm), ("fp64", q64))}
        if not (fin["mixed"] and fin["fp64"]):
            bad.append(dict(desc, finite=fin, max_abs={nm: (float(np.nanmax(np.abs(q))) if q is not None else None)
                                                       for nm, q in (("mixed", qm), ("fp64", q64))}))
            continue
        e64 = rel_l2(q64, r["q0"])
        if not e64 < 0.5:  # the FP64 run itself diverged (stencil systems beyond FP64, see DESIGN)
            bad.append(dict(desc, fp64_l2_vs_exact=e64, mixed_l2_vs_exact=rel_l2(qm, r["q0"])))
            continue
        d.append(rel_l2(qm, q64))
        ratios.append(abs(rel_l2(qm, r["q0"]) - e64) / e64)
    out["accuracy"] = {"compared": len(d), "mixed_vs_fp64_rel_l2_max": float(max(d)) if d else None,
                       "mixed_vs_fp64_rel_l2_median": float(np.median(d)) if d else None,
                       "mixed_error_excess_over_fp64_max": float(max(ratios)) if ratios else None,
                       "all_within_1pct_of_fp64_error": bool(ratios and max(ratios) <= 0.01),
                       "diverged_or_nonfinite": bad[:12], "diverged_or_nonfinite_count": len(bad)}
    import oracle
    oracle.build()
    small = [(r, q64) for (_, r, _), q64 in zip(reqs, results["fp64"]) if r["X"].shape[0] == min(Ns)][:4]
    checks = []
    for r, q64 in small:
        if r["method"] == rbfsl.LOCAL:
            ref = oracle.local_run(r["X"], r["q0"], r["n"], r["ell"], r["power"], r["vel_kind"], r["vel_params"],
                                   r["dt"], r["steps"], mode=oracle.CENTER)
        else:
            pu = oracle.PUInterpolator(r["X"], r["centers"], r["n"], r["ell"], r["power"])
            ref = r["q0"]
            for m in range(r["steps"]):
                ref = pu.apply(oracle.trace_rk4(r["X"], r["vel_kind"], r["vel_params"], (m + 1) * r["dt"], r["dt"]), ref)
        checks.append({"method": "local" if r["method"] == rbfsl.LOCAL else "pu", "N": r["X"].shape[0],
                       "steps": r["steps"], "fp64_vs_oracle_rel_l2": rel_l2(q64, ref)})
    out["oracle_check_smallest"] = checks
    return out


# ----------------------------------------------------------------------------- reference arm
def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    w = workload()
    import oracle
    oracle.build()
    X, q = w.X, w.q0()
    Xi = oracle.trace_rk4(X, w.vel_kind, w.vel_params, w.dt, w.dt)
    S = 512  # node-updates per reference step: a bounded sample of the workload's step
    for _ in range(args.warmup):
        oracle.local_apply(X, Xi[:64], q, w.n, w.ell, oracle.PHS, float(w.power))
    times = []
    for k in range(args.steps):
        rows = np.arange(k * S, (k + 1) * S) % w.N
        t0 = time.perf_counter()
        oracle.trace_rk4(X[rows], w.vel_kind, w.vel_params, w.dt, w.dt)
        oracle.local_apply(X, Xi[rows], q, w.n, w.ell, oracle.PHS, float(w.power))
        times.append(time.perf_counter() - t0)
    el = float(np.sum(times))
    v = S * args.steps / el
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "local-deformation N=40962 n=84 ell=4 r^9 T=32 (sampled)",
                   "sample_nodes_per_step": S},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": f"{S} node-updates per step of the workload, FP64 oracle"},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


# ----------------------------------------------------------------------------- our arm
def run_case(args):
    """One kernel of the workload, on the first --nq departure points, --repeat times."""
    import torch
    from paper_1804_01609_gb300 import rbfsl
    if args.case == "wq":
        stream = torch.cuda.current_stream()
        flush = torch.empty(64 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
        r = bench_wq_hbm(rbfsl, torch, stream, flush, K=args.repeat)
        print(f"case wq: {json.dumps(r)}", flush=True)
        return
    if args.case == "batched":  # the batched leg alone
        st = torch.cuda.Stream()
        r = bench_batched(rbfsl, torch, st)
        r["small_problems_256"] = bench_batched(rbfsl, torch, st, steps=20, seq_steps=5, P=256, Ns=(642, 2562),
                                                precisions=("mixed",))
        print(f"case batched: {json.dumps(json_safe(r))}", flush=True)
        return
    if args.case == "served":  # the served leg alone (--served-requests, --served-steps)
        r = bench_served(rbfsl, R=args.served_requests, steps=tuple(args.served_steps))
        print(f"case served: {json.dumps(json_safe(r))}", flush=True)
        return
    if args.case == "tceval":  # the tensor-core global evaluation at the global workload's size
        from paper_1804_01609_gb300 import inputs
        wg = inputs.config_global_rotation()
        xg = torch.as_tensor(wg.X, device="cuda")
        pg = torch.empty_like(xg)
        rbfsl.rbfsl_trace_rk4(xg, wg.vel_kind, wg.vel_params, wg.dt, wg.dt, rbfsl.FP64, pg)
        g = torch.Generator(device="cuda").manual_seed(11)
        C = torch.randn((wg.N, wg.T), generator=g, device="cuda", dtype=torch.float64)
        o = torch.empty((wg.N, wg.T), dtype=torch.float32, device="cuda")
        ws = rbfsl.rbfsl_global_eval_tc(pg, xg, rbfsl.GAUSS, wg.eps, C, o)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.repeat):
            rbfsl.rbfsl_global_eval_tc(pg, xg, rbfsl.GAUSS, wg.eps, C, o, workspace=ws)
        e1.record()
        torch.cuda.synchronize()
        print(f"case tceval: {e0.elapsed_time(e1) / args.repeat:.3f} ms per call (N = Nq = {wg.N}, T = {wg.T})",
              flush=True)
        return
    if args.case == "cardinal":  # q <- E q at the global workload's size, FP64 and FP32 pairs
        Ng, Tg = 10242, 64
        g = torch.Generator(device="cuda").manual_seed(12)
        for name, shape, dt in (("fp64", (Ng, Ng), torch.float64), ("pairs", (Ng, Ng, 2), torch.float32)):
            E = torch.randn(shape, generator=g, device="cuda", dtype=dt) / Ng ** 0.5
            q = torch.randn((Ng, Tg) + shape[2:], generator=g, device="cuda", dtype=dt)
            o = torch.empty_like(q)
            ws = rbfsl.rbfsl_cardinal_apply(E, q, o)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(args.repeat):
                rbfsl.rbfsl_cardinal_apply(E, q, o, workspace=ws)
            e1.record()
            torch.cuda.synchronize()
            print(f"case cardinal {name}: {e0.elapsed_time(e1) / args.repeat:.3f} ms per call "
                  f"(Nq = N = {Ng}, T = {Tg}, workspace {ws.numel()} B)", flush=True)
            del E, q, o, ws
        return
    w = workload()
    N, n = w.N, w.n
    nq = min(args.nq, N)
    x = torch.as_tensor(w.X, device="cuda")
    xi = torch.empty_like(x)
    rbfsl.rbfsl_trace_rk4(x, w.vel_kind, w.vel_params, 0.3, w.dt, rbfsl.FP64, xi)
    ix = rbfsl.rbfsl_knn_index_create(x, n)
    I = torch.empty((N, n), dtype=torch.int32, device="cuda")
    rbfsl.rbfsl_knn_query(ix, xi, n, I)
    W = torch.empty((N, n, 2), dtype=torch.float32, device="cuda")  # FP32 pairs, as the mixed step
    rbfsl.rbfsl_stencil_weights(x, I, n, w.ell, rbfsl.PHS, w.power, xi, W)
    q = torch.as_tensor(pairs_of(w.q0()), device="cuda")
    qo = torch.empty_like(q)
    ctx = None
    if args.case == "center":  # whole centre-stencil steps through the context
        ctx = make_ctx(w, rbfsl.MIXED, torch.cuda.current_stream(), rbfsl, mode=rbfsl.CENTER)
        ctx.step(1)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.repeat):
        if args.case == "weights":
            rbfsl.rbfsl_stencil_weights(x, I[:nq], n, w.ell, rbfsl.PHS, w.power, xi[:nq], W[:nq])
        elif args.case == "gather":
            rbfsl.rbfsl_gather_dot(I, W, q, qo, pairs=True)
        elif args.case == "knn":
            rbfsl.rbfsl_knn_query(ix, xi[:nq], n, I[:nq])
        elif args.case == "center":
            ctx.step(1)
        else:
            rbfsl.rbfsl_trace_rk4(x, w.vel_kind, w.vel_params, 0.3, w.dt, rbfsl.MIXED, xi)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.repeat
    extra = ""
    if args.case == "weights":
        m = n + (w.ell + 1) ** 2
        extra = f" {nq * weights_flops(m) / ms / 1e9:.3f} TFLOP/s ({nq} points, m={m})"
    print(f"case {args.case}: {ms:.3f} ms per launch{extra}", flush=True)
    if ctx is not None:
        ctx.close()
    ix.close()


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.case:
        return run_case(args)
    rank, world, local = dist_env()
    import torch
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_1804_01609_gb300 import rbfsl
    rbfsl.load()
    w = workload()
    N, n, T = w.N, w.n, w.T
    m = n + (w.ell + 1) ** 2
    stream = torch.cuda.Stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    # ---- timed region: mixed precision (headline), then FP64
    ctx = make_ctx(w, rbfsl.MIXED, stream, rbfsl)
    barrier()
    with ClockSampler(local) as clk:
        step_ms = timed_steps(ctx, args.steps, args.warmup, stream, flush, torch)
    barrier()
    total_s = job_seconds(float(step_ms.sum()) / 1e3, world)
    value = job_throughput(N * args.steps, world, total_s)

    # dominant kernel (FP64 stencil solve) and the gather-dot, timed alone on the same stream
    xi_t, I_t, _ = ctx.last_step_tensors(n, torch.float32)
    x_t = torch.as_tensor(w.X, device="cuda")
    wp = torch.empty((N, n, 2), dtype=torch.float32, device="cuda")  # FP32 pairs, as the step stores them
    rbfsl.rbfsl_stencil_weights(x_t, I_t, n, w.ell, rbfsl.PHS, w.power, xi_t, wp, stream=stream)
    w_ms = time_op(lambda: rbfsl.rbfsl_stencil_weights(x_t, I_t, n, w.ell, rbfsl.PHS, w.power,
                                                       xi_t, wp, stream=stream),
                   max(3, min(args.steps, 10)), stream, flush, torch)
    qp = torch.as_tensor(pairs_of(w.q0()), device="cuda")
    qo = torch.empty_like(qp)
    g_ms = time_op(lambda: rbfsl.rbfsl_gather_dot(I_t, wp, qp, qo, stream=stream, pairs=True), 10, stream,
                   flush, torch)
    ctx.close()

    ctx64 = make_ctx(w, rbfsl.FP64, stream, rbfsl)
    step64_ms = timed_steps(ctx64, max(3, min(args.steps, 10)), 1, stream, flush, torch)
    ctx64.close()
    value64 = N / (float(step64_ms.mean()) / 1e3)

    # the paper's centre stencils: each node's saddle-point matrix factorised once (set-up),
    # per step one nearest-node search and two triangular solves per point
    center = {}
    for prec, name in ((rbfsl.MIXED, "mixed"), (rbfsl.FP64, "fp64")):
        t0 = time.perf_counter()
        ctxc = make_ctx(w, prec, stream, rbfsl, mode=rbfsl.CENTER)
        ctxc.step(1)
        torch.cuda.synchronize()
        setup_s = time.perf_counter() - t0
        cms = timed_steps(ctxc, max(args.steps, 10), 2, stream, flush, torch)
        ctxc.close()
        center[name] = {"value": N / (float(cms.mean()) / 1e3), "ms_per_step": float(cms.mean()),
                        "p50_ms": float(np.percentile(cms, 50)), "p99_ms": float(np.percentile(cms, 99)),
                        "setup_s": setup_s}

    # the paper's final integrator (Fehlberg, fifth order) against RK4 at four times the step:
    # centre stencils, mixed precision, the deformation run in 150 steps; error vs exact
    integ = {}
    if args.accuracy_steps > 0:
        from paper_1804_01609_gb300 import inputs as _inp
        w4 = _inp.config_local_deformation(steps=150)
        for order in (rbfsl.RK4, rbfsl.RK5):
            c4 = make_ctx(w4, rbfsl.MIXED, stream, rbfsl, mode=rbfsl.CENTER)
            c4.set_integrator(order)
            c4.step(w4.steps)
            integ[f"rk{order}_l2_vs_exact"] = rel_l2(c4.get_q(), w4.q0())
            c4.close()
        integ["steps"] = 150

    # ---- end to end through the public API with host buffers (pinned), per step:
    # H2D of the field, one SL step, D2H of the new field
    ctx = make_ctx(w, rbfsl.MIXED, stream, rbfsl)
    hq = torch.from_numpy(w.q0().astype(np.float32)).pin_memory()
    ctx.step(1)
    torch.cuda.synchronize()
    K2 = args.steps
    t0 = time.perf_counter()
    for _ in range(K2):
        ctx.set_tracers(hq)
        ctx.step(1)
        ctx.get_q(out=hq)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    ctx.close()
    e2e = {"value": world * N * K2 / e2e_s if world == 1 else N * K2 / e2e_s * world,
           "unit": UNIT, "h2d_bytes_per_step": N * T * 4, "d2h_bytes_per_step": N * T * 4}

    # ---- accuracy of full trajectories (outside the timed region)
    acc = {}
    if args.accuracy_steps > 0:
        S = min(args.accuracy_steps, w.steps)
        q0 = w.q0()
        q64, st64 = accuracy_run(w, rbfsl.FP64, S, stream, rbfsl)
        qmx, stmx = accuracy_run(w, rbfsl.MIXED, S, stream, rbfsl)
        acc = {"steps": S, "t_final": S * w.dt}
        if S == w.steps:  # the flow reverses: exact solution at T_f is the initial field
            acc.update({"fp64_l2_vs_exact": rel_l2(q64, q0), "fp64_linf_vs_exact": rel_linf(q64, q0),
                        "mixed_l2_vs_exact": rel_l2(qmx, q0), "mixed_linf_vs_exact": rel_linf(qmx, q0)})
            acc["mixed_within_1pct_of_fp64"] = bool(
                abs(acc["mixed_l2_vs_exact"] - acc["fp64_l2_vs_exact"]) <= 0.01 * acc["fp64_l2_vs_exact"])
        acc["mixed_l2_vs_fp64"] = rel_l2(qmx, q64)
        acc["singular_points"] = int(st64.singular_points + stmx.singular_points)
        acc["knn_failures"] = int(st64.knn_failures + stmx.knn_failures)
        qc64, _ = accuracy_run(w, rbfsl.FP64, S, stream, rbfsl, mode=rbfsl.CENTER)
        qcmx, _ = accuracy_run(w, rbfsl.MIXED, S, stream, rbfsl, mode=rbfsl.CENTER)
        if S == w.steps:
            center["fp64"]["l2_vs_exact"] = rel_l2(qc64, q0)
            center["mixed"]["l2_vs_exact"] = rel_l2(qcmx, q0)

    # the metric's comparison: mixed against FP64 at equal l2 error (the 600-step reversal
    # returns the field, so the error is against the initial field), for the graded direct
    # stencils and for the paper's centre stencils
    equal_acc = {"direct": {"mixed_value": value, "fp64_value": value64,
                            "mixed_l2_vs_exact": acc.get("mixed_l2_vs_exact"),
                            "fp64_l2_vs_exact": acc.get("fp64_l2_vs_exact")},
                 "center": {"mixed_value": center["mixed"]["value"], "fp64_value": center["fp64"]["value"],
                            "mixed_l2_vs_exact": center["mixed"].get("l2_vs_exact"),
                            "fp64_l2_vs_exact": center["fp64"].get("l2_vs_exact")}}
    for v in equal_acc.values():
        v["mixed_over_fp64_speed"] = v["mixed_value"] / v["fp64_value"]
        if v["mixed_l2_vs_exact"] is not None:
            v["mixed_within_1pct_of_fp64_error"] = bool(
                abs(v["mixed_l2_vs_exact"] - v["fp64_l2_vs_exact"]) <= 0.01 * v["fp64_l2_vs_exact"])
    equal_acc["center_over_direct_mixed_speed"] = center["mixed"]["value"] / value

    wq = bench_wq_hbm(rbfsl, torch, stream, flush)
    glob = bench_global(rbfsl, torch, stream, flush,
                        accuracy_eps=(6.0, 9.0, 24.0) if args.accuracy_steps > 0 else ())
    glob["evaluation_alone"] = bench_global_eval(rbfsl, torch, stream, flush)
    glob["cardinal_form"] = bench_global_cardinal(rbfsl, torch, stream, flush,
                                                  accuracy_eps=(6.0, 9.0, 24.0) if args.accuracy_steps > 0 else ())
    paper_cases = bench_paper_cases(rbfsl, torch, stream) if args.accuracy_steps > 0 else {}
    batched = {}
    if not args.no_batched:
        batched = bench_batched(rbfsl, torch, stream)
        # many small problems (N = 642 or 2,562), where single-problem steps are launch-bound
        batched["small_problems_256"] = bench_batched(rbfsl, torch, stream, steps=20, seq_steps=5, P=256,
                                                      Ns=(642, 2562), precisions=("mixed",))
    served = {}
    if not args.no_served:
        served = bench_served(rbfsl, R=args.served_requests, steps=tuple(args.served_steps))

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w)

    pk = peaks()
    # FP64 FMA throughput measured in this run (the weights kernel is timed alone: a burst rate)
    with ClockSampler(local) as clk_peak:
        fp64_peak = rbfsl.rbfsl_fp64_fma_rate(1 << 15, stream=stream)
    w_flops = N * weights_flops(m)
    w_tflops = w_flops / (w_ms * 1e-3) / 1e12
    wk_tflops = N * weights_kernel_flops(m) / (w_ms * 1e-3) / 1e12
    g_bytes = N * n * (8 + 4) + N * T * 8 * 2  # FP32-pair weights and field
    g_gbs = g_bytes / (g_ms * 1e-3) / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": float(step_ms.mean()), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64 solves; f32 trace increments and f32-pair gather",
        "data": "synthetic",
        "config": {"workload": "local-deformation N=40962 n=84 ell=4 r^9 T=32 (direct stencils)",
                   "N": N, "n": n, "ell": w.ell, "phs_power": w.power, "tracers": T,
                   "precision": "mixed", "l2": "flushed between timed steps (256 MB write)"},
        "step_latency_ms": {"p50": float(np.percentile(step_ms, 50)),
                            "p99": float(np.percentile(step_ms, 99))},
        "fp64": {"value": value64, "ms_per_step": float(step64_ms.mean())},
        "mixed_vs_fp64_at_equal_l2": equal_acc,
        "center_stencils": center,
        "integrator_at_dt_1_150": integ,
        "global_N10242_T64": glob,
        "paper_test_cases": paper_cases,
        "batched_64_problems": batched,
        "served": served,
        "accuracy": acc,
        "clocks": clk.summary(),
        "e2e": e2e,
        "gpu_launches": 5 * args.steps,
        "roofline": {"bound": "alu", "kernel": "weights_kernel<4, float2> (FP64 blocked Bunch-Kaufman LDL^T, m = 109)",
                     "achieved": w_tflops, "peak": fp64_peak, "unit": "TFLOP/s",
                     "frac": w_tflops / fp64_peak, "traffic": WEIGHTS_DRAM_BYTES,
                     "traffic_unit": "bytes per launch (ncu dram__bytes_read + _write of this kernel version, "
                                     "full launch; null: not captured for this version)",
                     "peak_source": "measured in this run: rbfsl_fp64_fma_rate (dependent FMA chains, all SMs)",
                     "peak_clocks": clk_peak.summary(),
                     "peak_derived": FP64_PEAK_TFLOPS,
                     "frac_of_derived": w_tflops / FP64_PEAK_TFLOPS,
                     "flops_per_unit": "(2/3) m^3 + 2 m^2 per point (one saddle-point solve, elimination's count)",
                     "kernel_flops_per_unit": "(1/3) m^3 + 2 m^2 (the L D L^T the kernel performs)",
                     "kernel_achieved": wk_tflops, "kernel_frac": wk_tflops / fp64_peak,
                     "ms_per_launch": w_ms},
        "roofline_gather": {"bound": "hbm", "kernel": "gather_dot_vec_kernel<float, float4>",
                            "workload": "N=655362 Morton-ordered nodes, n=84, T=16, FP32 difference form",
                            "achieved": wq["f32"]["achieved_gbs"], "peak": pk.get("hbm_gbs"), "unit": "GB/s",
                            "frac": wq["f32"]["achieved_gbs"] / pk["hbm_gbs"] if pk.get("hbm_gbs") else None,
                            "traffic": None, "ms_per_launch": wq["f32"]["ms_per_launch"],
                            "fp64": wq["f64"],
                            "f32x2": wq["f32x2"],
                            "in_step_N40962_T32": {"kernel": "gather_dot_pair_kernel<2> (FP32 pairs)",
                                                   "achieved_gbs": g_gbs, "ms_per_launch": g_ms,
                                                   "note": "W and q fit in L2 at this N"}},
        "cpu_baseline": cpu,
    }
    if rank == 0:
        print(json.dumps(json_safe(line), allow_nan=False), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
