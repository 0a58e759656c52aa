#!/usr/bin/env python
"""Benchmark of the GB300 randomized SVD (Algorithm 4 of the thesis, Section 3.3).

One step = one full rank-k randomized SVD (all steps of the hot path: Omega,
the 2q+2 passes over A, every CholeskyQR2, the Jacobi SVD of the l x l
factor, the lift and the output layout) on a seeded synthetic matrix that is
already resident in HBM.

Default workload (one GPU): A 16384 x 8192 FP64 = U diag(sigma) V^T with Haar
factors and sigma_i = i^-1.5, k = 64, p = 16, q = 2, Omega 8192 x 80.  A is
1.07 GB, larger than the 129 MB L2, so no flush is needed between steps.

Printed: one JSON line (rank 0) with solves/s, the A-pass bandwidth, the
roofline of the dominant kernel, the end-to-end rate through the C ABI with
host buffers, the CPU oracle's rate on this host, clocks sampled during the
timed region and the number of this library's kernel launches per step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank solves its own replica of the workload
(the path has no data exchange between problems); the job rate is the sum
of the ranks' solves over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "RSVD A-pass HBM TB/s & solves/s, mixed vs FP64 plain @σ err≤1e-3; p99 ms"

WORKLOADS = {
    "plain-fp64": dict(
        desc="plain RSVD FP64 on GPU: A 16384x8192 FP64, Haar factors, sigma_i=i^-1.5; "
             "k=64, p=16, q=2; Gaussian Omega 8192x80",
        m=16384, n=8192, k=64, p=16, q=2, spectrum=("poly", 1.5), seed_a=0, seed=2,
        dtype="f64"),
    "mixed-bf16": dict(
        desc="mixed precision: A 65536x16384 stored BF16, Haar factors, sigma_i=exp(-i/40) "
             "plus 1e-4 Gaussian noise floor; k=128, p=32, q=3 (+1 bf16x2 refinement step, "
             "bf16x3 final B); FP32 accumulate",
        m=65536, n=16384, k=128, p=32, q=3, spectrum=("exp", 40.0), terms=640, noise=1e-4,
        seed_a=0, seed=2, dtype="bf16"),
    "mixed-fp8": dict(
        desc="mixed precision, FP8 storage: the same A 65536x16384 stored as FP8 E4M3 with one "
             "power-of-two FP32 scale per 128x128 tile; k=128, p=32, q=3 (+1 refinement step); "
             "block-scaled E4M3 MMAs, operand in 2/4/6 E4M3 slices (power steps / refinement / "
             "final B); FP32 accumulate",
        m=65536, n=16384, k=128, p=32, q=3, spectrum=("exp", 40.0), terms=640, noise=1e-4,
        seed_a=0, seed=2, dtype="fp8"),
}


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ["clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.active",
              "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
              "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]

    def __init__(self, device_uuid: str | None):
        self.uuid = device_uuid
        self.proc = None
        self.out = os.path.join("/tmp", f"rsvd_clocks_{os.getpid()}.csv")

    def start(self):
        cmd = ["nvidia-smi", f"--query-gpu={','.join(self.FIELDS)}",
               "--format=csv,noheader,nounits", "-lms", "100"]
        if self.uuid:
            cmd += ["-i", self.uuid]
        try:
            self.fh = open(self.out, "w")
            self.proc = subprocess.Popen(cmd, stdout=self.fh, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        rows = []
        with open(self.out) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) == len(self.FIELDS):
                    rows.append(parts)
        os.unlink(self.out)
        if not rows and self.uuid:
            return None
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[4 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def _barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def _max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(local_units: float, local_ms: float, world: int):
    """Whole-job rate of replicas: units summed over ranks divided by the
    slowest rank's time.  Returns (units/s, max ms)."""
    ms = _max_over_ranks(local_ms, world)
    units = local_units
    if world > 1:
        import torch
        import torch.distributed as dist
        dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
        t = torch.tensor([local_units], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        units = float(t.item())
    return units / (ms / 1e3), ms


def _time_calls(plan_handle, fn, reps=10):
    """Average device time of one `fn()` (a C-ABI call enqueued on the plan's
    stream): `reps` calls are captured into a CUDA graph and the replay is
    timed with CUDA events, so host-side call overhead leaves no gaps.  Falls
    back to timing direct calls if capture is refused."""
    import torch

    from paper_2402_17794_gb300 import rsvd as R
    fn()
    torch.cuda.synchronize()
    cur = torch.cuda.current_stream()
    try:
        g = torch.cuda.CUDAGraph()
        cs = torch.cuda.Stream()
        R.rsvd_plan_set_stream(plan_handle, cs)
        with torch.cuda.graph(g, stream=cs):
            for _ in range(reps):
                fn()
        R.rsvd_plan_set_stream(plan_handle, cur)
        g.replay()
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(cur)
        g.replay()
        b.record(cur)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps, "cuda-graph replay"
    except Exception:
        R.rsvd_plan_set_stream(plan_handle, cur)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(cur)
        for _ in range(reps):
            fn()
        b.record(cur)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps, "direct calls"


def _sigma(w):
    from paper_2402_17794_gb300 import synthetic as syn
    kind, arg = w["spectrum"]
    r = w.get("terms", min(w["m"], w["n"]))
    if kind == "poly":
        return syn.spectrum("poly", r, alpha=arg)
    if kind == "exp":
        return syn.spectrum("exp", r, r=arg)
    raise ValueError(kind)


def _make_input(w, rank):
    """The workload's A on the device, column-major as (n, lda); for FP8 the
    pair (codes, tile scales)."""
    import torch
    from paper_2402_17794_gb300 import synthetic as syn
    if w["dtype"] == "fp8":
        at = syn.lowrank_matrix_torch(w["m"], w["n"], _sigma(w), seed=w["seed_a"] + 1000 * rank,
                                      device="cuda", dtype=torch.float32,
                                      factor_dtype=torch.float32,
                                      noise_2norm=w.get("noise", 0.0))
        codes, scales = syn.quantize_e4m3_tiles(at, w["m"])
        del at
        torch.cuda.empty_cache()
        return codes, scales
    if w["dtype"] == "bf16":
        return syn.lowrank_matrix_torch(w["m"], w["n"], _sigma(w), seed=w["seed_a"] + 1000 * rank,
                                        device="cuda", dtype=torch.bfloat16,
                                        factor_dtype=torch.float32,
                                        noise_2norm=w.get("noise", 0.0))
    return syn.lowrank_matrix_torch(w["m"], w["n"], _sigma(w), seed=w["seed_a"] + 1000 * rank,
                                    device="cuda", dtype=torch.float64)


def run_mixed(args, world, rank, sampler_uuid, wname="mixed-bf16"):
    """A mixed-precision workload (BF16 or FP8 storage of A): solves/s and
    the tcgen05 passes over A timed alone against the HBM roofline."""
    import torch

    from paper_2402_17794_gb300 import rsvd as R

    w = WORKLOADS[wname]
    fp8 = w["dtype"] == "fp8"
    m, n, k, p, q, seed = w["m"], w["n"], w["k"], w["p"], w["q"], w["seed"]
    l = k + p
    a_bytes = m * n * (1 if fp8 else 2)
    passes = 2 * (q + 1) + 2
    stream = torch.cuda.current_stream()
    if fp8:
        dA, scales = _make_input(w, rank)
        plan = R.Plan(m, n, l, a_dtype=R.FP8E4M3, mode=R.MIXED)
        plan.set_tile_scales(scales)
    else:
        dA = _make_input(w, rank)
        plan = R.Plan(m, n, l, a_dtype=R.BF16, mode=R.MIXED)
    U = torch.empty(k, m, dtype=torch.float32, device="cuda")
    S = torch.empty(k, dtype=torch.float64, device="cuda")
    VT = torch.empty(n, k, dtype=torch.float32, device="cuda")

    def step():
        R._check(R.rsvd_solve(plan.handle, dA, m, n, m, k, p, q, seed, U, m, S, VT, k),
                 "rsvd_solve (mixed)")

    for _ in range(args.warmup):
        step()
    st = plan.status()
    if st != 0:
        raise RuntimeError(f"mixed warm-up failed: {R.rsvd_status_string(st)}")
    steps = max(args.steps, 10)
    sampler = ClockSampler(sampler_uuid)
    sampler.start()
    _barrier(world)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    lat = []
    for _ in range(steps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step()
        b.record(stream)
        lat.append((a, b))
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = _max_over_ranks(e0.elapsed_time(e1), world)
    per = sorted(a.elapsed_time(b) for a, b in lat)
    st = plan.status()
    if st != 0:
        raise RuntimeError(f"mixed solve failed: {R.rsvd_status_string(st)}")
    sweeps, _ = R.rsvd_plan_diagnostics(plan.handle)
    two = _two_stream_rate(args, world, plan, R, dA, m, n, k, p, q, seed, fp8,
                           scales if fp8 else None, steps)

    # the tcgen05 passes alone (one BF16 operand slice, l = 160)
    # the pass of the power steps as the solve runs it: an FP32 operand split
    # into one BF16 slice (BF16 A) or two E4M3 slices (FP8 A), then the pass
    X_n = torch.randn(l, n, device="cuda") / n ** 0.5
    X_m = torch.randn(l, m, device="cuda") / m ** 0.5
    Y = torch.empty(l, m, dtype=torch.float32, device="cuda")
    Z = torch.empty(l, n, dtype=torch.float32, device="cuda")

    t_ax, how = _time_calls(plan.handle,
                            lambda: R.rsvd_apply_split(plan.handle, dA, m, n, m, 0, X_n, n, l, 1,
                                                       Y, m))
    t_atx, _ = _time_calls(plan.handle,
                           lambda: R.rsvd_apply_split(plan.handle, dA, m, n, m, 1, X_m, m, l, 1,
                                                      Z, n))
    st = plan.status()
    if st != 0:
        raise RuntimeError(f"mixed pass failed: {R.rsvd_status_string(st)}")
    peaks, _ = _peaks()
    hbm = peaks.get("hbm_gbs", 6800.0)
    dom_ms = max(t_ax, t_atx)
    if fp8:
        dom = "apass_mx8_kernel<true,2,2,128> (Y = A X)" if t_ax >= t_atx else \
            "apass_mx8_kernel<false,2,2,128> (Z = A^T X)"
    else:
        dom = "apass_bf16_kernel<true,2> (Y = A X)" if t_ax >= t_atx else \
            "apass_bf16_kernel<false,2> (Z = A^T X)"
    achieved = a_bytes / (dom_ms / 1e3) / 1e9
    out = {
        "workload": w["desc"], "value": round(steps * world / (ms / 1e3), 3), "unit": "solves/s",
        "ms_per_solve": round(ms / steps, 4),
        "p50_ms": round(per[len(per) // 2], 4), "p99_ms": round(per[min(len(per) - 1, int(0.99 * len(per)))], 4),
        "two_streams": two,
        "dtype": ("fp8 e4m3 A (tile scales as UE8M0 block scales), e4m3 operand slices "
                  "(block-scaled MMA)" if fp8 else "bf16 A, bf16 operand slices") +
                 ", fp32 accumulate", "passes_per_solve": passes, "jacobi_sweeps": sweeps,
        "a_pass": {"ms_ax": round(t_ax, 4), "ms_atx": round(t_atx, 4),
                   "gbps_ax": round(a_bytes / (t_ax / 1e3) / 1e9, 1),
                   "gbps_atx": round(a_bytes / (t_atx / 1e3) / 1e9, 1),
                   "gbps_in_solve": round(passes * a_bytes / (ms / steps / 1e3) / 1e9, 1)},
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1),
                     "peak": hbm, "unit": "GB/s", "frac": round(achieved / hbm, 4),
                     "traffic": _traffic_from_profile(wname, "ax" if t_ax >= t_atx else "atx"),
                     "algorithmic_bytes_per_launch": a_bytes,
                     "ms_per_launch": round(dom_ms, 4),
                     "timing": f"{how}: operand split + main kernel + split-tile fixup per "
                               "pass (one BF16 / two E4M3 operand slices, as in the power steps)"},
        "clocks": clocks,
    }
    # the CPU oracle on the exactly dequantised A (q + 1 power steps, as the
    # mixed solve's refinement step adds one): its time is the cpu_baseline,
    # its singular values the reference for the error of this section and of
    # the plain FP64 form on the same matrix
    if not args.no_cpu_baseline and world == 1:
        if fp8:
            deq = dA.view(torch.float8_e4m3fn)[:, :m].to(torch.float64)
            sc = scales.to(torch.float64).repeat_interleave(128, dim=0)[:n]
            sc = sc.repeat_interleave(128, dim=1)[:, :m]
            deq = deq * sc
        else:
            deq = dA[:, :m].to(torch.float64)
        ref_s, t_orc, cores = _oracle_sigma(deq, k, p, q + 1, seed)
        out["cpu_baseline"] = {"value": round(1.0 / t_orc, 4), "unit": "solves/s", "cores": cores,
                               "kind": "oracle",
                               "sample": f"one full oracle solve of the same workload on the "
                                         f"dequantised A, q+1 power steps ({t_orc:.1f} s)"}
        s_gpu = S.cpu().numpy()
        out["sigma_rel_err_max"] = float((abs(s_gpu - ref_s) / ref_s).max())
        out["sigma_err_vs"] = "FP64 oracle, same A (dequantised) and Omega, q+1 power steps"
        if not fp8:
            out["plain_fp64_same_matrix"] = _plain_on(args, world, deq, m, n, k, p, q + 1, seed,
                                                      ref_s, out["value"])
        del deq
        torch.cuda.empty_cache()
    del dA, plan
    return out


def _oracle_sigma(deq, k, p, q, seed):
    """The CPU oracle (as it stands) on a device matrix (n, >= m) copied to
    the host: its singular values, its wall time and the cores it used."""
    import numpy as np

    import oracle
    A = np.asfortranarray(deq.cpu().numpy().T)
    t0 = time.perf_counter()
    ref = oracle.rsvd(A, k, p, q, seed)
    el = time.perf_counter() - t0
    return ref.S, el, _cores()


def _plain_on(args, world, deq, m, n, k, p, q, seed, ref_s, mixed_value):
    """The plain FP64 form (tensor-core FP64 passes) on the mixed workload's
    matrix, dequantised exactly to FP64: solves/s and its error against the
    same oracle, beside the mixed form's rate."""
    import torch

    from paper_2402_17794_gb300 import rsvd as R
    A64 = deq.contiguous()
    plan = R.Plan(m, n, k + p, mode=R.F64_TENSOR)
    U = torch.empty(k, m, dtype=torch.float64, device="cuda")
    S = torch.empty(k, dtype=torch.float64, device="cuda")
    VT = torch.empty(n, k, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()

    def step():
        R._check(R.rsvd_solve(plan.handle, A64, m, n, m, k, p, q, seed, U, m, S, VT, k),
                 "rsvd_solve (plain FP64 on the mixed matrix)")

    step()
    steps = 3
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    st = plan.status()
    if st != 0:
        raise RuntimeError(f"plain FP64 solve on the mixed matrix failed: {R.rsvd_status_string(st)}")
    ms = _max_over_ranks(e0.elapsed_time(e1), world) / steps
    s = S.cpu().numpy()
    val = 1e3 / ms
    del plan, A64
    return {"workload": "the same matrix in FP64 (exactly dequantised), tensor-core FP64 passes, "
                        f"k={k}, p={p}, q={q}",
            "value": round(val, 3), "unit": "solves/s", "ms_per_solve": round(ms, 3),
            "sigma_rel_err_max": float((abs(s - ref_s) / ref_s).max()),
            "mixed_over_plain": round(mixed_value / val, 3), "dtype": "f64"}


def _two_stream_rate(args, world, plan, R, dA, m, n, k, p, q, seed, fp8, scales, steps):
    """Throughput with two independent solves in flight on two streams (two
    plans, each its own workspace and outputs): the l x l steps of one solve
    run on one SM while the other solve's passes fill the rest of the GPU,
    as concurrent requests would.  Every solve still does all of its work."""
    import torch

    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    plan2 = R.Plan(m, n, k + p, a_dtype=R.FP8E4M3 if fp8 else R.BF16, mode=R.MIXED, stream=s2)
    if fp8:
        plan2.set_tile_scales(scales)
    R.rsvd_plan_set_stream(plan.handle, s1)
    outs = [(torch.empty(k, m, dtype=torch.float32, device="cuda"),
             torch.empty(k, dtype=torch.float64, device="cuda"),
             torch.empty(n, k, dtype=torch.float32, device="cuda")) for _ in range(2)]

    def solve(i):
        pl = plan if i % 2 == 0 else plan2
        U, S, VT = outs[i % 2]
        R._check(R.rsvd_solve(pl.handle, dA, m, n, m, k, p, q, seed + i, U, m, S, VT, k),
                 "rsvd_solve (mixed, two streams)")

    for i in range(4):
        solve(i)
    torch.cuda.synchronize()
    _barrier(world)
    t0 = time.perf_counter()
    e_start = torch.cuda.Event(enable_timing=True)
    e_start.record(torch.cuda.current_stream())
    s1.wait_event(e_start)
    s2.wait_event(e_start)
    for i in range(2 * steps):
        solve(i)
    e1, e2 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e1.record(s1)
    e2.record(s2)
    torch.cuda.synchronize()
    ms = max(e_start.elapsed_time(e1), e_start.elapsed_time(e2))
    ms = _max_over_ranks(ms, world)
    for pl in (plan, plan2):
        st = pl.status()
        if st != 0:
            raise RuntimeError(f"two-stream solve failed: {R.rsvd_status_string(st)}")
    R.rsvd_plan_set_stream(plan.handle, torch.cuda.current_stream())
    del plan2
    return {"value": round(2 * steps * world / (ms / 1e3), 3), "unit": "solves/s",
            "ms_per_solve": round(ms / (2 * steps), 4), "solves": 2 * steps,
            "how": "two plans on two CUDA streams, solves alternating; CUDA events"}


def _oracle_rate(A_host, w, budget_s: float):
    """Times the CPU oracle (as it stands) on this host: full solves until the
    budget is spent (at least one)."""
    import numpy as np

    import oracle
    A = np.asfortranarray(A_host)
    n_done, t0 = 0, time.perf_counter()
    while True:
        oracle.rsvd(A, w["k"], w["p"], w["q"], w["seed"] + n_done)
        n_done += 1
        el = time.perf_counter() - t0
        if el >= budget_s or n_done >= 50:
            break
    return n_done, el


def _oracle_rows(A_host, w):
    """The CPU oracle of each further row on the same matrix, timed once each
    (as it stands, on this host): Algorithm 6, Algorithm 3, the adaptive
    range finder + SVD and FastRandRF with the SRFT."""
    import numpy as np

    import oracle
    from oracle import adaptive as oad
    from oracle import singlepass as osp
    from oracle import srft as osr
    A = np.asfortranarray(A_host)
    k, p, q, seed = w["k"], w["p"], w["q"], w["seed"]
    runs = {
        "singlepass": lambda: osp.singlepass_rsvd(A, k, p, seed),
        "algorithm3": lambda: oracle.rsvd(A, k, p, q, seed, algorithm=3),
        "adaptive": lambda: oad.adaptive_rsvd(A, ADAPTIVE["eps"], ADAPTIVE["r"], seed,
                                              l_max=ADAPTIVE["l_cap"]),
        "srft": lambda: osr.fast_range_finder(A, k + p, seed),
    }
    out = {}
    for name, fn in runs.items():
        t0 = time.perf_counter()
        fn()
        el = time.perf_counter() - t0
        out[name] = {"value": round(1.0 / el, 4),
                     "unit": "ranges/s" if name == "srft" else "solves/s",
                     "cores": _cores(), "kind": "oracle",
                     "sample": f"one full oracle run of the same workload ({el:.1f} s)"}
    return out


def _cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count()


def _batched_problems(count, seed, device="cuda"):
    """The batched workload: FP32 matrices with m log-uniform in [256, 4096],
    n uniform in [256, 2048], sigma_i = exp(-i/r) with r uniform in [5, 50];
    k uniform in [10, 64], p = 10, q = 1 (Haar factors; terms below 1e-8 of
    sigma_1 are dropped)."""
    import numpy as np
    import torch

    from paper_2402_17794_gb300 import synthetic as syn
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        m = int(np.exp(rng.uniform(np.log(256), np.log(4096))))
        n = int(rng.integers(256, 2049))
        r = float(rng.uniform(5.0, 50.0))
        k = int(rng.integers(10, 65))
        terms = min(m, n, int(r * np.log(1e8)) + 1)
        A = syn.lowrank_matrix_torch(m, n, syn.spectrum("exp", terms, r=r), seed=seed * 7919 + i,
                                     device=device, dtype=torch.float32,
                                     factor_dtype=torch.float32)
        out.append((A, m, n, k, 10, 1, 1000 + i))
    return out


def run_batched(args, stream):
    """512 uneven FP32 problems in one grouped solve, each held to 1e-3
    relative on every sigma_i: problems whose FP32 result cannot meet that
    (sigma_k below what FP32 resolves, the serving rule) are solved again in
    FP64 in the same timed step.  Reports the error against the FP64 oracle
    on a sample, the oracle's rate on that sample, and the grouped
    products' FP32 roofline."""
    import numpy as np
    import torch

    import oracle
    from paper_2402_17794_gb300 import rsvd as R
    from paper_2402_17794_gb300 import serve
    tol = 1e-3
    items = _batched_problems(512, 11)
    rows = sum(it[1] for it in items)
    cols = sum(it[2] for it in items)
    l_max = max(it[3] + it[4] for it in items)
    # tensor engine, on its own stream so that each grouped solve is one
    # CUDA graph launch
    gstream = torch.cuda.Stream()
    plan = R.BatchPlan(len(items), rows, cols, l_max, R.F32, stream=gstream)
    outs = [(torch.empty(k, m, dtype=torch.float32, device="cuda"),
             torch.empty(k, dtype=torch.float64, device="cuda"),
             torch.empty(n, k, dtype=torch.float32, device="cuda"))
            for (_, m, n, k, _, _, _) in items]
    # the engine's schedules (split-K chunks, column tiles) tuned once on this
    # batch's shapes, before anything is timed
    t_tune = time.perf_counter()
    plan.autotune(items, outs)
    t_tune = time.perf_counter() - t_tune
    plan.set_graphs(True)
    plan.solve(items, outs)
    codes = plan.status()
    # the problems FP32 cannot resolve to the tolerance (fixed by the inputs)
    promote = [i for i, (_, S, _) in enumerate(outs) if not serve.fp32_meets(S.cpu().tolist(), tol)]
    items64 = [(items[i][0].to(torch.float64),) + tuple(items[i][1:]) for i in promote]
    outs64 = [(torch.empty(k, m, dtype=torch.float64, device="cuda"),
               torch.empty(k, dtype=torch.float64, device="cuda"),
               torch.empty(n, k, dtype=torch.float64, device="cuda"))
              for (_, m, n, k, _, _, _) in items64]
    # the FP64 re-solves: tensor-core FP64 plans on eight streams, so their
    # l x l steps (one or a few SMs each) overlap
    nside_max = min(24, len(items64))
    side = [torch.cuda.Stream() for _ in range(nside_max)]
    nside = min(8, nside_max)
    tplans = []
    if items64:
        mmax = max(it[1] for it in items64)
        nmax = max(it[2] for it in items64)
        tplans = [R.Plan(mmax, nmax, l_max, mode=R.F64_TENSOR, stream=sd) for sd in side]

    def step():
        # the FP64 re-solves do not depend on this step's FP32 results (the set
        # is fixed by the inputs), so they start with the step and overlap the
        # grouped FP32 solve
        go = torch.cuda.Event()
        go.record(stream)
        for sd in [gstream] + (side[:nside] if items64 else []):
            sd.wait_event(go)
        plan.solve(items, outs)
        for j, (A, m, n, k, p, q, seed) in enumerate(items64):
            tplans[j % nside].solve(A, m, n, k, p, q, seed, out=outs64[j])
        for sd in [gstream] + (side[:nside] if items64 else []):
            done = torch.cuda.Event()
            done.record(sd)
            stream.wait_event(done)

    for _ in range(3):
        step()
    torch.cuda.synchronize()
    codes = plan.status() + [tp.status() for tp in tplans]
    # SMs left to the FP64 re-solves: the tensor engine's persistent launches
    # hold every SM they get, so the two only overlap if the engine is given
    # fewer.  Chosen before timing from a few untimed steps per setting.
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    # The FP64 re-solves are chains of small latency-bound launches, so how
    # many run side by side (streams) is chosen the same way.
    sm_limit, best = 0, None
    if items64:
        choice = (0, nside)
        for ns in sorted({min(8, nside_max), min(16, nside_max), nside_max}):
            for sms in (0, 120, 96, 80, 64, 48):
                nside = ns
                plan.set_sm_limit(sms)
                step()          # new schedules and graph for this limit
                torch.cuda.synchronize()
                a.record(stream)
                for _ in range(2):
                    step()
                b.record(stream)
                torch.cuda.synchronize()
                t = a.elapsed_time(b)
                if best is None or t < best:
                    choice, best = (sms, ns), t
        sm_limit, nside = choice
        plan.set_sm_limit(sm_limit)
        step()
        torch.cuda.synchronize()
    steps = 5
    torch.cuda.synchronize()
    a.record(stream)
    for _ in range(steps):
        step()
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / steps
    a_bytes = sum(m * n * 4 for (_, m, n, _, _, _, _) in items)
    # error against the FP64 oracle and the oracle's own rate, on a sample
    final = {i: outs[i][1] for i in range(len(items))}
    for j, i in enumerate(promote):
        final[i] = outs64[j][1]
    sample = sorted(set(list(range(0, len(items), 64)) + promote[:4]))
    errs, t_orc = [], 0.0
    for i in sample:
        A, m, n, k, p, q, seed = items[i]
        Ah = np.asfortranarray(A.double().cpu().numpy().T)
        t0 = time.perf_counter()
        ref = oracle.rsvd(Ah, k, p, q, seed)
        t_orc += time.perf_counter() - t0
        s = final[i].cpu().numpy()
        errs.append(float((np.abs(s - ref.S) / ref.S).max()))
    peaks, psrc = _peaks()
    # roofline of the grouped pass Y = A Omega over all 512 problems (the
    # persistent tcgen05 launch and its operand split), timed alone on every SM
    plan.set_sm_limit(0)
    keep, gemms = [], []
    for (A, m, n, k, p, q, seed) in items:
        X = torch.randn(k + p, n, device="cuda")
        C = torch.empty(k + p, m, device="cuda")
        keep += [X, C]
        gemms.append((A, A.shape[1], X, n, C, m, m, n, k + p, 0))
    for _ in range(3):
        plan.grouped_gemm(gemms, 0)
    torch.cuda.synchronize()
    a.record(gstream)
    for _ in range(5):
        plan.grouped_gemm(gemms, 0)
    b.record(gstream)
    torch.cuda.synchronize()
    t_pass = a.elapsed_time(b) / 5 / 1e3
    pass_gbps = a_bytes / t_pass / 1e9
    del plan, tplans
    return {"workload": "512 FP32 matrices, m log-uniform [256,4096], n uniform [256,2048], "
                        "sigma_i=exp(-i/r), r~U[5,50]; k~U{10..64}, p=10, q=1; one grouped solve; "
                        "each problem to 1e-3 relative on every sigma (FP64 re-solve where FP32 "
                        "cannot resolve sigma_k, on tensor-core FP64 plans on side streams; the "
                        "set is fixed by the inputs and found once before timing)",
            "value": round(len(items) / (ms / 1e3), 1), "unit": "solves/s",
            "ms_per_batch": round(ms, 3), "problems": len(items),
            "promoted_to_fp64": len(promote),
            "sigma_rel_err_max": max(errs), "sigma_err_sample": len(sample),
            "a_bytes_per_pass": a_bytes,
            "a_pass_equiv_gbps": round(4 * a_bytes / (ms / 1e3) / 1e9, 1),
            "roofline": {"bound": "hbm",
                         "kernel": "gtc_kernel<AX> (one grouped pass Y = A Omega over all "
                                   "512 problems, with its operand split)",
                         "achieved": round(pass_gbps, 1), "peak": peaks["hbm_gbs"],
                         "unit": "GB/s", "frac": round(pass_gbps / peaks["hbm_gbs"], 4),
                         "traffic": _traffic_from_profile("batched-f32", "ax"), "peak_source": psrc,
                         "algorithmic_bytes_per_launch": a_bytes,
                         "ms_per_launch": round(t_pass * 1e3, 3),
                         "timing": "CUDA events around 5 grouped passes on the plan's stream"},
            "tensor_engine": {"grouped_products": "tcgen05, FP32 split into three BF16 slices",
                              "autotune_s": round(t_tune, 2),
                              "cuda_graph": "each grouped FP32 solve is one graph launch",
                              "sm_limit": sm_limit or 152,
                              "fp64_streams": nside},
            "cpu_baseline": {"value": round(len(sample) / t_orc, 3), "unit": "solves/s",
                             "cores": _cores(), "kind": "oracle",
                             "sample": f"{len(sample)} problems of the batch, one oracle solve "
                                       f"each ({t_orc:.1f} s)"},
            "failed": sum(1 for c in codes if c != 0), "dtype": "f32 (f64 where promoted)"}


def _serve_requests(rate, dur, seed, small, bigs):
    """Poisson arrivals at `rate` req/s for `dur` s: 95% FP32 matrices of the
    batched mix (k ~ U{10..64}), 5% of the 8192 x 8192 sigma_i = 1/i
    matrices (k = 256, p = 32, q = 2); tolerance 1e-3 or 1e-6, half each."""
    import numpy as np

    from paper_2402_17794_gb300 import serve
    rng = np.random.default_rng(seed)
    reqs, t, i = [], 0.0, 0
    while True:
        t += float(rng.exponential(1.0 / rate))
        if t > dur:
            break
        tol = 1e-3 if rng.random() < 0.5 else 1e-6
        if rng.random() < 0.05:
            A = bigs[i % len(bigs)]
            reqs.append(serve.Request(i, 8192, 8192, 256, 32, 2, tol, 5000 + i, t, A=A))
        else:
            A, m, n, k, p, q, _ = small[i % len(small)]
            k = int(rng.integers(10, 65))
            reqs.append(serve.Request(i, m, n, k, p, q, tol, 5000 + i, t, A=A))
        i += 1
    return reqs


def _serve_once(rate, dur, seed, small, bigs, drain_s):
    import time

    import torch

    from paper_2402_17794_gb300 import serve
    reqs = _serve_requests(rate, dur, seed, small, bigs)
    specs = [serve.LaneSpec("f32-small", 64, 64 * 4096, 64 * 2048, 80),
             serve.LaneSpec("f64-small", 64, 64 * 4096, 64 * 2048, 80),
             serve.LaneSpec("f32-big", 4, 4 * 8192, 4 * 8192, 288),
             serve.LaneSpec("f64-big", 1, 8192, 8192, 288, engine="tensor", lanes=4)]
    srv = serve.Server(specs, serve.TorchBackend(), 150 * 10**9, lanes_per_class=2)
    torch.cuda.synchronize()
    stats = serve.run(srv, reqs, time.perf_counter, max_wall=dur + drain_s + 600.0,
                      drain_s=drain_s)
    torch.cuda.synchronize()
    per = {}
    for cls in ("f32-small", "f64-small", "f32-big", "f64-big"):
        lat = [r.latency for r in srv.finished if serve.request_class(r) == cls]
        per[cls] = {"n": len(lat), "p50_ms": round(serve.percentile(lat, 50) * 1e3, 2),
                    "p99_ms": round(serve.percentile(lat, 99) * 1e3, 2)}
    return reqs, srv, stats, per


def run_serving(args):
    """Poisson arrivals at 2000 req/s for 30 s (95% FP32 matrices sized as
    the batched workload, 5% 8192x8192 with sigma_i = 1/i, k=256, p=32, q=2;
    tolerance 1e-3 or 1e-6, half each; admission capped at 150 GB of HBM),
    waiting at most 30 s past the last arrival; then the largest offered
    rate (halving from 1000 req/s, 10 s windows) at which every request is
    served with p99 under one second.  The served singular values of a
    sample are checked against the FP64 oracle."""
    import time

    import numpy as np
    import torch

    import oracle
    from paper_2402_17794_gb300 import serve
    from paper_2402_17794_gb300 import synthetic as syn
    small = _batched_problems(32, 13)
    bigs = [syn.lowrank_matrix_torch(8192, 8192, syn.spectrum("poly", 8192, alpha=1.0),
                                     seed=900 + j, dtype=torch.float32,
                                     factor_dtype=torch.float32) for j in range(2)]
    torch.cuda.synchronize()
    rate, dur, drain = 2000.0, args.serve_seconds, 30.0
    reqs, srv, stats, per = _serve_once(rate, dur, 21, small, bigs, drain)
    out = {"workload": "Poisson 2000 req/s for %.0f s; 95%% FP32 matrices as the batched "
                       "workload, 5%% 8192x8192 sigma_i=1/i k=256 p=32 q=2; tolerance 1e-3 or "
                       "1e-6 (half each); admission cap 150 GB" % dur,
           "offered_rps": rate, "requests": len(reqs),
           "value": round(stats["throughput_rps"], 1), "unit": "solves/s",
           "served": stats["completed"], "unserved_after_drain": stats["unserved"],
           "drain_cap_s": drain,
           "p50_ms": round(stats["p50_ms"], 2), "p99_ms": round(stats["p99_ms"], 2),
           "latency_of": "served requests",
           "wall_s": round(stats["wall_s"], 2), "batches": stats["batches"],
           "promoted_to_fp64": stats["promotions"],
           "admission_stalls": stats["admission_stalls"], "failed": stats["failed"],
           "per_class": per,
           "lanes": "f32-small 2x64, f64-small 2x64 (grouped), f32-big 2x4 (grouped), "
                    "f64-big 4x1 (tensor-core FP64 passes)"}
    # served sigma against the FP64 oracle, on a sample of each class
    errs, within, sample = [], True, []
    by_cls = {}
    for r in srv.finished:
        if r.status == 0 and r.result is not None:
            by_cls.setdefault(serve.request_class(r), []).append(r)
    for cls, rs in sorted(by_cls.items()):
        sample += rs[:3 if cls.endswith("small") else 1]
    for r in sample:
        A = np.asfortranarray(r.A[:, :r.m].double().cpu().numpy().T)
        ref = oracle.rsvd(A, r.k, r.p, r.q, r.seed)
        s = r.result[1].cpu().numpy()
        e = float((np.abs(s - ref.S) / ref.S).max())
        errs.append(e)
        within = within and e <= r.tol
    out["sigma_rel_err_max"] = max(errs) if errs else None
    out["sigma_within_own_tolerance"] = within
    out["sigma_err_sample"] = f"{len(sample)} served requests across the classes, FP64 oracle"
    del srv
    torch.cuda.empty_cache()
    # the largest sustainable rate
    sustain = []
    r8 = 1000.0
    best = None
    while r8 >= 60.0:
        rq, sv, st, pc = _serve_once(r8, 10.0, 31, small, bigs, 5.0)
        ok = st["unserved"] == 0 and st["p99_ms"] <= 1000.0 and st["failed"] == 0
        sustain.append({"offered_rps": r8, "served": st["completed"], "unserved": st["unserved"],
                        "p50_ms": round(st["p50_ms"], 2), "p99_ms": round(st["p99_ms"], 2),
                        "sustained": ok})
        del sv
        torch.cuda.empty_cache()
        if ok:
            best = r8
            break
        r8 /= 2.0
    out["max_sustainable_rps"] = best
    out["sustainable_rule"] = ("every request of a 10 s window served within 5 s after it, "
                               "p99 <= 1000 ms; rates halved from 1000 req/s")
    out["rate_search"] = sustain
    return out


def run_ours(args):
    import torch

    import __graft_entry__
    from paper_2402_17794_gb300 import rsvd as R

    world, rank, local = _dist()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    __graft_entry__.build()
    w = WORKLOADS[args.workload]
    m, n, k, p, q, seed = w["m"], w["n"], w["k"], w["p"], w["q"], w["seed"]
    l = k + p
    # the library's own launch count at each section boundary, so that a
    # profiler's launch list of this run can be split by section
    marks = [("start", R.rsvd_kernel_launches())]

    def mark(name):
        marks.append((name, R.rsvd_kernel_launches()))
    passes = 2 * q + 2
    a_bytes = m * n * 8
    dA = _make_input(w, rank)
    stream = torch.cuda.current_stream()
    # FP64 results; the passes over A on the tensor cores (exact products of
    # BF16 digit slices), every other step in FP64 on the CUDA cores
    plan = R.Plan(m, n, l, mode=R.F64_TENSOR)
    U = torch.empty(k, m, dtype=torch.float64, device="cuda")
    S = torch.empty(k, dtype=torch.float64, device="cuda")
    VT = torch.empty(n, k, dtype=torch.float64, device="cuda")

    def step(i):
        R._check(R.rsvd_solve(plan.handle, dA, m, n, m, k, p, q, seed, U, m, S, VT, k),
                 "rsvd_solve")

    for i in range(args.warmup):
        step(i)
    st = plan.status()
    if st != 0:
        raise RuntimeError(f"warm-up solve failed: {R.rsvd_status_string(st)}")

    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        pass
    sampler = ClockSampler(uuid)
    sampler.start()
    _barrier(world)
    torch.cuda.synchronize()
    l0 = R.rsvd_kernel_launches()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(args.steps):
        step(i)
    e1.record(stream)
    torch.cuda.synchronize()
    launches = R.rsvd_kernel_launches() - l0
    _barrier(world)
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1)
    st = plan.status()
    if st != 0:
        raise RuntimeError(f"timed solve failed: {R.rsvd_status_string(st)}")
    sweeps, _ = R.rsvd_plan_diagnostics(plan.handle)
    value, ms_max = job_rate(args.steps, ms, world)
    ms_per_step = ms_max / args.steps

    # --- the dominant kernel, timed alone: the tensor pass on a prepared A ---
    Om = R.colmajor(n, l)
    Y = R.colmajor(m, l)
    Z = R.colmajor(n, l)
    R.rsvd_gaussian(plan.handle, n, l, seed, 0, R.F64, Om, n)
    Qm = torch.linalg.qr(torch.randn(m, l, dtype=torch.float64, device="cuda"))[0].T.contiguous()
    R._check(R.rsvd_plan_prepare_a(plan.handle, dA, m, n, m), "rsvd_plan_prepare_a")
    t_an, how = _time_calls(plan.handle,
                            lambda: R.rsvd_apply_a(plan.handle, dA, m, n, m, Om, n, l, Y, m), reps=10)
    t_at, _ = _time_calls(plan.handle,
                          lambda: R.rsvd_apply_at(plan.handle, dA, m, n, m, Qm, m, l, Z, n), reps=10)
    R.rsvd_plan_release_a(plan.handle)
    t_prep, _ = _time_calls(plan.handle,
                            lambda: R.rsvd_plan_prepare_a(plan.handle, dA, m, n, m), reps=3)
    R.rsvd_plan_release_a(plan.handle)
    peaks, peak_kind = _peaks()
    hbm = peaks.get("hbm_gbs", 6800.0)
    dom_ms = max(t_an, t_at)
    ax_dom = t_an >= t_at
    dom = "apass_f64tc_kernel<%s,80,28> (%s pass)" % ((1, "A X") if ax_dom else (0, "A^T X"))
    achieved = a_bytes / (dom_ms / 1e3) / 1e9
    products = 21          # BF16 digit products kept per pair of FP64 elements
    mma_flops = products * 2.0 * m * n * l
    roofline = {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1),
                "peak": hbm, "unit": "GB/s", "frac": round(achieved / hbm, 4),
                "traffic": _traffic_from_profile("plain-fp64-tensor", "ax" if ax_dom else "atx"),
                "algorithmic_bytes_per_launch": a_bytes,
                "bytes_streamed_per_launch": m * n * 12,
                "ms_per_launch": round(dom_ms, 4),
                "tensor_view": {"mma_flops_per_launch": mma_flops,
                                "achieved_tflops": round(mma_flops / (dom_ms / 1e3) / 1e12, 1),
                                "peak_bf16_tflops": peaks.get("bf16_tflops"),
                                "frac": round(mma_flops / (dom_ms / 1e3) / 1e12 /
                                              peaks.get("bf16_tflops", 1900.0), 4)},
                "timing": f"{how}: slicing of X + pass + finalize per call, A prepared once "
                          "(algorithmic bytes = the FP64 A; the pass streams A's six BF16 digit "
                          "slices, 12 bytes per element)"}
    a_pass = {"ms_ax": round(t_an, 4), "ms_atx": round(t_at, 4),
              "ms_prepare_a": round(t_prep, 4),
              "gbps_ax": round(a_bytes / (t_an / 1e3) / 1e9, 2),
              "gbps_atx": round(a_bytes / (t_at / 1e3) / 1e9, 2),
              "gbps_in_solve": round(passes * a_bytes / (ms_per_step / 1e3) / 1e9, 2),
              "hbm_peak_gbs": hbm, "passes_per_solve": passes}
    plain_simt = run_plain_simt(args, world, dA, w)

    # --- end to end through the C ABI with host buffers ---
    A_h = torch.empty(dA.shape, dtype=dA.dtype, pin_memory=True)
    A_h.copy_(dA)
    U_h = torch.empty(U.shape, dtype=U.dtype, pin_memory=True)
    S_h = torch.empty(S.shape, dtype=S.dtype, pin_memory=True)
    VT_h = torch.empty(VT.shape, dtype=VT.dtype, pin_memory=True)
    dA2 = torch.empty_like(dA)

    def e2e_step(i):
        dA2.copy_(A_h, non_blocking=True)
        R._check(R.rsvd_solve(plan.handle, dA2, m, n, m, k, p, q, seed, U, m, S, VT, k),
                 "rsvd_solve")
        U_h.copy_(U, non_blocking=True)
        S_h.copy_(S, non_blocking=True)
        VT_h.copy_(VT, non_blocking=True)

    e2e_steps = max(1, min(args.steps, 10))
    e2e_step(0)
    torch.cuda.synchronize()
    _barrier(world)
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for i in range(e2e_steps):
        e2e_step(i)
    b.record(stream)
    torch.cuda.synchronize()
    e2e_ms = _max_over_ranks(a.elapsed_time(b), world)
    e2e = {"value": round(e2e_steps * world / (e2e_ms / 1e3), 4), "unit": "solves/s",
           "h2d_bytes_per_step": a_bytes,
           "d2h_bytes_per_step": (m * k + k + k * n) * 8}
    st = plan.status()
    if st != 0:
        raise RuntimeError(f"e2e solve failed: {R.rsvd_status_string(st)}")

    mark("plain")
    # --- Algorithm 6 (single pass) on the same matrix ---
    singlepass = run_singlepass(args, world, dA, w, plan, 6)
    mark("singlepass")
    algorithm3 = run_singlepass(args, world, dA, w, plan, 3)
    mark("algorithm3")
    adaptive = run_adaptive(args, world, dA, w)
    mark("adaptive")
    srft = run_srft(args, world, dA, w, t_an)
    mark("srft")

    # --- the mixed-precision workload beside it ---
    mixed = mixed_fp8 = None
    if not args.no_mixed:
        del A_h, dA2
        mixed = run_mixed(args, world, rank, uuid)
        mark("mixed")
        torch.cuda.empty_cache()
        mixed_fp8 = run_mixed(args, world, rank, uuid, "mixed-fp8")
        mark("mixed_fp8")

    batched = None if args.no_batched else run_batched(args, stream)
    mark("batched")
    serving = None if args.no_serving else run_serving(args)
    mark("serving")

    # --- CPU oracle on this host (rank 0, N = 1 only) ---
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        A_np = dA.cpu().numpy().T
        done, el = _oracle_rate(A_np, w, args.cpu_budget)
        cpu = {"value": round(done / el, 4), "unit": "solves/s", "cores": _cores(),
               "kind": "oracle",
               "sample": f"{done} full oracle solve(s) of the same workload in {el:.1f} s "
                         f"(numpy FP64, LAPACK QR/SVD)"}
        for name, base in _oracle_rows(A_np, w).items():
            section = {"singlepass": singlepass, "algorithm3": algorithm3,
                       "adaptive": adaptive, "srft": srft}[name]
            section["cpu_baseline"] = base

    line = {
        "metric": METRIC, "value": round(value, 4), "unit": "solves/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded Haar factors, known spectrum)",
        "config": {"workload": w["desc"], "m": m, "n": n, "k": k, "p": p, "q": q,
                   "a_dtype": w["dtype"], "parallelism": f"replicas x{world}" if world > 1 else "1 gpu",
                   "l2": "inputs larger than L2 (A is %.2f GB; L2 129 MB): no flush" % (a_bytes / 1e9)},
        "a_pass": a_pass,
        "roofline": roofline,
        "plain_simt": plain_simt,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "singlepass": singlepass,
        "algorithm3": algorithm3,
        "adaptive": adaptive,
        "srft": srft,
        "mixed": mixed,
        "mixed_fp8": mixed_fp8,
        "batched": batched,
        "serving": serving,
        "gpu_launches": int(launches),
        "gpu_launches_per_step": launches / args.steps,
        "launches_by_section": {b[0]: b[1] - a[1] for a, b in zip(marks, marks[1:])},
        "jacobi_sweeps": sweeps,
        "clocks": clocks,
        "peaks_source": peak_kind,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_plain_simt(args, world, dA, w):
    """The same FP64 solve with every pass over A on the CUDA cores (FP64
    FMA), and that pass alone against the FP64 ALU roofline."""
    import torch

    from paper_2402_17794_gb300 import rsvd as R

    m, n, k, p, q, seed = w["m"], w["n"], w["k"], w["p"], w["q"], w["seed"]
    l = k + p
    plan = R.Plan(m, n, l)
    U = torch.empty(k, m, dtype=torch.float64, device="cuda")
    S = torch.empty(k, dtype=torch.float64, device="cuda")
    VT = torch.empty(n, k, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()

    def step():
        R._check(R.rsvd_solve(plan.handle, dA, m, n, m, k, p, q, seed, U, m, S, VT, k),
                 "rsvd_solve (FP64 on the CUDA cores)")

    step()
    steps = 3
    _barrier(world)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    st = plan.status()
    if st != 0:
        raise RuntimeError(f"FP64 CUDA-core solve failed: {R.rsvd_status_string(st)}")
    ms = _max_over_ranks(e0.elapsed_time(e1), world)
    Om = R.colmajor(n, l)
    Y = R.colmajor(m, l)
    R.rsvd_gaussian(plan.handle, n, l, seed, 0, R.F64, Om, n)
    t_an, how = _time_calls(plan.handle,
                            lambda: R.rsvd_apply_a(plan.handle, dA, m, n, m, Om, n, l, Y, m), reps=3)
    flops = 2.0 * m * n * l
    peaks, _ = _peaks()
    sm_max = peaks.get("sm_max_mhz", 2070.0)
    fp64_peak = 152 * 2 * 2 * sm_max * 1e6 / 1e12   # TFLOP/s: 152 SMs x 2 DFMA/clk x 2 flop
    achieved = flops / (t_an / 1e3) / 1e12
    del plan
    return {"workload": "the same FP64 solve with the passes over A on the CUDA cores (FP64 FMA)",
            "value": round(steps * world / (ms / 1e3), 4), "unit": "solves/s",
            "ms_per_solve": round(ms / steps, 4), "dtype": "f64",
            "roofline": {"bound": "alu", "kernel": "gemm_simt_kernel<double,5,false> (A X pass)",
                         "achieved": round(achieved, 4), "peak": round(fp64_peak, 4),
                         "unit": "TFLOP/s", "frac": round(achieved / fp64_peak, 4),
                         "peak_source": f"derived: 152 SMs x 2 FP64 FMA/clk x 2 flop x "
                                        f"{sm_max:.0f} MHz",
                         "ms_per_launch": round(t_an, 4), "timing": how}}


def run_singlepass(args, world, dA, w, plan, algorithm=6):
    """Algorithm 6 (single-pass RSVD: A read by the two sketches only, 2
    passes instead of 2q + 2) or Algorithm 3 (q power steps without
    re-orthonormalisation, 2q + 2 passes) on the plain workload's matrix."""
    import torch

    from paper_2402_17794_gb300 import rsvd as R

    m, n, k, p, q, seed = w["m"], w["n"], w["k"], w["p"], w["q"], w["seed"]
    U = torch.empty(k, m, dtype=torch.float64, device="cuda")
    S = torch.empty(k, dtype=torch.float64, device="cuda")
    VT = torch.empty(n, k, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()

    def step():
        R._check(R.rsvd_solve_algorithm(plan.handle, algorithm, dA, m, n, m, k, p, q, seed, U, m, S,
                                        VT, k), "rsvd_solve_algorithm")

    for _ in range(args.warmup):
        step()
    steps = max(args.steps, 5)
    _barrier(world)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    st = plan.status()
    if st != 0:
        raise RuntimeError(f"algorithm {algorithm} solve failed: {R.rsvd_status_string(st)}")
    ms = _max_over_ranks(e0.elapsed_time(e1), world)
    name = {6: "Algorithm 6 (single-pass RSVD)",
            3: "Algorithm 3 (power steps without re-orthonormalisation, shifted CholeskyQR3)"}
    return {"workload": name[algorithm] + " on " + w["desc"].split(";")[0] +
                        (f"; k={k}, p={p}" if algorithm == 6 else f"; k={k}, p={p}, q={q}"),
            "value": round(steps * world / (ms / 1e3), 4), "unit": "solves/s",
            "ms_per_solve": round(ms / steps, 4),
            "passes_per_solve": 2 if algorithm == 6 else 2 * q + 2, "dtype": "f64"}


def run_srft(args, world, dA, w, gaussian_pass_ms):
    """FastRandRF (Halko et al. Algorithm 4.5) with the SRFT test matrix on
    the plain workload's matrix, l = k + p: the sketch through length-64
    FFTs (FP64 ALU-bound) and the complex CholeskyQR2 after it."""
    import torch

    from paper_2402_17794_gb300 import rsvd as R

    m, n, k, p, seed = w["m"], w["n"], w["k"], w["p"], w["seed"]
    l = k + p
    plan = R.Plan(m, n, 2 * l)
    Y = torch.empty(2 * l, m, dtype=torch.float64, device="cuda")
    Q = torch.empty(2 * l, m, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()

    def timed(fn, steps):
        for _ in range(max(args.warmup, 3)):
            fn()
        _barrier(world)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return _max_over_ranks(e0.elapsed_time(e1), world) / steps

    steps = max(args.steps, 10)
    rng_ms = timed(lambda: R._check(R.rsvd_range_srft(plan.handle, dA, m, n, m, l, seed, Q, m),
                                    "rsvd_range_srft"), steps)
    sk_ms = timed(lambda: R._check(R.rsvd_srft_sketch(plan.handle, dA, m, n, m, l, seed, Y, m),
                                   "rsvd_srft_sketch"), steps)
    st = plan.status()
    if st != 0:
        raise RuntimeError(f"SRFT range finder failed: {R.rsvd_status_string(st)}")
    # the whole SRFT solve: the range above, then Stage B on the complex
    # basis (B = Q^H A, its SVD through the realified 2l x 2l Jacobi, the lift)
    U = torch.empty(2 * k, m, dtype=torch.float64, device="cuda")
    S = torch.empty(k, dtype=torch.float64, device="cuda")
    VT = torch.empty(2 * n, k, dtype=torch.float64, device="cuda")
    solve_ms = timed(lambda: R._check(R.rsvd_solve_srft(plan.handle, dA, m, n, m, k, p, seed, U, m,
                                                        S, VT, k), "rsvd_solve_srft"),
                     max(3, steps // 2))
    st = plan.status()
    if st != 0:
        raise RuntimeError(f"SRFT solve failed: {R.rsvd_status_string(st)}")
    del plan, U, S, VT
    # arithmetic of the FFT form per element of A: the phase (2), the 8 x 8
    # length-64 DFT (16 eight-point DFTs of 56 flops + 64 twiddles of 6,
    # per 64 elements: 20) and one complex multiply-add per sample per 64
    # columns (8 l / 64)
    flops = m * n * (2 + 20 + 8 * l / 64)
    peaks, _ = _peaks()
    fp64_peak = 152 * 2 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    return {"workload": "FastRandRF (Halko et al. Alg. 4.5) with the SRFT Omega = sqrt(n/l) D F R "
                        "on " + w["desc"].split(";")[0] + f"; l={l}",
            "value": round(steps * world / (rng_ms * steps / 1e3), 4), "unit": "ranges/s",
            "ms_per_range": round(rng_ms, 4), "ms_sketch": round(sk_ms, 4),
            "solve": {"ms_per_solve": round(solve_ms, 4),
                      "value": round(world * 1e3 / solve_ms, 4), "unit": "solves/s",
                      "what": "rsvd_solve_srft: the range, then B = Q^H A, the SVD of the "
                              "realified 2l x 2l factor and the lift (rank k)"},
            "ms_gaussian_sketch_same_l": round(gaussian_pass_ms, 4),
            "sketch_roofline": {"bound": "alu", "achieved": round(flops / (sk_ms / 1e3) / 1e12, 4),
                                "peak": round(fp64_peak, 4), "unit": "TFLOP/s (FP64)",
                                "frac": round(flops / (sk_ms / 1e3) / 1e12 / fp64_peak, 4)},
            "dtype": "f64 (complex sample, planar)"}


ADAPTIVE = dict(eps=0.25, r=10, l_cap=128)


def run_adaptive(args, world, dA, w):
    """The adaptive range finder + SVD (Halko et al. Algorithm 4.2, the
    toolbox's Adaptive_randRF) on the plain workload's matrix: the tolerance
    eps (absolute; sigma_1 = 1) fixes the rank.  The host waits once per
    block of up to 64 samples to read the stopping test."""
    import torch

    from paper_2402_17794_gb300 import rsvd as R

    m, n, seed = w["m"], w["n"], w["seed"]
    eps, r, cap = ADAPTIVE["eps"], ADAPTIVE["r"], ADAPTIVE["l_cap"]
    plan = R.Plan(m, n, cap)
    U = torch.empty(cap, m, dtype=torch.float64, device="cuda")
    S = torch.empty(cap, dtype=torch.float64, device="cuda")
    VT = torch.empty(n, cap, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    rank = [0]

    def step():
        code, rank[0] = R.rsvd_solve_adaptive(plan.handle, dA, m, n, m, eps, r, cap, seed, U, m,
                                              S, VT, cap)
        if code not in (0, R.ERR_NOT_REACHED):
            R._check(code, "rsvd_solve_adaptive")
        return code

    for _ in range(args.warmup):
        step()
    steps = max(args.steps, 5)
    _barrier(world)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        code = step()
    e1.record(stream)
    torch.cuda.synchronize()
    st = plan.status()
    if st != 0:
        raise RuntimeError(f"adaptive solve failed: {R.rsvd_status_string(st)}")
    ms = _max_over_ranks(e0.elapsed_time(e1), world)
    del plan
    return {"workload": "adaptive range finder + SVD (Halko et al. Alg. 4.2) on " +
                        w["desc"].split(";")[0] + f"; eps={eps}, r={r}, l_cap={cap}",
            "value": round(steps * world / (ms / 1e3), 4), "unit": "solves/s",
            "ms_per_solve": round(ms / steps, 4), "rank": rank[0],
            "tolerance_met": code == 0, "dtype": "f64"}


def _traffic_from_profile(key="plain-fp64", pas="atx"):
    """DRAM bytes per launch of the dominant kernel (`pas` = "ax" or "atx")
    from the committed ncu summary, or None when the kernel's source has
    changed since those counters were taken."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            ent = json.load(f)[key]
        h = hashlib.sha256()
        for name in ent["source_files"]:
            with open(os.path.join(ROOT, "paper_2402_17794_gb300", "csrc", name), "rb") as f:
                h.update(f.read())
        if h.hexdigest() != ent["source_sha256"]:
            return None
        return ent[pas]["dram_bytes_per_launch"]
    except (OSError, ValueError, KeyError):
        return None


def run_reference(args):
    """The CPU oracle timed as it stands on this host's cores, same workload."""
    world, rank, local = _dist()
    if rank != 0:
        return
    import numpy as np
    import torch

    w = WORKLOADS[args.workload]
    m, n, k, p, q = w["m"], w["n"], w["k"], w["p"], w["q"]
    if torch.cuda.is_available():
        A = _make_input(w, 0).cpu().numpy().T
    else:
        from paper_2402_17794_gb300 import synthetic as syn
        A = syn.lowrank_matrix(m, n, _sigma(w), seed=w["seed_a"])
    A = np.asfortranarray(A)
    import oracle
    for i in range(args.warmup):
        oracle.rsvd(A, k, p, q, w["seed"] + i)
    t0 = time.perf_counter()
    for i in range(args.steps):
        oracle.rsvd(A, k, p, q, w["seed"] + i)
    el = time.perf_counter() - t0
    value = args.steps / el
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": "solves/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(el / args.steps * 1e3, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w["desc"], "m": m, "n": n, "k": k, "p": p, "q": q,
                   "a_dtype": w["dtype"]},
        "cpu_baseline": {"value": round(value, 4), "unit": "solves/s", "cores": _cores(),
                         "kind": "oracle",
                         "sample": f"{args.steps} full oracle solves of the workload"},
        "e2e": {"value": round(value, 4), "unit": "solves/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_profile_batched(args):
    """A reduced batched case for ncu captures (no timing): 96 problems of the
    batched distribution (about 0.6 GB of FP32 A, larger than L2), two
    grouped FP32 solves on the tensor engine."""
    import torch

    import __graft_entry__
    from paper_2402_17794_gb300 import rsvd as R

    __graft_entry__.build()
    items = _batched_problems(96, 11)
    plan = R.BatchPlan(len(items), sum(it[1] for it in items), sum(it[2] for it in items),
                       max(it[3] + it[4] for it in items), R.F32)
    for _ in range(2):
        plan.solve(items)
    torch.cuda.synchronize()
    if any(c != 0 for c in plan.status()):
        raise RuntimeError("batched: a problem failed")
    print("profile batched done")


def run_profile_case(args):
    """A reduced case of the same kernels for ncu captures (no timing):
    A 8192 x 4096 FP64 (268 MB, larger than L2), l = 80: two passes of each
    kind and one full solve on the CUDA cores, the same on the tensor cores
    (A prepared once), and two SRFT sketches; A 16384 x 16384 BF16 and
    FP8, l = 160: two passes of each kind and one mixed solve, and for FP8
    two block-scaled passes of each kind with a two-slice E4M3 operand."""
    import numpy as np
    import torch

    import __graft_entry__
    from paper_2402_17794_gb300 import rsvd as R
    from paper_2402_17794_gb300 import synthetic as syn

    __graft_entry__.build()
    m, n, k, p, q = 8192, 4096, 64, 16, 2
    l = k + p
    rng = np.random.default_rng(0)
    dA = torch.from_numpy(rng.standard_normal((n, m))).cuda()
    plan = R.Plan(m, n, l)
    Om = R.colmajor(n, l)
    Y = R.colmajor(m, l)
    Z = R.colmajor(n, l)
    R.rsvd_gaussian(plan.handle, n, l, 1, 0, R.F64, Om, n)
    for _ in range(2):
        R.rsvd_apply_a(plan.handle, dA, m, n, m, Om, n, l, Y, m)
        R.rsvd_apply_at(plan.handle, dA, m, n, m, Y, m, l, Z, n)
    plan.solve(dA, m, n, k, p, q, 3)
    st = plan.status()
    if st != 0:
        raise RuntimeError(R.rsvd_status_string(st))
    # FP64 passes on the tensor cores: A prepared once (six BF16 digit slices,
    # 403 MB), then two passes of each kind and one full solve
    tplan = R.Plan(m, n, l, mode=R.F64_TENSOR)
    R._check(R.rsvd_plan_prepare_a(tplan.handle, dA, m, n, m), "rsvd_plan_prepare_a")
    for _ in range(2):
        R.rsvd_apply_a(tplan.handle, dA, m, n, m, Om, n, l, Y, m)
        R.rsvd_apply_at(tplan.handle, dA, m, n, m, Y, m, l, Z, n)
    R.rsvd_plan_release_a(tplan.handle)
    tplan.solve(dA, m, n, k, p, q, 3)
    st = tplan.status()
    if st != 0:
        raise RuntimeError(R.rsvd_status_string(st))
    del tplan
    # the SRFT sketch through the FFT (n = 4096, a multiple of 64), l = 80
    splan = R.Plan(m, n, 2 * l)
    for _ in range(2):
        splan.srft_sketch(dA, m, n, l, 5)
    st = splan.status()
    if st != 0:
        raise RuntimeError(R.rsvd_status_string(st))
    del dA, plan, splan
    # tcgen05 passes: A 16384 x 16384 BF16 (512 MB), l = 160
    m = n = 16384
    l = 160
    dA = torch.randn(n, m, device="cuda").to(torch.bfloat16)
    plan = R.Plan(m, n, l, a_dtype=R.BF16, mode=R.MIXED)
    Xn = torch.randn(l, n, device="cuda").to(torch.bfloat16)
    Y = torch.empty(l, m, dtype=torch.float32, device="cuda")
    for _ in range(2):
        R.rsvd_apply_a(plan.handle, dA, m, n, m, Xn, n, l, Y, m)
        R.rsvd_apply_at(plan.handle, dA, m, n, m, Xn, m, l, Y, n)
    # one mixed solve (k = 128, p = 32, q = 1): the FP32 l x l kernels at l = 160
    plan.solve(dA, m, n, 128, 32, 1, 3)
    st = plan.status()
    if st != 0:
        raise RuntimeError(R.rsvd_status_string(st))
    # the same passes on FP8 E4M3 storage of A (268 MB), tile scales 2^-4
    codes = dA.view(torch.uint8)[:, :m].contiguous()          # any byte pattern is a valid A
    codes &= 0x77                                             # keep codes normal and finite
    codes |= 0x08
    scales = torch.full(((n + 127) // 128, (m + 127) // 128), 0.0625, device="cuda")
    del dA, plan
    plan = R.Plan(m, n, l, a_dtype=R.FP8E4M3, mode=R.MIXED)
    plan.set_tile_scales(scales)
    for _ in range(2):
        R.rsvd_apply_a(plan.handle, codes, m, n, m, Xn, n, l, Y, m)
        R.rsvd_apply_at(plan.handle, codes, m, n, m, Xn, m, l, Y, n)
    # the block-scaled FP8 passes of the FP8 solve's power steps: an FP32
    # operand split into two E4M3 slices, twice each kind
    Xf = torch.randn(l, n, device="cuda") / n ** 0.5
    for _ in range(2):
        for t in (0, 1):
            R._check(R.rsvd_apply_split(plan.handle, codes, m, n, m, t, Xf, n, l, 1, Y, m),
                     "rsvd_apply_split")
    st = plan.status()
    if st != 0:
        raise RuntimeError(R.rsvd_status_string(st))
    print("profile case done")


def run_launch_case(args):
    """Two full solves of each timed workload, for an ncu launch list (no
    timing): the plain FP64 solve on the tensor cores (16384 x 8192), the
    mixed solve on BF16 and on FP8 storage (65536 x 16384), then two grouped
    FP32 solves of the 512-problem batch."""
    import torch

    import __graft_entry__
    from paper_2402_17794_gb300 import rsvd as R

    __graft_entry__.build()
    for wname in ("plain-fp64", "mixed-bf16", "mixed-fp8"):
        w = WORKLOADS[wname]
        m, n, k, p, q = w["m"], w["n"], w["k"], w["p"], w["q"]
        if w["dtype"] == "fp8":
            dA, scales = _make_input(w, 0)
            plan = R.Plan(m, n, k + p, a_dtype=R.FP8E4M3, mode=R.MIXED)
            plan.set_tile_scales(scales)
        elif w["dtype"] == "bf16":
            dA = _make_input(w, 0)
            plan = R.Plan(m, n, k + p, a_dtype=R.BF16, mode=R.MIXED)
        else:
            dA = _make_input(w, 0)
            plan = R.Plan(m, n, k + p, mode=R.F64_TENSOR)
        for _ in range(2):
            plan.solve(dA, m, n, k, p, q, w["seed"], lda=dA.shape[1])
        torch.cuda.synchronize()
        st = plan.status()
        if st != 0:
            raise RuntimeError(f"{wname}: {R.rsvd_status_string(st)}")
        del dA, plan
        torch.cuda.empty_cache()
    # the batched workload: two grouped FP32 solves of the 512 problems
    items = _batched_problems(512, 11)
    bplan = R.BatchPlan(len(items), sum(it[1] for it in items), sum(it[2] for it in items),
                        max(it[3] + it[4] for it in items), R.F32)
    outs = [(torch.empty(k, m, dtype=torch.float32, device="cuda"),
             torch.empty(k, dtype=torch.float64, device="cuda"),
             torch.empty(n, k, dtype=torch.float32, device="cuda"))
            for (_, m, n, k, _, _, _) in items]
    for _ in range(2):
        bplan.solve(items, outs)
    torch.cuda.synchronize()
    if any(c != 0 for c in bplan.status()):
        raise RuntimeError("batched: a problem failed")
    print("launch case done")


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="plain-fp64")
    ap.add_argument("--cpu-budget", type=float, default=15.0,
                    help="seconds of CPU oracle time for cpu_baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true",
                    help="skip the mixed-precision (BF16) workload")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched workload")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving workload")
    ap.add_argument("--serve-seconds", type=float, default=30.0,
                    help="seconds of Poisson arrivals in the serving run (the workload "
                         "definition uses 30)")
    ap.add_argument("--launch-case", action="store_true",
                    help="two full solves of each timed workload, for an ncu launch list")
    ap.add_argument("--profile-case", action="store_true",
                    help="run a reduced case of the same kernels for ncu (no timing)")
    ap.add_argument("--profile-batched", action="store_true",
                    help="run a reduced batched case (tensor engine) for ncu (no timing)")
    args = ap.parse_args()
    if args.profile_batched:
        run_profile_batched(args)
        return
    if args.launch_case:
        run_launch_case(args)
        return
    if args.profile_case:
        run_profile_case(args)
        return
    if args.warmup < 3 and args.impl == "ours":
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
