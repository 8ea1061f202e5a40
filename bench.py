#!/usr/bin/env python3
"""Throughput of the segment-parallel Riccati solve (LQR stages/s) on GB300.

One step = one full solve (parametric segment sweeps, link solve, policy
sweeps, rollout with multipliers and cost, and in the refined modes the FP64
KKT residual passes and refinement corrections) of one workload, on synthetic
seeded data with inputs resident in HBM. The default workload is the long
horizon n=64, m=32, T=4096, rho(A_t) <= 1.02, solved in LQR_MIXED_FP32 (FP32
solve, FP64 residual, refinement to |r|/|b| <= 1e-10): an answer of FP64
grade, compared with the plain FP64 segment-parallel solve of the same data
on the same GPU at its best segment count. --config 2 runs the n=128, m=64,
T=1024, K=64 mixed-precision workload; --config 0 the n=12, m=4, T=128, K=8
FP64 workload. Under torchrun every rank solves its own replica (the method
does not shard across GPUs); value = all ranks' stages / max-over-ranks time.

--impl reference times the FP64 serial Riccati oracle on the host cores on a
bounded sample of the same workload (there is no reference implementation).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads  # noqa: E402

METRIC = "LQR stages/sec at stated KKT residual vs plain FP64 segment-parallel solve"
UNIT = "stages/s"

# peaks: HBM and bf16 tensor are measured (MEASURED_PEAKS.json); the DFMA and
# FFMA pipes are derived from unit counts and the maximum SM clock: 152 SMs x
# 2 DFMA/clk (1.25 TFLOP/s FP64 nominal) and x 128 FFMA/clk, at 2070 MHz.
SMS, SM_MHZ = 152, 2070.0
PEAK_FP64_TFLOPS = SMS * 2 * 2 * SM_MHZ * 1e6 / 1e12      # 1.259
PEAK_FP32_TFLOPS = SMS * 128 * 2 * SM_MHZ * 1e6 / 1e12    # 80.5
# dense TF32 tensor peak: the measured bf16 cuBLAS peak x the nominal TF32:BF16
# ratio 1.1 : 2.25 PFLOP/s (dense)


def _tf32_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)["bf16_tflops"] * 1.1 / 2.25
    except (OSError, ValueError, KeyError):
        return 1900.0 * 1.1 / 2.25


PEAK_TF32_TFLOPS = _tf32_peak()

# DRAM bytes per launch (read + write) measured by ncu for the kernel as it now
# stands, keyed by (kernel, workload config, precision); an entry is removed
# whenever its kernel changes. seg_sweep_f32_kernel on the long-horizon
# workload in LQR_MIXED_FP32: A1 227.6 MB, A4 309.4 MB (it also writes K_t, P_t,
# M_uu^-1), mean of the two launches (profiles/seg_sweep_f32_n64_m32_T4096_K152.md)
NCU_TRAFFIC: dict = {("seg_sweep_f32_kernel", 1, "mixed_fp32"): (227.6e6 + 309.4e6) / 2}


def link_flops(n: int, K: int) -> float:
    """Algorithmic FP64 flops of the block-elimination link solve (dual form): per
    link two n x n factorisations (n^3/3 each), W C, C'Z, C'(W C), L^-1 E, F'F,
    L^-T F (n^3 each, triangular or symmetric halves) and (W C) G (2n^3)."""
    return (K - 1) * (2 * n ** 3 / 3 + 6 * n ** 3 + 2 * n ** 3)


def link_scan_flops(n: int, K: int) -> float:
    """Algorithmic FP32 flops of the scan link solve as implemented: every
    composition has one Cholesky factor (n^3/3) and one Gauss-Jordan inverse
    (2n^3) of n x n matrices plus 2n^3 per n x n product: 11 products for a
    full composition, 5 when the later element already holds the global value
    function (P, p only), 6 for the feedback pass; levels s = 1, 2, 4, .. < K
    have max(0, K - 2s) full and min(K - s, s) final compositions."""
    fac = n ** 3 / 3 + 2 * n ** 3
    full, final, post = fac + 22 * n ** 3, fac + 10 * n ** 3, fac + 12 * n ** 3
    tot, s = 0.0, 1
    while s < K:
        tot += max(0, K - 2 * s) * full + min(K - s, s) * final
        s *= 2
    return tot + (K - 1) * post


def rollout_bytes(n: int, m: int, T: int, es: int) -> float:
    """Algorithmic bytes of one rollout launch: per stage it reads K, k, A, B, c,
    Q, R, S, q, r (twice A, Q, S for the multipliers) and writes x, u, lambda."""
    per = (m * n + m + 2 * n * n + n * m + n + 2 * n * n + m * m + 2 * m * n + n + m) + (n + m + n)
    return T * per * es


def sweep_flops(n: int, m: int, T: int, K: int, phase: str) -> float:
    """Algorithmic FLOPs of one launch of a segment-sweep kernel, counted for the
    FP32 kernel's evaluation order (2 flops per multiply-add).

    Per stage of a parametric segment: V[A|B|c], B'(V[A|B|c]) (M_ux, M_uu, m_u),
    A'V A, Z B, Z A, the Gauss-Jordan inverse of M_uu (2m^3), H = M_uu^-1 [M_ux |
    M_zu' | m_u] and the V_xx, Z, -W downdates:
        6n^3 + 12n^2 m + 6n m^2 + 2m^3
    Per stage of a plain Riccati sweep (terminal segment, policy sweep):
        4n^3 + 6n^2 m + 4n m^2 + 2m^3
    """
    par = 6 * n ** 3 + 12 * n ** 2 * m + 6 * n * m ** 2 + 2 * m ** 3
    pla = 4 * n ** 3 + 6 * n ** 2 * m + 4 * n * m ** 2 + 2 * m ** 3
    last = T - (K - 1) * T // K
    if phase == "sweep":
        return (T - last) * par + last * pla
    return (T - last) * pla  # policy sweep: segments 0..K-2


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=5)
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _prefix(prob, T_sample):
    return {k: np.ascontiguousarray(v[:T_sample] if k in ("A", "B", "c", "R", "S", "r") else
                                    (v[:T_sample + 1] if k in ("Q", "q") else v)) for k, v in prob.items()}


def cpu_baseline(wl, prob_full, budget_s=12.0):
    """The FP64 serial Riccati oracle on one host core: whole solves of the
    workload when one takes at most a few seconds (their last result also
    serves as the reference for the per-quantity errors of the GPU answer),
    else runs over a prefix of the workload, repeated for about budget_s s."""
    import oracle
    n, m, T = wl["n"], wl["m"], wl["T"]
    T_sample = wl["cpu_stages"]
    sample = prob_full if T_sample >= T else _prefix(prob_full, T_sample)
    oracle.riccati(_prefix(prob_full, 2), want_P=False)  # build/load outside the timing
    runs, t0, ref = 0, time.perf_counter(), None
    while True:
        ref = oracle.riccati(sample, want_P=True)
        runs += 1
        el = time.perf_counter() - t0
        if el >= budget_s:
            break
    what = ("the whole %d-stage workload" % T) if T_sample >= T else ("the first %d stages of the workload" % T_sample)
    out = {"value": runs * min(T_sample, T) / el, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": "%d runs of the FP64 serial Riccati oracle (single thread, C) on %s (n=%d m=%d), %.1f s" %
                     (runs, what, n, m, el)}
    return out, (ref if T_sample >= T else None)


def max_over_ranks(values, world, device):
    """Elementwise maximum of per-rank floats over the process group (the
    slowest replica sets the job's time); the values themselves at world 1."""
    if world == 1:
        return [float(v) for v in values]
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def whole_job_rate(stages_per_replica_step: int, steps: int, world: int, seconds: float) -> float:
    """Stages per second over all replicas: every rank solves its own copy of the
    workload (weak scaling, no data-path collective), timed by the slowest."""
    return world * steps * stages_per_replica_step / seconds


def run_reference(args, rank, world):
    """Reference arm: the oracle on host cores (rank 0 only), per step one
    bounded sample of the workload."""
    if rank != 0:
        return
    wl = WORKLOADS[args.config]
    if wl.get("batch"):
        import oracle
        probs = wl["make"]()[:wl["ref_problems"]]
        oracle.riccati(_prefix(probs[0], 2), want_P=False)
        stages = sum(p["B"].shape[0] for p in probs)
        for _ in range(args.warmup):
            oracle.riccati(probs[0], want_P=False)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            for p in probs:
                oracle.riccati(p, want_P=False)
        el = time.perf_counter() - t0
        value = args.steps * stages / el
        print(json.dumps({"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
                          "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
                          "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                          "data": "synthetic (seeded PCG64)",
                          "config": {"workload": "%s (per step: the first %d problems, serial FP64 Riccati oracle "
                                                 "on the host, forward solves)" % (wl["name"], len(probs))},
                          "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                                           "sample": "%d steps x %d problems (%d stages), one thread" %
                                                     (args.steps, len(probs), stages)},
                          "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}),
              flush=True)
        return
    n, m, T = wl["n"], wl["m"], wl["T"]
    prob = wl["make"]()
    T_sample = min(wl["ref_stages"], T)
    import oracle
    oracle.riccati(_prefix(prob, 2), want_P=False)
    sample = prob if T_sample >= T else _prefix(prob, T_sample)
    for _ in range(args.warmup):
        oracle.riccati(sample, want_P=False)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.riccati(sample, want_P=False)
    el = time.perf_counter() - t0
    value = args.steps * T_sample / el
    what = "the whole workload" if T_sample >= T else "a %d-stage prefix" % T_sample
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded PCG64)",
            "config": {"workload": "%s (per step: %s, serial FP64 Riccati oracle on the host)" % (wl["name"], what),
                       "n": n, "m": m, "T": T},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": "%d steps x %d stages of the serial FP64 oracle, one thread" %
                                       (args.steps, T_sample)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# The workloads a bench line can be quoted on (seeded synthetic data).
WORKLOADS = {
    1: dict(name="long-horizon LQR n=64 m=32 T=4096 rho(A)<=1.02", n=64, m=32, T=4096, K=0, prec="mixed_fp32",
            make=lambda: workloads.config1(4096), Kgrid=(16, 64, 256, 1024), fp64_K=(64, 128, 152, 256),
            cpu_stages=4096, ref_stages=256, unrefined="fp32"),
    2: dict(name="mixed-precision LQR n=128 m=64 T=1024 rho(A)<=1.02", n=128, m=64, T=1024, K=64, prec="mixed",
            make=lambda: workloads.config2(1024), Kgrid=(), fp64_K=(16, 32, 64), cpu_stages=1024, ref_stages=128,
            unrefined="fp32"),
    0: dict(name="single LQR n=12 m=4 T=128", n=12, m=4, T=128, K=8, prec="fp64", make=workloads.config0,
            Kgrid=(1, 8, 16), fp64_K=(8,), cpu_stages=128, ref_stages=128, unrefined=None),
    3: dict(name="uneven batch of 4096 LQR problems, T~U{32..512}, n in {8,16,32,48}, m~U{2..16}", batch=True,
            make=workloads.config3, K=0, backward=False, ref_problems=64),
    4: dict(name="differentiable batch of 256 LQR problems n=32 m=8 T=256, forward + adjoint, loss sum |x|^2+|u|^2",
            batch=True, make=workloads.config4, K=16, backward=True, ref_problems=16),
}


def stage_policy_flops(n: int, m: int) -> float:
    """Algorithmic FLOPs of one stage of the per-stage global-policy
    reconstruction: the factor of Vzz + P_e (n^3/3), the two triangular solves
    with n + 1 right-hand sides (2 n^2 (n + 1)), X'X (2n^3) and Kz Y (2 m n^2)."""
    return n ** 3 / 3.0 + 2.0 * n * n * (n + 1) + 2.0 * n ** 3 + 2.0 * m * n * n


def ls_mult_flops(n: int, m: int, T: int, K: int) -> float:
    """Algorithmic FLOPs of the least-squares multipliers (block Cholesky of
    the normal equations): per dynamics block A A' (2n^3), B B' (2n^2 m), the
    coupling solve (n^3), its downdate (2n^3) and the n x n factor (n^3/3);
    per interior segment the mu block (n^3 + 2n^3 + n^3/3); per segment its
    first block (n^3/3). Vector work is O(n^2) and left out."""
    return (T * (16.0 / 3.0 * n ** 3 + 2.0 * n * n * m) + (K - 1) * (10.0 / 3.0) * n ** 3
            + K * n ** 3 / 3.0)


def riccati_stage_flops(n: int, m: int) -> float:
    """Algorithmic FLOPs of one plain Riccati stage as the FP32 sweep evaluates it
    (V[A|B|c], [A|B]'V[A|B], the M_uu inverse, H and the downdate)."""
    return 4 * n ** 3 + 6 * n ** 2 * m + 4 * n * m ** 2 + 2 * m ** 3


def run_batch_bench(args, wl, rank, world, local):
    """A batch workload: one step = one batched solve (the uneven batch) or one
    batched forward solve plus one batched adjoint solve (the differentiable
    batch), all problems, FP32."""
    import torch
    import torch.distributed as dist
    from paper_1809_06360_gb300 import lqr

    device = f"cuda:{local}"
    probs_np = wl["make"]()
    stages = sum(p["B"].shape[0] for p in probs_np)
    dev = [{k: torch.from_numpy(v).to(device, torch.float32) for k, v in p.items()} for p in probs_np]
    solver = lqr.Solver(local)
    outs = [solver.alloc_solution(p, ("K", "k", "x", "u", "lam")) for p in dev]
    stream = torch.cuda.current_stream()
    K = args.segments or wl["K"]
    back = wl["backward"]
    gx = [torch.zeros_like(o["x"]) for o in outs] if back else None
    gu = [torch.zeros_like(o["u"]) for o in outs] if back else None

    def step():
        solver.solve_batched(dev, prec="fp32", num_segments=K, outs=outs)
        if back:
            for o, a, b in zip(outs, gx, gu):  # dL/dx, dL/du of the loss sum |x|^2 + |u|^2
                torch.mul(o["x"], 2.0, out=a)
                torch.mul(o["u"], 2.0, out=b)
            solver.backward_batched(dev, outs, gx, gu, prec="fp32", num_segments=K)

    for _ in range(args.warmup):
        step()
    st, _ = solver.report_batched(len(dev))
    if any(x != 0 for x in st):
        raise SystemExit("batched solve failed: %s" % sorted(set(st)))
    solver.solve_batched(dev, prec="fp32", num_segments=K, outs=outs)
    fwd_launches = lqr.lqr_last_launch_count(solver.h)
    step_launches = fwd_launches
    if back:  # the adjoint's batched solve with its right-hand-side and gradient kernels
        solver.backward_batched(dev, outs, gx, gu, prec="fp32", num_segments=K)
        step_launches += lqr.lqr_last_launch_count(solver.h)
    clocks = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    ms = _timed(stream, step, args.steps) * args.steps
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    ms = max_over_ranks([ms], world, device)[0]
    value = whole_job_rate(stages, args.steps, world, ms / 1e3)
    # roofline: the algorithmic FLOPs of the Riccati stages (the adjoint solve
    # runs the same sweeps once more) over the device time of the step
    flops = sum(p["B"].shape[0] * riccati_stage_flops(p["B"].shape[1], p["B"].shape[2]) for p in probs_np)
    if back:
        flops *= 2
    ach = flops / (ms / args.steps / 1e3) / 1e12
    sched = "one persistent launch" if fwd_launches == 1 else "per-step launches (%d)" % fwd_launches
    roofline = {"bound": "alu", "achieved": ach, "peak": PEAK_FP32_TFLOPS, "unit": "TFLOP/s",
                "frac": ach / PEAK_FP32_TFLOPS, "traffic": None,
                "kernel": ("batch_persistent_kernel (A10: sweep, rollout and objective per problem)" if fwd_launches == 1
                           else "seg_sweep_f32_kernel, link, rollout (per-step launches)") +
                          (", then the batched adjoint solve" if back else ""),
                "peak_source": "derived: 152 SMs x 128 FFMA/clk x 2070 MHz", "work_flops_per_step": flops}
    e2e = None
    if not args.no_e2e:
        # inputs copied in from pinned host memory and x, u read back, every step
        pin = [{k: torch.from_numpy(v.astype(np.float32)).pin_memory() for k, v in p.items()} for p in probs_np]
        hx = [torch.empty(o["x"].shape, dtype=torch.float32).pin_memory() for o in outs]
        hu = [torch.empty(o["u"].shape, dtype=torch.float32).pin_memory() for o in outs]

        def e2e_step():
            for d, hp in zip(dev, pin):
                for k in d:
                    d[k].copy_(hp[k], non_blocking=True)
            step()
            for o, a, b in zip(outs, hx, hu):
                a.copy_(o["x"], non_blocking=True)
                b.copy_(o["u"], non_blocking=True)
            torch.cuda.synchronize()

        e2e_step()
        n_e2e = max(2, args.steps // 2)
        t0 = time.perf_counter()
        for _ in range(n_e2e):
            e2e_step()
        el = max_over_ranks([time.perf_counter() - t0], world, device)[0]
        e2e = {"value": whole_job_rate(stages, n_e2e, world, el), "unit": UNIT,
               "h2d_bytes_per_step": int(sum(v.nbytes for hp in pin for v in hp.values())),
               "d2h_bytes_per_step": int(sum(a.numel() * 4 + b.numel() * 4 for a, b in zip(hx, hu))),
               "steps": n_e2e}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        import oracle
        oracle.riccati(_prefix(probs_np[0], 2), want_P=False)
        t0, done, st_done = time.perf_counter(), 0, 0
        while time.perf_counter() - t0 < 12.0 and done < len(probs_np):
            oracle.riccati(probs_np[done], want_P=False)
            st_done += probs_np[done]["B"].shape[0]
            done += 1
        el = time.perf_counter() - t0
        cpu = {"value": st_done / el, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": "the FP64 serial Riccati oracle (single thread, C) on the first %d problems of the batch "
                         "(%d stages, forward solves only), %.1f s" % (done, st_done, el)}
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
                "data": "synthetic (seeded PCG64), inputs resident in HBM",
                "config": {"workload": wl["name"], "problems": len(probs_np), "stages": stages,
                           "K": K if K else "chosen by the batch schedule", "schedule": sched,
                           "precision": "FP32 data and sweeps",
                           "l2": "inputs (%.2f GB FP32) larger than L2 (129 MB)" % (
                               sum(v.nbytes for p in probs_np for v in p.values()) / 2e9),
                           "parallelism": "replicas" if world > 1 else "single GPU"},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk,
                "gpu_launches": step_launches * args.steps}
        print(json.dumps(line), flush=True)
    solver.close()
    if world > 1:
        dist.destroy_process_group()

def _timed(stream, fn, reps):
    """Mean device time (ms) of fn() over reps calls, CUDA events on stream."""
    import torch
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", type=int, default=1, choices=sorted(WORKLOADS))
    ap.add_argument("--prec", default=None, choices=["fp64", "fp32", "mixed", "mixed_fp32"],
                    help="default: the workload's (mixed_fp32 for the long horizon)")
    ap.add_argument("--tol", type=float, default=1e-10, help="refinement target |r|/|b| (mixed modes)")
    ap.add_argument("--max-refine", type=int, default=8)
    ap.add_argument("--segments", type=int, default=0, help="0 = the workload's K (or the library's choice)")
    ap.add_argument("--form", default="multiplier", choices=["multiplier", "constrained"])
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the FP64 comparison, K grid and unrefined form")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    import torch.distributed as dist
    from paper_1809_06360_gb300 import build, lqr

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    build.build()

    wl = WORKLOADS[args.config]
    if wl.get("batch"):
        run_batch_bench(args, wl, rank, world, local)
        return
    n, m, T = wl["n"], wl["m"], wl["T"]
    K = args.segments or wl["K"]
    prec = args.prec or wl["prec"]
    prob_np = wl["make"]()
    dt = torch.float32 if prec == "fp32" else torch.float64
    npdt = np.float32 if prec == "fp32" else np.float64
    device = f"cuda:{local}"
    dev = {k: torch.from_numpy(v).to(device, dt) for k, v in prob_np.items()}
    solver = lqr.Solver(local)
    out = solver.alloc_solution(dev, want=("K", "k", "x", "u", "lam"))
    stream = torch.cuda.current_stream()

    mr = args.max_refine if prec.startswith("mixed") else 0

    def step():
        solver.solve(dev, num_segments=K, prec=prec, out=out, form=args.form, max_refine=mr, tol=args.tol)

    for _ in range(args.warmup):
        step()
    rep = solver.report()
    if rep["status"] != 0:
        raise SystemExit("solve failed: %s" % rep)
    launches_per_step = lqr.lqr_last_launch_count(solver.h)
    K = rep["num_segments"]

    # KKT residual of the benchmarked solution, by the library's own FP64 residual
    # pass (step A7), once, outside the timing
    solver.solve(dev, num_segments=K, prec=prec, out=out, form=args.form, residual=True, max_refine=mr, tol=args.tol)
    rep_res = solver.report()
    res = {"eta": rep_res["kkt_residual"], "rel": rep_res["kkt_rel"], "iters": rep_res["refine_iters"]}
    answer = {k: v.double().cpu().numpy() for k, v in out.items()}

    clocks = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    lqr.lqr_profile_enable(solver.h, True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    phase_ms, nprof = lqr.lqr_profile_read(solver.h)
    lqr.lqr_profile_enable(solver.h, False)
    ms = max_over_ranks([ms], world, device)[0]
    value = whole_job_rate(T, args.steps, world, ms / 1e3)

    # per-phase achieved rates; the roofline entry is the kernel that takes the most time
    nsolve = max(nprof, 1)
    ph = {k: v / nsolve for k, v in phase_ms.items()}
    fp64_pipe = prec == "fp64"
    alu_peak = PEAK_FP64_TFLOPS if fp64_pipe else PEAK_FP32_TFLOPS
    hbm = measured_peaks().get("hbm_gbs", 6780.4)
    # the FP32 fast path (FP32 sweeps, link scan and rollout) also runs every
    # solve of the mixed FP32 mode, on its FP32 copy of the data
    fast = prec in ("fp32", "mixed_fp32") and args.form == "multiplier" and n <= 64
    es = 4 if prec in ("fp32", "mixed_fp32") else 8
    sweep_k = "seg_sweep_f32_kernel" if fast else "seg_sweep_kernel"
    fp32_link = prec in ("fp32", "mixed_fp32") or (prec == "mixed" and n > 67)
    if fast and K > 1:
        link = {"kernel": "link_scan_kernel levels + feedback pass + link states (A3, FP32 scan)", "bound": "alu",
                "unit": "TFLOP/s", "work": link_scan_flops(n, K), "peak": PEAK_FP32_TFLOPS}
    elif fp32_link and n > 67:
        link = {"kernel": "link_chain_f32_kernel + link_post_kernel<float> + link_forward_kernel (A3, FP32 chain)",
                "bound": "alu", "unit": "TFLOP/s", "work": link_flops(n, K), "peak": PEAK_FP32_TFLOPS}
    else:
        link = {"kernel": ("link_solve_dual_cluster_kernel" if n <= 67 else "link_solve_dual_kernel") +
                          " (A3, FP64 block elimination)", "bound": "alu",
                "unit": "TFLOP/s", "work": link_flops(n, K), "peak": PEAK_FP64_TFLOPS}
    # the mixed TF32 mode runs the policy sweeps on the tensor cores for 64 < n <= 128, m <= 64
    tc_policy = prec == "mixed" and 64 < n <= 128 and m <= 64
    phases = {
        "sweep": {"kernel": sweep_k + " phase 0 (A1)", "bound": "alu", "unit": "TFLOP/s",
                  "work": sweep_flops(n, m, T, K, "sweep"), "peak": alu_peak},
        "policy": ({"kernel": "seg_sweep_tc_kernel (A4, tcgen05 TF32 products, FP64 factor of M_uu)",
                    "bound": "tensor", "unit": "TFLOP/s", "work": sweep_flops(n, m, T, K, "policy"),
                    "peak": PEAK_TF32_TFLOPS} if tc_policy else
                   {"kernel": sweep_k + " phase 1 (A4)", "bound": "alu", "unit": "TFLOP/s",
                    "work": sweep_flops(n, m, T, K, "policy"), "peak": alu_peak}),
        "link": link,
        "rollout": {"kernel": ("rollout_f32_kernel" if fast else "rollout_stream_kernel") + " + finalize (A5/A6)",
                    "bound": "hbm", "unit": "GB/s",
                    "work": rollout_bytes(n, m, T, es), "peak": hbm},
    }
    for k, d in phases.items():
        t = ph.get(k, 0.0)
        scale = 1e12 if d["unit"] == "TFLOP/s" else 1e9
        d["ms"] = t
        d["achieved"] = (d["work"] / (t / 1e3) / scale) if t > 0 else 0.0
        d["frac"] = d["achieved"] / d["peak"]
    # per kernel function: the A1 and A4 sweeps are two launches of one kernel
    kern = {
        sweep_k: ({"kernel": sweep_k + " (A1)", "bound": "alu", "unit": "TFLOP/s",
                   "work": phases["sweep"]["work"], "ms": phases["sweep"]["ms"], "peak": alu_peak, "launches": 1}
                  if tc_policy else
                  {"kernel": sweep_k + " (A1 + A4, two launches per solve)", "bound": "alu", "unit": "TFLOP/s",
                   "work": phases["sweep"]["work"] + phases["policy"]["work"],
                   "ms": phases["sweep"]["ms"] + phases["policy"]["ms"], "peak": alu_peak, "launches": 2}),
        "link": dict(phases["link"], launches=None),
        "rollout": dict(phases["rollout"], launches=2),
    }
    if tc_policy:
        kern["seg_sweep_tc_kernel"] = dict(phases["policy"], launches=1)
    for d in kern.values():
        d["achieved"] = (d["work"] / (d["ms"] / 1e3) / 1e12) if d["ms"] > 0 and d["unit"] == "TFLOP/s" else d["achieved"]
        d["frac"] = d["achieved"] / d["peak"]
    dom = max(kern, key=lambda k: kern[k]["ms"])
    dd = kern[dom]
    # DRAM traffic per launch of the dominant kernel from an ncu capture of this
    # workload (dram__bytes_read.sum + dram__bytes_write.sum), None when not taken
    # for the kernel as it now stands
    traffic = NCU_TRAFFIC.get((dd["kernel"].split(" ")[0], args.config, prec))
    roofline = {"bound": dd["bound"], "achieved": dd["achieved"], "peak": dd["peak"], "unit": dd["unit"],
                "frac": dd["frac"], "traffic": traffic, "kernel": dd["kernel"],
                "peak_source": ("derived: 152 SMs x 2 DFMA/clk x 2070 MHz" if dd["peak"] == PEAK_FP64_TFLOPS else
                                "derived: 152 SMs x 128 FFMA/clk x 2070 MHz" if dd["peak"] == PEAK_FP32_TFLOPS else
                                "measured bf16 x 1.1/2.25 (nominal TF32:BF16)" if dd["peak"] == PEAK_TF32_TFLOPS else
                                "measured (MEASURED_PEAKS.json hbm_gbs)"),
                "phases": {k: {kk: (round(vv, 6) if isinstance(vv, float) else vv) for kk, vv in d.items()}
                           for k, d in phases.items()},
                "phase_ms_per_step": ph}

    extras = {}
    gpp_answer = None
    if not args.no_extras:
        # the plain FP64 segment-parallel solve of the same workload on the same GPU,
        # at its best segment count
        dev64 = dev if dt == torch.float64 else {k: torch.from_numpy(v).to(device, torch.float64)
                                                 for k, v in prob_np.items()}
        out64 = solver.alloc_solution(dev64, want=("K", "k", "x", "u", "lam"))
        sweep64 = {}
        for Kf in wl["fp64_K"]:
            f = lambda: solver.solve(dev64, num_segments=Kf, prec="fp64", out=out64)
            f()
            sweep64[Kf] = _timed(stream, f, 2)
        Kbest = min(sweep64, key=sweep64.get)
        f = lambda: solver.solve(dev64, num_segments=Kbest, prec="fp64", out=out64)
        nref = 10
        ms64 = _timed(stream, f, nref)
        solver.solve(dev64, num_segments=Kbest, prec="fp64", out=out64, residual=True)
        rep64 = solver.report()
        extras["plain_fp64"] = {"stages_per_s": T / (ms64 / 1e3), "ms_per_solve": ms64, "K": Kbest,
                                "K_swept_ms": {str(k): round(v, 4) for k, v in sweep64.items()},
                                "kkt_backward_error": rep64["kkt_residual"], "kkt_rel_residual": rep64["kkt_rel"],
                                "steps": nref}
        extras["speedup_vs_plain_fp64"] = value / world / extras["plain_fp64"]["stages_per_s"]
        del out64
        # the same mode over the segment-count grid of the workload
        grid = {}
        for Kg in wl["Kgrid"]:
            if Kg > T // max(1, -(-n // m)):
                continue
            f = lambda: solver.solve(dev, num_segments=Kg, prec=prec, out=out, form=args.form, max_refine=mr,
                                     tol=args.tol)
            f()
            t = _timed(stream, f, 5)
            solver.solve(dev, num_segments=Kg, prec=prec, out=out, form=args.form, residual=True, max_refine=mr,
                         tol=args.tol)
            r = solver.report()
            grid[str(Kg)] = {"stages_per_s": T / (t / 1e3), "ms_per_solve": t, "kkt_rel_residual": r["kkt_rel"],
                             "refinement_corrections": r["refine_iters"] if mr else 0}
        if grid:
            extras["K_grid"] = grid
        # the unrefined FP32 answer of the same workload (what the refined mode starts from)
        if wl["unrefined"] and prec != wl["unrefined"]:
            d32 = {k: v.float() for k, v in dev64.items()}
            o32 = solver.alloc_solution(d32, want=("K", "k", "x", "u", "lam"))
            f = lambda: solver.solve(d32, num_segments=K, prec="fp32", out=o32, form=args.form)
            f()
            t = _timed(stream, f, 10)
            solver.solve(d32, num_segments=K, prec="fp32", out=o32, form=args.form, residual=True)
            r = solver.report()
            extras["fp32_unrefined"] = {"stages_per_s": T / (t / 1e3), "ms_per_solve": t, "K": K,
                                        "kkt_backward_error": r["kkt_residual"], "kkt_rel_residual": r["kkt_rel"]}
            del d32, o32
        # the multipliers from Section II-B's least-squares system at the FP64
        # optimum (lqr_ls_multipliers: block Cholesky of the normal equations, FP64)
        o64 = solver.alloc_solution(dev64, want=("K", "k", "x", "u", "lam"))
        solver.solve(dev64, num_segments=K, prec="fp64", out=o64)
        f = lambda: solver.ls_multipliers(dev64, o64["x"], o64["u"], K)
        lsm = f()
        torch.cuda.synchronize()
        t = _timed(stream, f, 3)
        work = ls_mult_flops(n, m, T, K)
        ach = work / (t * 1e-3) / 1e12
        extras["ls_multipliers"] = {
            "kernel": "ls_mult_kernel (Section II-B least-squares multipliers, FP64 block Cholesky, one CTA per segment)",
            "ms": t, "K": K, "bound": "alu", "unit": "TFLOP/s", "work": work, "achieved": ach,
            "peak": PEAK_FP64_TFLOPS, "frac": ach / PEAK_FP64_TFLOPS,
            "peak_source": "derived: 152 SMs x 2 DFMA/clk x 2070 MHz",
            "rel_diff_vs_solve_lambda": float((lsm["lam"] - o64["lam"]).abs().max() / o64["lam"].abs().max())}
        del o64, lsm
        # the per-stage reconstruction of the global policy (constrained form, FP64)
        # beside the sequential policy sweep of the FP64 constrained solve
        f = lambda: solver.global_policy_parallel(dev64, K)
        gpp = f()
        torch.cuda.synchronize()
        reps = 3
        lqr.lqr_profile_enable(solver.h, True)
        for _ in range(reps):
            f()
        ph, nprof = lqr.lqr_profile_read(solver.h)
        lqr.lqr_profile_enable(solver.h, False)
        oc = solver.alloc_solution(dev64, want=("K", "k", "x", "u"))
        solver.solve(dev64, num_segments=K, prec="fp64", form="constrained", out=oc)
        lqr.lqr_profile_enable(solver.h, True)
        for _ in range(reps):
            solver.solve(dev64, num_segments=K, prec="fp64", form="constrained", out=oc)
        ph2, nprof2 = lqr.lqr_profile_read(solver.h)
        lqr.lqr_profile_enable(solver.h, False)
        del oc
        reach = -(-n // m)
        nst = sum(max(0, (j + 1) * T // K - j * T // K - (reach - 1)) for j in range(K - 1))
        work = stage_policy_flops(n, m) * nst
        ms_stage = ph["rollout"] / nprof
        ach = work / (ms_stage * 1e-3) / 1e12
        extras["global_policy_parallel"] = {
            "kernel": "stage_policy_kernel (per-stage global P_t, K_t from the constrained segment values, FP64, "
                      "one CTA per stage)",
            "ms_total": sum(ph.values()) / nprof, "K": K,
            "phase_ms": {"A1 constrained sweep": ph["sweep"] / nprof, "link": ph["link"] / nprof,
                         "policy sweep of the segment ends": ph["policy"] / nprof, "per-stage kernel": ms_stage},
            "sequential_policy_sweep_ms": ph2["policy"] / nprof2, "fp64_constrained_solve_ms": sum(ph2.values()) / nprof2,
            "stages_in_parallel": nst, "bound": "alu", "unit": "TFLOP/s", "work": work, "achieved": ach,
            "peak": PEAK_FP64_TFLOPS, "frac": ach / PEAK_FP64_TFLOPS,
            "peak_source": "derived: 152 SMs x 2 DFMA/clk x 2070 MHz"}
        gpp_answer = {k: v.cpu().numpy() for k, v in gpp.items()}
        del gpp
        del dev64
        # the trajectory-optimisation outer loop (Section I) on a nonlinear
        # tracking model of the same size, its LQR subproblems in this mode
        nlm = workloads.make_nl_model(n, m, T, seed=84, beta=0.05)
        dm = {k: (torch.from_numpy(v).to(device, torch.float64) if isinstance(v, np.ndarray) else v)
              for k, v in nlm.items()}

        def sqp_run():
            xs = torch.zeros((T + 1, n), dtype=torch.float64, device=device)
            us = torch.zeros((T, m), dtype=torch.float64, device=device)
            return solver.sqp_solve(dm, xs, us, max_iters=30, tol=1e-8, num_segments=K, prec="mixed_fp32",
                                    max_refine=8, sub_tol=1e-10)
        sqp_run()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        so = sqp_run()
        el = (time.perf_counter() - t0) * 1e3
        extras["sqp_outer_loop"] = {
            "model": "x' = A x + B u + 0.05 tanh(C x), tracking cost, n=%d m=%d T=%d, from x = u = 0" % (n, m, T),
            "subproblem": "MIXED_FP32, K=%d, refined to rel 1e-10" % K,
            "iterations": so["report"]["iters"], "converged": so["report"]["converged"],
            "final_defect_l1": so["report"]["defect"], "final_cost": so["report"]["cost"],
            "ms_total": el, "ms_per_iteration": el / so["report"]["iters"],
            "stages_per_s_per_iteration": T * so["report"]["iters"] / (el / 1e3),
            "step_lengths": [h["alpha"] for h in so["hist"]]}
        del dm, so

    # end to end through the C-ABI with host buffers (pinned), copies inside the timing
    e2e = None
    if not args.no_e2e:
        pin = {k: torch.from_numpy(np.ascontiguousarray(v.astype(npdt))).pin_memory() for k, v in prob_np.items()}
        pin_np = {k: v.numpy() for k, v in pin.items()}
        shapes = dict(K=(T, m, n), k=(T, m), x=(T + 1, n), u=(T, m))
        if mr:
            shapes["lam"] = (T + 1, n)  # refinement corrects the multipliers too
        outp = {k: torch.empty(s, dtype=dt).pin_memory().numpy() for k, s in shapes.items()}
        for _ in range(2):
            solver.solve_host(pin_np, num_segments=K, prec=prec, out_np=outp, form=args.form, max_refine=mr,
                              tol=args.tol)
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        e2e_steps = max(3, args.steps // 2)
        for _ in range(e2e_steps):
            solver.solve_host(pin_np, num_segments=K, prec=prec, out_np=outp, form=args.form, max_refine=mr,
                              tol=args.tol)
        el = max_over_ranks([time.perf_counter() - t0], world, device)[0]
        h2d = sum(v.nbytes for v in pin_np.values())
        d2h = sum(v.nbytes for v in outp.values())
        e2e = {"value": whole_job_rate(T, e2e_steps, world, el), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "steps": e2e_steps}

    cpu, errors = None, None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu, ref = cpu_baseline(wl, prob_np, budget_s=12.0)
        if ref is not None:
            errors = {k: float(np.abs(answer[k] - ref[k]).max() / np.abs(ref[k]).max())
                      for k in ("K", "k", "x", "u", "lam")}
            if gpp_answer is not None and "global_policy_parallel" in extras:
                extras["global_policy_parallel"]["errors_vs_fp64_oracle"] = {
                    k: float(np.abs(gpp_answer[k] - ref[k]).max() / np.abs(ref[k]).max()) for k in ("K", "k", "P", "p")}

    if rank == 0:
        config = {"workload": "%s, K=%d segments, %s" % (wl["name"], K, prec.upper()),
                  "n": n, "m": m, "T": T, "K": K, "precision": prec, "form": args.form,
                  "kkt_backward_error": res["eta"], "kkt_rel_residual": res["rel"],
                  "refinement_corrections": res["iters"] if mr else 0,
                  "refine_tol": args.tol if mr else None,
                  "errors_vs_fp64_oracle": errors,
                  "l2": "inputs (%.0f MB) larger than L2 (129 MB)" % (
                      sum(v.nbytes for v in prob_np.values()) * (1 if es == 8 else 0.5) / 1e6),
                  "parallelism": "replicas" if world > 1 else "single GPU"}
        config.update(extras)
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": {"fp64": "f64", "fp32": "f32", "mixed": "f32+f64", "mixed_fp32": "f32+f64"}[prec],
                "data": "synthetic (seeded PCG64), inputs resident in HBM",
                "config": config, "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk,
                "gpu_launches": launches_per_step * args.steps}
        print(json.dumps(line), flush=True)
    solver.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
