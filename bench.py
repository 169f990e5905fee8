#!/usr/bin/env python3
"""Benchmark: QNG steps per second on the 12-qubit, P = 192, complex128 workload.

One step = the whole hot path for one instance: per-parameter coefficients, the checkpoint /
energy / adjoint-seed sweep, the O(P^2) recurrence of Algorithm 1 plus the reverse gradient
sweep, the assembly of g = Re G and the Cholesky solve of (g + lambda I) dtheta = -dt grad<E>.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload NAME]

Prints one JSON line (rank 0). Under torchrun each rank runs an independent replica of the
workload (no collective on the data path); the timed region is bracketed by barriers and the
slowest rank's time is used. ``--impl reference`` times the CPU oracle (the plain complex128
definition) on the host cores instead.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "QNG steps/s (g,∇E,Δθ) per config; HBM GB/s vs GB300 peak; max err vs FP64 oracle"
# float64 peak: 2 FMA lanes per SM per clock (measured DFMA issue rate on this part) x 2 flop x
# 152 SMs x 2.07 GHz maximum SM clock
FP64_PEAK_TFLOPS = 2 * 2 * 152 * 2.07e9 / 1e12
FP32_PEAK_TFLOPS = 128 * 2 * 152 * 2.07e9 / 1e12


def workloads():
    from paper_2011_02991_gb300 import workloads as W
    return {
        "rand12_p192_c128": lambda: W.config_rand12(precision=W.C128),
        "rand12_p192_c64": lambda: W.config_rand12(precision=W.C64),
        "tfim4_p16_c128": W.config_tfim4,
    }


DESCRIPTION = {
    "rand12_p192_c128": "12 qubits, 8 x [Ry all, Rz all, CZ ladder] (P=192), 40 random Pauli strings "
                        "(weight 1-4, N(0,1) coefficients), theta ~ U[0,2pi), complex128, dt=0.1, lambda=1e-3",
    "rand12_p192_c64": "as rand12_p192_c128 with complex64 amplitudes (float64 accumulation)",
    "tfim4_p16_c128": "4 qubits, 2 x [Ry, Rz, CZ ladder] (P=16), open TFIM, complex128",
}


# ------------------------------------------------------------------------------------------
def column_flops(P: int, n: int) -> float:
    """Float arithmetic of the recurrence kernel per launch (metric columns + gradient column).

    Per amplitude: the real (or imaginary) part of one inner product = 2 FMA = 4 flop; one
    adjoint rotation in scaled form = 1 FMA per real component = 4 flop. Counts: inner products
    P(P-1)/2 (L_ij, i<j) + P (<sigma_j>) + P (gradient); rotations (P-1)(P-2)/2 + (P-1).
    """
    N = float(1 << n)
    ips = P * (P - 1) / 2 + P + P
    rots = (P - 1) * (P - 2) / 2 + (P - 1)
    return N * 4.0 * (ips + rots)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 100 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines: list[str] = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------------------------------
def oracle_step_time(problem, budget_s: float, max_steps: int):
    """Time full oracle QNG steps for about budget_s seconds (at least one)."""
    from oracle import oracle as O
    O.build()
    times = []
    t_all = time.perf_counter()
    while len(times) < max_steps and (not times or time.perf_counter() - t_all < budget_s):
        t0 = time.perf_counter()
        O.qng_step(problem)
        times.append(time.perf_counter() - t0)
    return times


def cpu_threads_used(n: int) -> int:
    # the oracle's loops only go parallel for states of at least 2^16 amplitudes
    from oracle import oracle as O
    return O.num_threads() if n >= 16 else 1


def run_reference(args, name, problem, rank, world):
    if rank != 0:
        return
    from oracle import oracle as O
    O.build()
    for _ in range(min(args.warmup, 1)):
        O.qng_step(problem)
    t0 = time.perf_counter()
    O.qng_step(problem)
    t_one = time.perf_counter() - t0
    k = max(1, min(args.steps, int(100.0 / max(t_one, 1e-6))))
    t0 = time.perf_counter()
    for _ in range(k):
        O.qng_step(problem)
    el = time.perf_counter() - t0
    value = k / el
    cores = cpu_threads_used(problem.n)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": world,
            "steps": k, "steps_requested": args.steps, "warmup": min(args.warmup, 1),
            "ms_per_step": 1e3 * el / k, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{name}: {DESCRIPTION[name]}", "n_qubits": problem.n, "P": problem.P,
                       "parallelism": "single host process"},
            "cpu_baseline": {"value": value, "unit": "steps/s", "cores": cores, "kind": "oracle",
                             "sample": f"{k} full oracle QNG steps (of {args.steps} requested, capped at ~100 s)"},
            "e2e": {"value": value, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args, name, problem, rank, world, local_rank):
    import torch
    import torch.distributed as dist
    from paper_2011_02991_gb300 import build as B
    from paper_2011_02991_gb300 import qng
    from paper_2011_02991_gb300 import workloads as W

    B.build()
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(stream):
        ctx = qng.Context(problem, device=dev, stream=stream)
        theta = ctx.theta0()
        outs = {"dtheta": ctx._f64(ctx.total_params), "g": ctx._f64(ctx.total_metric),
                "grad": ctx._f64(ctx.total_params), "energy": ctx._f64(ctx.count)}
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > 129 MB L2

        # accuracy against the oracle (outside the timed region, rank 0)
        err = None
        if rank == 0:
            from oracle import oracle as O
            ctx.step(theta, problem.dt, problem.lam, outs)
            ctx.sync()
            ref = O.qng_step(problem)
            rel = lambda a, b: float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))  # noqa: E731
            err = {"g": rel(outs["g"].cpu().numpy(), ref["g"].ravel()),
                   "grad": rel(outs["grad"].cpu().numpy(), ref["grad"]),
                   "dtheta": rel(outs["dtheta"].cpu().numpy(), ref["dtheta"]),
                   "E": rel(outs["energy"].cpu().numpy(), np.array([ref["E"]]))}

        for _ in range(args.warmup):
            flush.zero_()
            ctx.step(theta, problem.dt, problem.lam, outs)
        ctx.sync()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)
        clocks = ClockSampler(local_rank)
        clocks.start()
        time.sleep(0.25)
        ctx.profile(True)
        launches0 = 0
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record(stream)
            ctx.step(theta, problem.dt, problem.lam, outs)
            launches0 += ctx.last_launch_count()
            ev[k][1].record(stream)
        torch.cuda.synchronize(dev)
        prof = ctx.profile_read()
        ctx.profile(False)
        ck = clocks.stop()
        ctx.sync()
        ms = sum(a.elapsed_time(b) for a, b in ev)
        t = torch.tensor([ms], dtype=torch.float64, device=dev)
        if world > 1:
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            dist.barrier()
        ms_max = float(t.item())

        # end to end through the public host-buffer entry point (pinned host memory)
        th_host = torch.from_numpy(problem.theta.copy()).pin_memory().numpy()
        hout = {"dtheta": torch.empty(ctx.total_params, dtype=torch.float64).pin_memory().numpy(),
                "g": torch.empty(ctx.total_metric, dtype=torch.float64).pin_memory().numpy(),
                "grad": torch.empty(ctx.total_params, dtype=torch.float64).pin_memory().numpy(),
                "energy": torch.empty(ctx.count, dtype=torch.float64).pin_memory().numpy()}
        for _ in range(max(1, args.warmup // 2)):
            ctx.step_host(th_host, problem.dt, problem.lam, hout)
        if world > 1:
            dist.barrier()
        e2e_ms = 0.0
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            ctx.step_host(th_host, problem.dt, problem.lam, hout)
            e2e_ms += 1e3 * (time.perf_counter() - t0)
        te = torch.tensor([e2e_ms], dtype=torch.float64, device=dev)
        if world > 1:
            dist.all_reduce(te, op=dist.ReduceOp.MAX)
        e2e_ms = float(te.item())

    if rank != 0:
        return
    steps_total = args.steps * world
    value = steps_total / (ms_max / 1e3)
    col_ms, col_n = prof["columns"]
    col_avg_s = col_ms / max(col_n, 1) / 1e3
    flops = column_flops(problem.P, problem.n)
    prec64 = problem.precision == W.C128
    peak = FP64_PEAK_TFLOPS if prec64 else FP32_PEAK_TFLOPS
    achieved = flops / col_avg_s / 1e12
    kernel_share = {k: round(v[0] / max(sum(x[0] for x in prof.values()), 1e-12), 4) for k, v in prof.items()}

    # CPU baseline: the oracle on the host cores, a bounded sample
    times = oracle_step_time(problem, budget_s=args.cpu_budget, max_steps=30)
    cpu_value = len(times) / sum(times)

    P, N = problem.P, ctx.count
    line = {
        "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if prec64 else "f32 (f64 accumulation, assembly, solve)",
        "data": "synthetic",
        "config": {"workload": f"{name}: {DESCRIPTION[name]}", "n_qubits": problem.n, "P": P,
                   "precision": "c128" if prec64 else "c64",
                   "l2": "flushed between timed steps (256 MiB write, untimed)",
                   "parallelism": "independent replica per GPU" if world > 1 else "single GPU"},
        "max_err_vs_oracle": err,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": None,
                     "kernel": "k_columns (recurrence + gradient sweep)",
                     "peak_source": "derived: float64 2 FMA/clk/SM x 152 SMs x 2.07 GHz" if prec64 else
                                    "derived: float32 128 FMA/clk/SM x 152 SMs x 2.07 GHz",
                     "kernel_avg_ms": col_avg_s * 1e3, "flops_per_launch": flops},
        "kernel_share": kernel_share,
        "cpu_baseline": {"value": cpu_value, "unit": "steps/s", "cores": cpu_threads_used(problem.n), "kind": "oracle",
                         "sample": f"{len(times)} full oracle QNG steps of the same workload ({sum(times):.1f} s)"},
        "e2e": {"value": steps_total / (e2e_ms / 1e3), "unit": "steps/s", "h2d_bytes_per_step": 8 * P,
                "d2h_bytes_per_step": 8 * (P * P + 2 * P + N)},
        "gpu_launches": int(launches0),
        "clocks": {k: ck[k] for k in ("sm_mhz", "sm_max_mhz", "reasons")},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="rand12_p192_c128")
    ap.add_argument("--cpu-budget", type=float, default=12.0, help="seconds of oracle time for cpu_baseline")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    name = args.workload
    problem = workloads()[name]()
    if args.impl == "reference":
        run_reference(args, name, problem, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", init_method="env://")
    try:
        run_ours(args, name, problem, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
