#!/usr/bin/env python3
"""Benchmark: QNG steps per second per configuration; the headline line is the largest single-GPU
configuration, 28 qubits complex64 (3 x [Ry, Rx, Rz all, CNOT ladder], P = 252, 2 GiB per state).

One step = the whole hot path for one instance (or a batch): per-parameter coefficients, the forward
sweep, the energy and the reverse gradient sweep, the O(P^2) recurrence of Algorithm 1, the assembly
of g = Re G and the solve of (g + lambda I) dtheta = -dt grad<E>.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload NAME]

Prints one JSON line (rank 0). Under torchrun each rank runs an independent replica of the
workload (no collective on the data path); the timed region is bracketed by barriers and the
slowest rank's time is used. The line carries a per_config block: the other configurations
(12 qubits complex128 and complex64, the 256-instance batch in both precisions, 26 qubits
complex128) measured in the same run, so the batched and complex64 forms are reported next to the
plain complex128 form. ``--impl reference`` times the CPU oracle (the plain complex128 definition)
on the host cores instead.
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
HBM_PEAK_GBS = 6669.2  # measured copy bandwidth of this GPU pool
# DRAM bytes (read + write) per launch of the timed kernel, from one ncu capture of this build's
# kernel on the workload; None where no capture of the current kernel exists. 12 qubits
# (profiles/rand12_p192_c128_step.md): only the first read of the checkpoints reaches DRAM. 28 qubits
# (profiles/rand28_p252_c64_step.md): mean over 30 consecutive metric passes, each reading the
# registers it loads and writing the ones it stores.
TRAFFIC = {"rand12_p192_c128": 12894976, "rand28_p252_c64": 11972552388}


def workloads():
    """name -> (problem or list of problems, kind: single | batch | stream | loop).
    loop: one instance, each timed step is one descent iteration (qng_optimize: step + update)."""
    from paper_2011_02991_gb300 import workloads as W
    return {
        "rand12_p192_c128": (lambda: W.config_rand12(precision=W.C128), "single"),
        "rand12_p192_c64": (lambda: W.config_rand12(precision=W.C64), "single"),
        "tfim4_p16_c128": (W.config_tfim4, "single"),
        "batch256_c64": (lambda: W.config_batch(precision=W.C64), "batch"),
        "batch256_c128": (lambda: W.config_batch(precision=W.C128), "batch"),
        "tfim26_p208_c128": (W.config_tfim26, "stream"),
        "rand28_p252_c64": (lambda: W.config_rand28(precision=W.C64), "stream"),
        "rand28_p252_c128": (lambda: W.config_rand28(precision=W.C128), "stream"),
        "tfim24_p48_c128": (lambda: W.config_tfim26(n=24, layers=1), "stream"),
        "tfim24_p48_c64": (lambda: _c64(W.config_tfim26(n=24, layers=1)), "stream"),
        "general12_p192_c128": (lambda: W.general_problem(12, 192, W.BASE_SEED + 6), "single"),
        "vqe_tfim12_p144_c128": (lambda: W.vqe_tfim(12, 6), "loop"),
    }


def _c64(p):
    from paper_2011_02991_gb300 import workloads as W
    return W.Problem(p.name.replace("c128", "c64"), p.circuit, p.hamiltonian, p.theta, precision=W.C64, meta=p.meta)


DESCRIPTION = {
    "rand12_p192_c128": "12 qubits, 8 x [Ry all, Rz all, CZ ladder] (P=192), 40 random Pauli strings "
                        "(weight 1-4, N(0,1) coefficients), theta ~ U[0,2pi), complex128, dt=0.1, lambda=1e-3",
    "rand12_p192_c64": "as rand12_p192_c128 with complex64 amplitudes (float64 accumulation, assembly, solve)",
    "tfim4_p16_c128": "4 qubits, 2 x [Ry, Rz, CZ ladder] (P=16), open TFIM, complex128",
    "batch256_c64": "256 instances, n ~ U{6..14}, 2-10 Ry/Rz/CZ layers (P 24-280), 16-48 strings each, complex64",
    "batch256_c128": "the same 256 instances in complex128",
    "tfim26_p208_c128": "26 qubits, 4 x [Ry, Rz, CZ ladder] (P=208), TFIM J=1, h ~ U[0.2,1], complex128 (1 GiB per state)",
    "rand28_p252_c64": "28 qubits, 3 x [Ry, Rx, Rz all, CNOT ladder] (P=252), 64 strings, complex64 (2 GiB per state)",
    "rand28_p252_c128": "as rand28_p252_c64 in complex128 (4 GiB per state)",
    "tfim24_p48_c128": "24 qubits, 1 x [Ry, Rz, CZ ladder] (P=48), TFIM, complex128 (streaming, profiling case)",
    "tfim24_p48_c64": "as tfim24_p48_c128 in complex64",
    "general12_p192_c128": "12 qubits, P=192 mixing Rx/Ry/Rz, CRx/CRy/CRz and (controlled) Pauli-string rotations "
                           "of weight 1-3 with CZ/CNOT/H between them, 24 random Pauli strings, complex128 "
                           "(roofline flops count the ordinary-rotation work per element)",
    "vqe_tfim12_p144_c128": "natural-gradient descent (qng_optimize, one iteration per step: step + theta update) "
                            "on the open TFIM chain, 12 qubits, 6 x [Ry, Rz, CZ ladder] (P=144), complex128",
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


def stream_flops_per_amp(P: int) -> float:
    """Float64 arithmetic of the streaming metric segment per amplitude, as the schedule runs it.

    Columns l, l + 1 (l odd, l + 1 < P) walk together: column l + 1's first step alone, then one
    paired step per i < l (two inner products, rotations of a, b and b2); other columns alone.
    Per amplitude: an inner product's real part = 2 FMA = 4 flop; an adjoint rotation in scaled
    form = 2 FMA = 4 flop per register; the step i = 0 has no rotation.
    """
    def single(i):
        return 4.0 + (8.0 if i > 0 else 0.0)

    def paired(i):
        return 8.0 + (12.0 if i > 0 else 0.0)

    total, j = 0.0, 1
    while j < P:
        if j % 2 == 1 and j + 1 < P:
            total += single(j) + sum(paired(i) for i in range(j))
            j += 2
        else:
            total += sum(single(i) for i in range(j))
            j += 1
    return total


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
def _rel(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def sample_ids(kind, problems):
    """Instances (batch) or parameter indices (stream) the oracle checks and times."""
    if kind == "batch":
        rng = np.random.default_rng(11)
        return sorted(rng.choice(len(problems), min(8, len(problems)), replace=False).tolist())
    if kind == "stream":
        P = problems[0].P
        return [0, P // 2, P - 1][: max(1, min(3, P))]
    return None


def oracle_check(kind, problems, ctx, outs):
    """Max relative error of the GPU outputs against the oracle (sampled where the full oracle is out of reach)."""
    from oracle import oracle as O
    g, grad, dth, en = (outs[k].cpu().numpy() for k in ("g", "grad", "dtheta", "energy"))
    if kind == "single":
        ref = O.qng_step(problems[0])
        return {"g": _rel(g, ref["g"]), "grad": _rel(grad, ref["grad"]), "dtheta": _rel(dth, ref["dtheta"]),
                "E": _rel(en, [ref["E"]])}
    if kind == "batch":
        err = {"g": 0.0, "grad": 0.0, "dtheta": 0.0, "E": 0.0}
        for b in sample_ids(kind, problems):
            ref = O.qng_step(problems[b])
            p0, p1 = ctx.param_offsets[b], ctx.param_offsets[b + 1]
            m0, m1 = ctx.metric_offsets[b], ctx.metric_offsets[b + 1]
            err["g"] = max(err["g"], _rel(g[m0:m1], ref["g"]))
            err["grad"] = max(err["grad"], _rel(grad[p0:p1], ref["grad"]))
            err["dtheta"] = max(err["dtheta"], _rel(dth[p0:p1], ref["dtheta"]))
            err["E"] = max(err["E"], _rel(en[b:b + 1], [ref["E"]]))
        err["sample"] = f"{len(sample_ids(kind, problems))} instances"
        return err
    p = problems[0]
    idx = np.array(sample_ids(kind, problems), dtype=np.int32)
    Gs, Ts, grads, E = O.sampled(p, idx)
    gm = g.reshape(p.P, p.P)
    r = (gm + p.lam * np.eye(p.P)) @ dth + p.dt * grad
    return {"g": _rel(gm[np.ix_(idx, idx)], Gs.real), "grad": _rel(grad[idx], grads), "E": _rel(en, [E]),
            "dtheta_residual": float(np.linalg.norm(r) / max(np.linalg.norm(p.dt * grad), 1e-300)),
            "sample": f"parameters {idx.tolist()} (sampled oracle entries)"}


def cpu_info() -> dict:
    """Host cores and CPU model of the machine the oracle runs on."""
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                k, _, v = ln.partition(":")
                if k.strip() in ("model name", "Model Name"):
                    model = v.strip()
                    break
    except OSError:
        pass
    if model is None:
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            for ln in out.splitlines():
                if ln.startswith("Model name:"):
                    model = ln.split(":", 1)[1].strip()
                    break
        except (OSError, subprocess.SubprocessError):
            pass
    import platform
    return {"cores": os.cpu_count(), "cpu_model": model or platform.machine()}


def oracle_baseline(kind, problems, budget_s):
    """Oracle throughput on all host cores: (steps/s, sample description, threads used)."""
    from oracle import oracle as O
    O.build()
    O.set_num_threads(os.cpu_count() or 1)
    threads = O.num_threads()
    if kind == "single":
        times, t_all = [], time.perf_counter()
        while len(times) < 30 and (not times or time.perf_counter() - t_all < budget_s):
            t0 = time.perf_counter()
            O.qng_step(problems[0])
            times.append(time.perf_counter() - t0)
        return len(times) / sum(times), f"{len(times)} full oracle QNG steps of the same workload ({sum(times):.1f} s)", threads
    if kind == "batch":
        ids, times, t_all = sample_ids(kind, problems), [], time.perf_counter()
        k = 0
        while not times or (time.perf_counter() - t_all < budget_s and k < 64):
            t0 = time.perf_counter()
            O.qng_step(problems[ids[k % len(ids)]])
            times.append(time.perf_counter() - t0)
            k += 1
        per_instance = sum(times) / len(times)
        return 1.0 / (per_instance * len(problems)), (
            f"{len(times)} oracle QNG steps of {len(ids)} sampled instances ({sum(times):.1f} s), "
            f"extrapolated to all {len(problems)} instances"), threads
    p = problems[0]
    idx = np.array([p.P // 2], dtype=np.int32)
    t0 = time.perf_counter()
    O.sampled(p, idx)
    t = time.perf_counter() - t0
    m = len(idx)
    full = t * (p.P + 2) / (m + 2)  # one circuit run per derivative state dominates the definition's cost
    return 1.0 / full, (f"oracle sampled-entry mode at the full size: psi, H psi and {m} derivative state "
                        f"in {t:.1f} s, extrapolated to the P + 2 circuit runs of a full step"), threads


def alg1_mirror(problem, budget_s=20.0):
    """The literal Algorithm 1 (Sec. 3) on the CPU: metric recurrences per second (L and T, no
    gradient or solve), the same algorithm the GPU runs, timed on the host for context."""
    from oracle import oracle as O
    O.build()
    O.set_num_threads(os.cpu_count() or 1)
    times, t_all = [], time.perf_counter()
    while len(times) < 10 and (not times or time.perf_counter() - t_all < budget_s):
        t0 = time.perf_counter()
        O.alg1(problem.circuit, problem.theta)
        times.append(time.perf_counter() - t0)
    return {"value": len(times) / sum(times), "unit": "metric recurrences/s",
            "sample": f"{len(times)} runs of the literal Algorithm 1 ({sum(times):.1f} s)",
            "threads": O.num_threads() if problem.n >= 16 else 1}


def run_reference(args, name, problems, kind, rank, world):
    if rank != 0:
        return
    from oracle import oracle as O
    O.build()
    O.set_num_threads(os.cpu_count() or 1)
    threads = O.num_threads()
    if kind == "single":
        p = problems[0]
        warm, tw = 0, time.perf_counter()
        while warm < args.warmup and (warm == 0 or time.perf_counter() - tw < 30.0):  # bounded host time
            O.qng_step(p)
            warm += 1
        t0 = time.perf_counter()
        O.qng_step(p)
        t_one = time.perf_counter() - t0
        k = max(1, min(args.steps, int(100.0 / max(t_one, 1e-6))))
        t0 = time.perf_counter()
        for _ in range(k):
            O.qng_step(p)
        el = time.perf_counter() - t0
        value, steps, sample = k / el, k, f"{k} full oracle QNG steps (of {args.steps} requested, capped at ~100 s)"
        ms = 1e3 * el / k
    else:
        value, sample, threads = oracle_baseline(kind, problems, budget_s=60.0)
        steps, ms, warm = 1, 1e3 / value, 0
    info = cpu_info()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": world,
            "steps": steps, "steps_requested": args.steps, "warmup": warm, "warmup_requested": args.warmup,
            "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{name}: {DESCRIPTION[name]}", "parallelism": "single host process"},
            "cpu_baseline": {"value": value, "unit": "steps/s", "cores": threads, "cpu_model": info["cpu_model"],
                             "host_cores": info["cores"], "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def make_problems(name, world, rank, shard):
    make, kind = workloads()[name]
    loop = kind == "loop"
    if loop:
        kind = "single"
    made = make()
    problems = made if isinstance(made, list) else [made]
    sharded = False
    if shard and kind == "batch" and world > 1:
        from paper_2011_02991_gb300 import dist as D
        problems = [problems[b] for b in D.shard_batch(problems, world)[rank]]
        sharded = True
    return problems, kind, loop, sharded


def measure(name, steps, warmup, dev, rank, world, local_rank, check=True, shard=False, e2e_steps=None,
            clocks=False):
    """Time `steps` QNG steps of workload `name` (after `warmup` untimed ones) on `dev`; returns a dict."""
    import torch
    import torch.distributed as dist
    from paper_2011_02991_gb300 import qng

    problems, kind, loop, sharded = make_problems(name, world, rank, shard)
    stream = torch.cuda.Stream(device=dev)
    dt, lam = problems[0].dt, problems[0].lam
    res = {"name": name, "kind": kind, "problems": problems, "sharded": sharded}
    with torch.cuda.stream(stream):
        ctx = qng.Context(problems if kind == "batch" else problems[0], device=dev, stream=stream)
        theta = ctx.theta0()
        outs = {"dtheta": ctx._f64(ctx.total_params), "g": ctx._f64(ctx.total_metric),
                "grad": ctx._f64(ctx.total_params), "energy": ctx._f64(ctx.count)}
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > 129 MB L2

        res["err"] = None
        if rank == 0 and check:
            ctx.step(theta, dt, lam, outs)
            ctx.sync()
            res["err"] = oracle_check(kind, problems, ctx, outs)

        theta_loop = theta.clone()
        if loop:  # one descent iteration per step, theta updated on the device
            def one_step():
                ctx.optimize(theta_loop, dt, lam, 1)
        else:
            def one_step():
                ctx.step(theta, dt, lam, outs)
        for _ in range(warmup):
            flush.zero_()
            one_step()
        ctx.sync()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)
        sampler = ClockSampler(local_rank) if clocks else None
        if sampler:
            sampler.start()
            time.sleep(0.25)
        ctx.profile(True)
        launches = 0
        for k in range(steps):
            flush.zero_()
            ev[k][0].record(stream)
            one_step()
            launches += ctx.last_launch_count()
            ev[k][1].record(stream)
        torch.cuda.synchronize(dev)
        prof = ctx.profile_read()
        ctx.profile(False)
        res["clocks"] = sampler.stop() if sampler else None
        ctx.sync()
        ms = sum(a.elapsed_time(b) for a, b in ev)
        t = torch.tensor([ms], dtype=torch.float64, device=dev)
        if world > 1:
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            dist.barrier()
        res["ms_total"] = float(t.item())
        res["launches"] = launches
        res["prof"] = prof
        res["pipeline"] = ctx.pipeline() if kind != "stream" else 0
        res["sizes"] = (ctx.total_params, ctx.total_metric, ctx.count)
        if kind == "stream":
            res["traffic"] = ctx.stream_traffic()
            res["segments"] = ctx.stream_segments()

        # end to end through the public host-buffer entry point (pinned host memory)
        res["e2e_ms"] = None
        if e2e_steps:
            th_host = torch.from_numpy(np.concatenate([p.theta for p in problems]).astype(np.float64)).pin_memory().numpy()
            hout = {"dtheta": torch.empty(ctx.total_params, dtype=torch.float64).pin_memory().numpy(),
                    "g": torch.empty(ctx.total_metric, dtype=torch.float64).pin_memory().numpy(),
                    "grad": torch.empty(ctx.total_params, dtype=torch.float64).pin_memory().numpy(),
                    "energy": torch.empty(ctx.count, dtype=torch.float64).pin_memory().numpy()}
            ctx.step_host(th_host, dt, lam, hout)
            if world > 1:
                dist.barrier()
            e2e_ms = 0.0
            for _ in range(e2e_steps):
                flush.zero_()
                torch.cuda.synchronize(dev)
                t0 = time.perf_counter()
                ctx.step_host(th_host, dt, lam, hout)
                e2e_ms += 1e3 * (time.perf_counter() - t0)
            te = torch.tensor([e2e_ms / e2e_steps], dtype=torch.float64, device=dev)
            if world > 1:
                dist.all_reduce(te, op=dist.ReduceOp.MAX)
            res["e2e_ms"] = float(te.item())
            res["e2e_steps"] = e2e_steps
        ctx.close()
        del flush, outs, theta, theta_loop
    torch.cuda.synchronize(dev)
    torch.cuda.empty_cache()
    return res


def roofline(res, steps):
    """Roofline of the step's dominant kernel class (see DESIGN: algorithmic work per unit)."""
    from paper_2011_02991_gb300 import workloads as W
    problems, kind, prof, name = res["problems"], res["kind"], res["prof"], res["name"]
    prec64 = problems[0].precision == W.C128
    col_ms, col_n = prof["columns"]
    if kind == "stream":
        mb, ob, mp = res["traffic"]
        p = problems[0]
        met_s = col_ms / steps / 1e3
        if prec64:
            flops = (1 << p.n) * stream_flops_per_amp(p.P)  # paired columns share the rotation of a
            achieved = flops / met_s / 1e12
            return {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                    "frac": achieved / FP64_PEAK_TFLOPS, "traffic": None,
                    "kernel": "k_pass metric passes", "kernel_avg_ms": met_s * 1e3 * steps / max(col_n, 1),
                    "flops_per_step": flops, "launches_per_step": col_n / steps,
                    "peak_source": "derived: float64 2 FMA/clk/SM x 152 SMs x 2.07 GHz"}
        achieved = mb / met_s / 1e9
        traffic = TRAFFIC.get(name)
        return {"bound": "hbm", "achieved": achieved, "peak": HBM_PEAK_GBS, "unit": "GB/s",
                "frac": achieved / HBM_PEAK_GBS, "traffic": traffic,
                "kernel": "k_pass_phased metric passes (registers loaded and stored per pass)",
                "kernel_avg_ms": col_ms / max(col_n, 1), "bytes_per_launch": mb / max(mp, 1),
                "bytes_per_step": mb, "launches_per_step": mp, "peak_source": "measured copy bandwidth (of measured)"}
    col_avg_s = col_ms / max(col_n, 1) / 1e3
    launches_per_step = col_n / max(steps, 1)
    flops_step = sum(column_flops(p.P, p.n) for p in problems)  # all instances, all column launches of a step
    flops = flops_step / max(launches_per_step, 1)                # per launch, averaged
    peak = FP64_PEAK_TFLOPS if prec64 else FP32_PEAK_TFLOPS
    achieved = flops_step * steps / (col_ms / 1e3) / 1e12 if col_ms > 0 else 0.0
    # complex128 batches run their launch groups side by side: the column launches overlap, and the
    # sum of their durations overstates the time; the whole step's time bounds it from above
    overlap = kind == "batch" and prec64
    if overlap:
        achieved = flops_step * steps / (res["ms_total"] / 1e3) / 1e12
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": TRAFFIC.get(name), "kernel": "k_columns (recurrence + gradient sweep)",
            "peak_source": "derived: float64 2 FMA/clk/SM x 152 SMs x 2.07 GHz" if prec64 else
                           "derived: float32 128 FMA/clk/SM x 152 SMs x 2.07 GHz",
            "kernel_avg_ms": col_avg_s * 1e3, "flops_per_launch": flops, "launches_per_step": launches_per_step}
    if overlap:
        roof["note"] = ("launch groups side by side: achieved divides the step's column flops by the whole "
                        "step's time (sweep and solve included), a lower bound")
    if res["pipeline"]:
        roof["note"] = ("pipelined sweep: the column launches overlap one another and the sweep; achieved divides "
                        "the step's column flops by the sum of their durations, a lower bound")
    return roof


def segment_rates(res, steps):
    """Streaming path: algorithmic HBM bytes and GB/s of every kernel class in one step."""
    out = {}
    for k, (b, n) in res["segments"].items():
        ms, launches = res["prof"][k]
        if n == 0 or launches == 0:
            continue
        out[k] = {"bytes_per_step": int(b), "launches_per_step": int(n), "ms_per_step": ms / steps,
                  "GBps": b / (ms / steps / 1e3) / 1e9 if ms > 0 else None,
                  "frac_of_hbm": (b / (ms / steps / 1e3) / 1e9) / HBM_PEAK_GBS if ms > 0 else None}
    return out


# configurations reported beside the headline (per_config): name -> (timed steps, warm-up steps)
PER_CONFIG = {
    "rand12_p192_c128": (100, 10),
    "rand12_p192_c64": (100, 10),
    "batch256_c128": (6, 3),
    "batch256_c64": (20, 3),
    "tfim26_p208_c128": (2, 3),
}


def run_ours(args, name, rank, world, local_rank):
    import torch
    from paper_2011_02991_gb300 import build as B
    from paper_2011_02991_gb300 import workloads as W

    B.build()
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    kind0 = workloads()[name][1]
    e2e_steps = args.steps if kind0 != "stream" else min(args.steps, 2)
    res = measure(name, args.steps, args.warmup, dev, rank, world, local_rank, check=not args.no_check,
                  shard=args.shard, e2e_steps=e2e_steps, clocks=True)
    per = {}
    if rank == 0 and world == 1 and not args.no_per_config:
        plain = None
        for other, (k, w) in PER_CONFIG.items():
            if other == name:
                continue
            r = measure(other, k, w, dev, rank, world, local_rank, check=not args.no_check)
            v = k / (r["ms_total"] / 1e3)
            rf = roofline(r, k)
            per[other] = {"value": v, "unit": "steps/s", "ms_per_step": r["ms_total"] / k, "steps": k, "warmup": w,
                          "workload": DESCRIPTION[other], "max_err_vs_oracle": r["err"],
                          "roofline": {key: rf[key] for key in ("bound", "achieved", "peak", "unit", "frac")}}
            if r["kind"] == "stream":
                per[other]["segments"] = segment_rates(r, k)
            if other == "rand12_p192_c128":
                plain = v
        if plain:
            for other in per:
                if other.startswith("rand12") or other.startswith("batch256"):
                    per[other]["vs_rand12_c128_steps"] = per[other]["value"] / plain
        if "rand12_p192_c128" in per:
            per["rand12_p192_c128"]["cpu_alg1_mirror"] = alg1_mirror(W.config_rand12())
    if rank != 0:
        return
    problems, kind, prof = res["problems"], res["kind"], res["prof"]
    steps = args.steps
    value = steps * (1 if res["sharded"] else world) / (res["ms_total"] / 1e3)
    prec64 = problems[0].precision == W.C128
    roof = roofline(res, steps)
    total_prof = max(sum(x[0] for x in prof.values()), 1e-12)
    kernel_share = {k: round(v[0] / total_prof, 4) for k, v in prof.items() if v[1] > 0}
    if args.cpu_budget > 0:
        cpu_value, cpu_sample, cpu_threads = oracle_baseline(kind, problems, args.cpu_budget)
    else:
        cpu_value, cpu_sample, cpu_threads = None, "skipped", None
    P_tot, M_tot, cnt = res["sizes"]
    info = cpu_info()
    line = {
        "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": world, "steps": steps,
        "warmup": args.warmup, "ms_per_step": res["ms_total"] / steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if prec64 else "f32 (f64 accumulation, assembly, solve)",
        "data": "synthetic",
        "config": {"workload": f"{name}: {DESCRIPTION[name]}", "instances": cnt,
                   "n_qubits": sorted({p.n for p in problems}), "P_total": P_tot,
                   "precision": "c128" if prec64 else "c64",
                   "path": "streaming" if kind == "stream" else "on-chip",
                   "sweep_chunks": res["pipeline"],
                   "l2": ("inputs larger than L2 (2^n-amplitude registers) and L2 flushed between timed steps "
                          "(256 MiB write, untimed)"),
                   "parallelism": ("batch instances sharded over GPUs (LPT by work), no collective on the data path"
                                   if res["sharded"] else "independent replica per GPU" if world > 1 else "single GPU")},
        "max_err_vs_oracle": res["err"],
        "roofline": roof,
        "kernel_share": kernel_share,
        "cpu_baseline": {"value": cpu_value, "unit": "steps/s", "cores": cpu_threads, "host_cores": info["cores"],
                         "cpu_model": info["cpu_model"], "kind": "oracle", "sample": cpu_sample},
        "e2e": {"value": world / (res["e2e_ms"] / 1e3), "unit": "steps/s", "h2d_bytes_per_step": 8 * P_tot,
                "d2h_bytes_per_step": 8 * (M_tot + 2 * P_tot + cnt), "steps": res["e2e_steps"]},
        "gpu_launches": int(res["launches"]),
        "clocks": {k: res["clocks"][k] for k in ("sm_mhz", "sm_max_mhz", "reasons")},
    }
    if kind == "stream":
        line["segments"] = segment_rates(res, steps)
    if per:
        line["per_config"] = per
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="rand28_p252_c64", choices=sorted(DESCRIPTION))
    ap.add_argument("--cpu-budget", type=float, default=20.0, help="seconds of oracle time for cpu_baseline (0: skip)")
    ap.add_argument("--no-check", action="store_true", help="skip the oracle accuracy checks")
    ap.add_argument("--no-per-config", action="store_true", help="skip the per_config block")
    ap.add_argument("--shard", action="store_true",
                    help="batch workloads under torchrun: split the instances over the ranks (strong scaling) "
                         "instead of one replica per rank")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    name = args.workload
    if args.impl == "reference":
        problems, kind, _, _ = make_problems(name, world, rank, args.shard)
        run_reference(args, name, problems, kind, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", init_method="env://")
    try:
        run_ours(args, name, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
