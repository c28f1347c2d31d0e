"""Benchmark of the DIAM hot path on one B300 (or N replicas under torchrun).

Workload (tanh4096): Bayesian tanh regression, d = 4096, d_y = 2048, prior N(0, diag(i^-2)), A (2048 x 4096)
N(0, 1/4096) in FP32, y = tanh(A x*) + 0.05 eps; P = 256 chains, n_lag = 128, BF16 factor / noise / map on
the tensor cores, FP32 chain states, FP64 Cholesky refresh and moment fold. A_0 = Cholesky of the prior
covariance, x_0 drawn from the prior. One benchmark step = one interval of n_lag steps of all P chains
(noise product, n_lag x (propose, target, accept), moment fold, beta rule and the Cholesky refresh that is
due every interval). Metric: chain-steps/s = P n_lag steps / wall time of the interval, refreshes included.

Prints one JSON line (rank 0). --impl reference times the CPU oracle (the reference arm for this build).
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

PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FP64_PEAK_TFLOPS = 1.25   # B300 nominal FP64 (vector and tensor), the profiling recipe's figure


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=8, help="timed intervals (of n_lag steps each)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--P", type=int, default=256)
    ap.add_argument("--n-lag", type=int, default=128)
    ap.add_argument("--fp64-steps", type=int, default=1, help="timed intervals of the plain FP64 form (0: skip)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline")
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-profile", action="store_true", help="skip the per-phase profile pass (roofline)")
    return ap.parse_args()


def peaks():
    try:
        with open(PEAKS_FILE) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.rows = []
        if self.proc is None:
            return
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out = ""
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def summary(self):
        rows = getattr(self, "rows", [])
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def workload(P, n_lag):
    import workloads
    run = workloads.tanh4096(P=P, n_lag=n_lag)
    ts = run.target
    x0 = workloads.start_state(ts.d, P, 1) * np.sqrt(ts.lam)
    C0 = np.diag(ts.lam)
    return run, ts, x0, C0


def make_sampler(run, ts, x0, C0, prec, profile=0, stream=None):
    import paper_1506_05741_b300 as dm
    cfg = dm.default_config(ts.d, run.P, n_lag=run.n_lag, beta0=run.beta0, seed=run.seed, prec=prec, profile=profile)
    return dm.Sampler(cfg, ts, x0=x0, C0=C0, stream=stream)


def time_intervals(s, n_lag, K, torch, stream):
    """Device time of K intervals with CUDA events on the sampler's stream (synchronised on both sides)."""
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s.run(K * n_lag)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3


def roofline(prof, run, ts, K, pk, pk_src):
    """Dominant phase of the profiled intervals, with its algorithmic work per launch."""
    d, dy, P, nl = ts.d, ts.d_y, run.P, run.n_lag
    N = P * nl
    # algorithmic work per launch of each phase
    work = {
        "refresh": ("alu", d ** 3 / 3.0 + d ** 2, "TFLOP/s", FP64_PEAK_TFLOPS),       # FP64 Cholesky
        "xi_gemm": ("tensor", float(d) * d * N, "TFLOP/s", pk.get("bf16_tflops_sustained", pk["bf16_tflops"])),
        "fold": ("tensor", float(d) * d * N, "TFLOP/s", pk.get("bf16_tflops_sustained", pk["bf16_tflops"])),
        "target": ("tensor", 2.0 * dy * d * P * 2, "TFLOP/s", pk.get("bf16_tflops_sustained", pk["bf16_tflops"])),
        # bytes per launch: propose reads x, z, xi (FP32), W (BF16), writes x*, z* (FP32) and the BF16 split
        "propose": ("hbm", P * d * (4 + 4 + 4 + 2 + 4 + 4 + 2 + 2), "GB/s", pk["hbm_gbs"]),
        # accept reads x*, z* and writes x, z (accepted chains) and the BF16 record; bound at full traffic
        "accept": ("hbm", P * d * (4 + 4 + 4 + 4 + 2), "GB/s", pk["hbm_gbs"]),
        "noise": ("hbm", N * d * 2, "GB/s", pk["hbm_gbs"]),
        "rewhiten": ("alu", float(d) * d * P, "TFLOP/s", FP64_PEAK_TFLOPS),
    }
    total = sum(ms for _, ms in prof.values())
    dom = max(prof.items(), key=lambda kv: kv[1][1])
    name, (cnt, ms) = dom
    bound, units, unit, peak = work[name]
    per_launch_s = ms / 1e3 / max(cnt, 1)
    if unit == "TFLOP/s":
        achieved = units / per_launch_s / 1e12
    else:
        achieved = units / per_launch_s / 1e9
    shares = {k: round(v[1] / total, 4) for k, v in prof.items() if total > 0}
    return {"kernel": name, "bound": bound, "achieved": round(achieved, 3), "peak": peak, "unit": unit,
            "frac": round(achieved / peak, 4), "traffic": None, "launch_ms": round(per_launch_s * 1e3, 4),
            "peak_source": ("nominal FP64 of the profiling recipe" if bound == "alu" else pk_src),
            "phase_share": shares}


def cpu_leg(run, ts, x0, C0, seconds, cores):
    import oracle
    t = oracle.Target(ts.kind, ts.d, ts.d_y, lam=ts.lam, G=ts.G, A=ts.A, y=ts.y, sigma=ts.sigma)
    Ps = max(cores, 8)
    cfg = oracle.default_config(d=ts.d, P=Ps, n_lag=run.n_lag, beta0=run.beta0, seed=run.seed, threads=cores)
    o = oracle.Sampler(cfg, t, x0=x0[:Ps], C0=C0)
    steps = 0
    t0 = time.time()
    while time.time() - t0 < seconds and steps < run.n_lag - 1:
        o.run(1)
        steps += 1
    dt = time.time() - t0
    return {"value": round(Ps * steps / dt, 3), "unit": "chain-steps/s", "cores": cores, "kind": "oracle",
            "sample": f"{steps} steps x {Ps} chains of tanh4096 (FP64 oracle, OpenMP over chains; refresh-free "
                      f"prefix: its amortised Cholesky is ~1.4% of the oracle's per-step work)"}


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    cores = os.cpu_count() or 1
    run, ts, x0, C0 = workload(args.P, args.n_lag)
    N = run.P * run.n_lag
    config = {"workload": f"tanh4096: d={ts.d}, d_y={ts.d_y}, P={run.P}, n_lag={run.n_lag}, BF16 factor/noise/map, "
                          f"FP32 states, FP64 Cholesky refresh every interval",
              "d": ts.d, "d_y": ts.d_y, "P": run.P, "n_lag": run.n_lag,
              "step": "one interval: n_lag steps of all chains + moment fold + beta rule + Cholesky refresh",
              "l2": "working set per interval > L2 (noise product 537 MB, BF16 noise 268 MB)",
              "parallelism": f"replicas x{world} (chains independent; no data-path collective)"}

    if args.impl == "reference":
        if rank != 0:
            return
        cores_used = cores
        t0 = time.time()
        leg = cpu_leg(run, ts, x0, C0, args.cpu_seconds, cores_used)
        line = {"impl": "reference", "metric": "chain-steps/s", "value": leg["value"], "unit": "chain-steps/s",
                "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config,
                "cpu_baseline": leg,
                "e2e": {"value": leg["value"], "unit": "chain-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
                "ms_per_step": round(N / leg["value"] * 1e3, 3), "wall_s": round(time.time() - t0, 2)}
        print(json.dumps(line), flush=True)
        return

    import torch
    import paper_1506_05741_b300 as dm
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    # one non-default stream for the sampler, its CUDA events and its graph replays
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    pk, pk_src = peaks()

    # ---- main timed region: BF16 path
    s = make_sampler(run, ts, x0, C0, dm.BF16, stream=stream.cuda_stream)
    s.run(args.warmup * run.n_lag)
    if world > 1:
        torch.distributed.barrier()
    l0 = dm.kernel_launches()
    with ClockSampler(local) as clk:
        dt = time_intervals(s, run.n_lag, args.steps, torch, stream)
    launches = dm.kernel_launches() - l0
    st = s.stats()
    if world > 1:
        t = torch.tensor([dt], device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        dt = t.item()
    value = world * N * args.steps / dt
    s.close()
    del s

    # ---- profile pass: per-phase device time with CUDA events on the same stream
    roof = None
    if not args.no_profile:
        sp = make_sampler(run, ts, x0, C0, dm.BF16, profile=1, stream=stream.cuda_stream)
        sp.run(args.warmup * run.n_lag)
        sp.profile(reset=True)
        sp.run(max(2, args.steps // 2) * run.n_lag)
        prof = sp.profile()
        sp.close()
        del sp
        roof = roofline(prof, run, ts, args.steps, pk, pk_src)

    # ---- plain FP64 form on the same workload (fewer intervals: FP64 is ~1 TFLOP/s on B300)
    fp64 = None
    if args.fp64_steps > 0:
        s64 = make_sampler(run, ts, x0, C0, dm.FP64, stream=stream.cuda_stream)
        s64.run(run.n_lag)
        dt64 = time_intervals(s64, run.n_lag, args.fp64_steps, torch, stream)
        fp64 = {"value": round(N * args.fp64_steps / dt64, 1), "unit": "chain-steps/s",
                "ms_per_step": round(dt64 / args.fp64_steps * 1e3, 2), "steps": args.fp64_steps}
        s64.close()
        del s64

    # ---- end to end through the public API with host buffers: init (target + start state uploaded from
    # host memory), K intervals each followed by a read of log pi, then the pooled moments read back
    e2e = None
    if not args.no_e2e:
        torch.cuda.synchronize()
        t0 = time.time()
        se = make_sampler(run, ts, x0, C0, dm.BF16, stream=stream.cuda_stream)
        for _ in range(args.steps):
            se.run(run.n_lag)
            se.log_pi()
        m, cov, n = se.moments()
        torch.cuda.synchronize()
        te = time.time() - t0
        se.close()
        h2d = (ts.A.nbytes + ts.y.nbytes + ts.lam.nbytes + x0.nbytes + C0.nbytes)
        d2h_final = m.nbytes + cov.nbytes
        e2e = {"value": round(world * N * args.steps / te, 1), "unit": "chain-steps/s",
               "h2d_bytes_per_step": int(h2d / args.steps), "d2h_bytes_per_step": int(run.P * 8 + d2h_final / args.steps),
               "includes": "diam_init from host arrays, K intervals each with a log-pi read, final moments read"}

    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = cpu_leg(run, ts, x0, C0, args.cpu_seconds, cores)

    if rank == 0:
        line = {"metric": "chain-steps/s", "value": round(value, 1), "unit": "chain-steps/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 3),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
                "data": "synthetic", "config": config, "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": int(launches), "clocks": clk.summary(), "fp64_plain": fp64,
                "accept_rate": round(st["accepted"] / max(1, st["steps"] * run.P), 4), "refreshes": st["refreshes"],
                "chol_attempts": st["chol_attempts"]}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
