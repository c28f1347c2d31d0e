"""Benchmark of the DIAM hot path on one B300 (or N replicas under torchrun).

Workload (tanh4096): Bayesian tanh regression, d = 4096, d_y = 2048, prior N(0, diag(i^-2)), A (2048 x 4096)
N(0, 1/4096) in FP32, y = tanh(A x*) + 0.05 eps; P = 512 chains, n_lag = 128. A_0 = Cholesky of the prior
covariance, x_0 drawn from the prior. One benchmark step = one interval of n_lag steps of all P chains
(noise product, n_lag x (propose, screen, target, accept), moment fold, beta rule and the Cholesky refresh
that is due every interval). With --refresh-delay D >= 1 (the paper's lag-time between a refresh and its use,
Sec. "Computational introduction"; default D = 2, a lag of 2 n_lag = 256 steps at d = 4096) the factor built
from interval k's moments drives interval k + 1 + D and its Cholesky runs on its own streams beside the
following intervals (two at a time for D >= 2); the timed region still holds the K intervals' K refreshes.
Arms, same workload and start:
  mixed_da  (the headline value): BF16 factor / noise / map on the tensor cores, FP32 states, FP64-accurate
            refresh and moment fold, plus delayed acceptance with the MLP surrogate 4096 -> 512 -> 512 -> 1
            trained on the GPU (first training once 2e4 exactly evaluated pairs are in the 2e5-pair ring,
            then every 20 synchronisations; stage 1 off while the held-out RMSE exceeds 0.5 nats);
  mixed     the same without the surrogate;
  mixed_da_delay1    the headline arm with refresh_delay 1 (one factorisation beside the next interval);
  mixed_da_in_order  the headline arm with refresh_delay 0 (each factor used right after its refresh);
  mixed_tf32 the mixed arm with the factor quantised to TF32 instead of BF16 (prec FP32, no surrogate);
  fp64      the plain FP64 form (every kernel FP64, DFMA Cholesky).
Metrics: chain-steps/s = P n_lag / device time of an interval (everything above included), and min-ESS/s =
min over coordinates of the batch-means effective sample size of the ESS window (batches of b intervals of
one chain, b doubling while 4 batches per chain remain) / the window's device time.

Prints one JSON line (rank 0). --impl reference times the CPU oracle (the reference arm: a plain FP64 CPU program).
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
OZ_PRODUCTS = 28          # BF16 slice products per FP64 product in the Ozaki-split updates (7 slices, a + b <= 6)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=32, help="timed intervals (of n_lag steps each) of the headline arm")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--P", type=int, default=512)
    ap.add_argument("--n-lag", type=int, default=128)
    ap.add_argument("--no-da", action="store_true", help="headline arm without the surrogate")
    ap.add_argument("--refresh-delay", type=int, default=2,
                    help="interval k's factor drives interval k+1+delay (>= 1: its Cholesky runs beside interval k+1)")
    ap.add_argument("--in-order-steps", type=int, default=-1,
                    help="timed intervals of the headline arm with refresh_delay 0 and 1 (-1: --steps, 0: skip)")
    ap.add_argument("--mixed-steps", type=int, default=-1, help="timed intervals of the mixed arm (-1: --steps, 0: skip)")
    ap.add_argument("--fp64-steps", type=int, default=2, help="timed intervals of the plain FP64 arm (0: skip)")
    ap.add_argument("--tf32-steps", type=int, default=8,
                    help="timed intervals of the mixed arm with the factor quantised to TF32 (prec FP32; 0: skip)")
    ap.add_argument("--fp64-warmup", type=int, default=-1, help="-1: the headline arm's warm-up (the same burn-in)")
    ap.add_argument("--ess-intervals", type=int, default=192,
                    help="intervals of the headline arm's ESS window (the timed intervals, continued)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline")
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-profile", action="store_true", help="skip the per-phase profile pass (roofline)")
    ap.add_argument("--convergence", action="store_true",
                    help="instead of the throughput bench: samples and device time to convergence on a dense Gaussian "
                         "of known covariance, over n_lag (Sec. 3.3)")
    ap.add_argument("--conv-ds", default="100,200,400", help="dimensions of the n_lag experiment")
    ap.add_argument("--conv-target", default="pi1", choices=["pi1", "dense"])
    ap.add_argument("--conv-P", type=int, default=64)
    ap.add_argument("--conv-tol-mean", type=float, default=0.01, help="|m_n - mu|_2 (the n_lag tuning criterion)")
    ap.add_argument("--conv-tol-cov", type=float, default=1e-3, help="|C_n - Sigma|_F / |Sigma|_F")
    ap.add_argument("--conv-max-s", type=float, default=25.0, help="device seconds per (d, n_lag) row at most")
    ap.add_argument("--config2", action="store_true",
                    help="instead of the throughput bench: the dense d=1024 multi-chain workload, 50 batches of 10 "
                         "intervals, in the FP64, FP32 and BF16 modes (moment errors and chain-steps/s)")
    ap.add_argument("--c2-modes", default="fp64,fp32,bf16")
    ap.add_argument("--c2-batches", type=int, default=50)
    ap.add_argument("--compare", action="store_true",
                    help="instead of the throughput bench: integrated autocorrelation times of DIAM, AM, pCN and RW on "
                         "the Gaussian test targets of Sec. 3.1 over d (Sec. 3.2)")
    ap.add_argument("--cmp-d", default="32,64,128,256")
    ap.add_argument("--cmp-targets", default="1,2,4")
    ap.add_argument("--cmp-intervals", type=int, default=3000, help="measured intervals (n_lag = d / 2 steps each)")
    ap.add_argument("--cmp-warmup", type=int, default=3000, help="adaptation intervals before the window")
    ap.add_argument("--cmp-prec", default="bf16", choices=["bf16", "fp64"])
    ap.add_argument("--multi", action="store_true",
                    help="instead of the throughput bench: the uneven batch of 64 problems (d log-uniform in [256, 8192], "
                         "dense Gaussians and bananas, P = 32, n_lag = 64, BF16) at its full size")
    ap.add_argument("--da-gain", action="store_true",
                    help="instead of the throughput bench: delayed acceptance with and without the surrogate on the tanh "
                         "regression with an expensive exact target (map carried off), over d")
    ap.add_argument("--dag-ds", default="256,512,1024,2048,4096")
    ap.add_argument("--dag-warmup", type=int, default=50)
    ap.add_argument("--dag-steps", type=int, default=48)
    ap.add_argument("--multi-n", type=int, default=64)
    ap.add_argument("--multi-warmup", type=int, default=48,
                    help="warm-up intervals of --multi: from x_0 = 0 and A_0 = Id the step size must first adapt down "
                         "(about 30 intervals) before moves are accepted and the refreshes start")
    ap.add_argument("--multi-steps", type=int, default=16, help="timed intervals of --multi")
    ap.add_argument("--multi-delay", type=int, default=0,
                    help="refresh_delay of every problem (measured: 0 gives 1.16 M chain-steps/s, 2 gives 0.88 M: with "
                         "64 problems the streams already overlap, and three more per problem only add contention)")
    return ap.parse_args()


def multi(args):
    """The uneven batch: 64 independent problems, d_j = round(exp(U(ln 256, ln 8192))) (seed 7), even j the dense
    Gaussian Sigma = Q diag(1/i) Q^T (Q from QR of a seeded N(0,1) matrix, seed 7000 + j), odd j the banana with
    lambda_i = 1/i; each P = 32 chains, n_lag = 64, BF16 mode, x_0 = 0, A_0 = Id, refresh every interval (once
    d + 1 moves are accepted; refresh_delay --multi-delay), run together through diam_multi_run. --multi-warmup intervals (the step size adapts
    down first), then --multi-steps timed (wall clock with the device synchronised on both sides, the problems'
    streams run concurrently); aggregate chain-steps/s = sum_j P n_lag K / time; per problem the acceptance rate
    and refreshes of the timed window. One JSON line."""
    import torch
    import paper_1506_05741_b300 as dm
    import workloads
    t0 = time.time()
    specs = workloads.multi64(args.multi_n, with_cov=False)
    gen_s = time.time() - t0
    cfgs = [dm.default_config(r.target.d, r.P, n_lag=r.n_lag, beta0=r.beta0, seed=r.seed, problem_id=j, prec=dm.BF16,
                              refresh_delay=args.multi_delay)
            for j, r in enumerate(specs)]
    t1 = time.time()
    m = dm.MultiSampler(cfgs, [r.target for r in specs])
    init_s = time.time() - t1
    nl = specs[0].n_lag
    m.run(args.multi_warmup * nl)
    torch.cuda.synchronize()
    st0 = [v.stats() for v in m.views]
    t2 = time.time()
    m.run(args.multi_steps * nl)
    torch.cuda.synchronize()
    dt = time.time() - t2
    steps = sum(r.P for r in specs) * nl * args.multi_steps
    per = []
    for j, r in enumerate(specs):   # over the timed window
        st = m.views[j].stats()
        acc = st["accepted"] - st0[j]["accepted"]
        per.append({"j": j, "d": r.target.d, "kind": "dense" if j % 2 == 0 else "banana",
                    "accept_rate": round(acc / max(1, (st["steps"] - st0[j]["steps"]) * r.P), 3),
                    "refreshes": st["refreshes"] - st0[j]["refreshes"], "beta": round(st["beta"], 4)})
    m.close()
    ds = [r.target.d for r in specs]
    print(json.dumps({"metric": "aggregate chain-steps/s, uneven batch of problems", "value": round(steps / dt, 1),
                      "unit": "chain-steps/s", "timed_intervals": args.multi_steps, "warmup_intervals": args.multi_warmup,
                      "seconds": round(dt, 3), "ms_per_interval": round(dt / args.multi_steps * 1e3, 2),
                      "config": {"workload": f"multi{len(specs)}: d log-uniform in [256, 8192] (seed 7), even j dense "
                                             f"Gaussian, odd j banana, P=32, n_lag=64, BF16, refresh every interval, "
                                             f"refresh_delay {args.multi_delay}",
                                 "problems": len(specs), "d_min": int(min(ds)), "d_max": int(max(ds)),
                                 "sum_d": int(sum(ds)), "timing": "wall clock, device synchronised on both sides"},
                      "generate_s": round(gen_s, 1), "init_s": round(init_s, 1), "problems": per}), flush=True)


# Sec. 3.2's four samplers on the library's kernels: proposal (0 = DIAM's eq. (diam), 1 = the random walk of eq.
# (rw)), whether the factor adapts (refresh from the pooled moments, A_0 = Id, x_ref the running mean for DIAM) or
# stays the prior's Id (pCN, eq. (pcn), and RW), and the acceptance window the step size is adapted to (0.3-0.5 for
# DIAM and pCN, 0.1-0.3 for AM and RW).
SAMPLERS = {
    "DIAM": dict(proposal=0, adapt=True, acc=(0.3, 0.5)),
    "AM": dict(proposal=1, adapt=True, acc=(0.1, 0.3)),
    "pCN": dict(proposal=0, adapt=False, acc=(0.3, 0.5)),
    "RW": dict(proposal=1, adapt=False, acc=(0.1, 0.3)),
}


def iact_batch_means(bsum, n_lag, f_var, bmax):
    """IACT of a functional from its per-interval, per-chain sums bsum (K, P): with batches of b intervals,
    tau_b = b n_lag var(batch means) / var(f), var(f) known exactly; returns {b: tau_b} for b = 1, 2, 4, ..."""
    K, P = bsum.shape
    out = {}
    b = 1
    while b <= bmax and K // b >= 4:
        nb = K // b
        bm = bsum[: nb * b].reshape(nb, b, P).sum(axis=1) / (b * n_lag)
        mu = bm.mean()
        out[b] = float(b * n_lag * ((bm - mu) ** 2).sum() / (bm.size - 1) / f_var)
        b *= 2
    return out


def compare(args):
    """Sec. 3.2 on the GPU: integrated autocorrelation times of log pi, v_d^T x (the direction of the largest
    variance) and v_1^T x (the smallest) for DIAM, AM, pCN and RW on pi_1, pi_2, pi_4 of Sec. 3.1, over d. BF16
    mode (or FP64 with --cmp-prec fp64), P = 32 chains started from exact draws of the target, n_lag = d / 2 (the paper's choice), beta_0 =
    2.4 / sqrt(d) adapted to each sampler's acceptance window; the adaptive samplers keep their first 20
    intervals out of the moments (n_0 of Algorithm 1's footnote) and refresh after 5 d accepted moves. The IACT is
    read off batch means of per-interval chain sums (batches of b intervals, b doubling; var(f) exact: d/2 for log pi
    of a Gaussian, the eigenvalue for v^T x); 'tau' is the value at the largest b with at least 4 batches per chain,
    'plateau' whether the last doubling changed it by less than 20%. One JSON line."""
    import torch
    import paper_1506_05741_b300 as dm
    import workloads
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    P = 32
    rows = []
    for d in [int(v) for v in args.cmp_d.split(",")]:
        nl = max(2, d // 2)
        targets = workloads.paper_targets(d)
        for j in [int(v) for v in args.cmp_targets.split(",")]:
            ts = targets[j]
            ev, V = np.linalg.eigh(ts.cov)
            x0 = workloads.start_state(d, P, 11) @ np.linalg.cholesky(ts.cov).T
            for name, sp in SAMPLERS.items():
                cfg = dm.default_config(d, P, n_lag=nl, seed=100 + d + j, proposal=sp["proposal"], acc_lo=sp["acc"][0],
                                        acc_hi=sp["acc"][1], prec=dm.BF16 if args.cmp_prec == "bf16" else dm.FP64)
                if sp["adapt"]:
                    cfg.update(burnin=20 * nl, min_samples_refresh=5 * d)
                else:
                    cfg.update(min_samples_refresh=10 ** 15, xref_mode=0)
                cfg["keep_block_sums"] = 1
                t0 = time.time()
                s = dm.Sampler(cfg, ts, x0=x0, stream=stream.cuda_stream)
                W, K = args.cmp_warmup, args.cmp_intervals
                s.run((W + K) * nl)
                xs, ls = s.block_sums(W + K)
                st = s.stats()
                s.close()
                xs, ls = xs[W:], ls[W:]
                funcs = {"log_pi": (ls, d / 2.0), "v_d": (xs @ V[:, -1], ev[-1]), "v_1": (xs @ V[:, 0], ev[0])}
                res = {}
                for fname, (bs, var) in funcs.items():
                    taus = iact_batch_means(bs, nl, var, bmax=K // 4)
                    bl = sorted(taus)
                    tau = taus[bl[-1]]
                    res[fname] = {"tau": round(tau, 2), "plateau": bool(len(bl) > 1 and abs(tau / taus[bl[-2]] - 1) < 0.2),
                                  "by_batch_intervals": {str(b): round(v, 2) for b, v in taus.items()}}
                row = {"d": d, "target": f"pi_{j}", "sampler": name, "n_lag": nl,
                       "accept_rate": round(st["accepted"] / max(1, st["steps"] * P), 3), "beta": round(st["beta"], 4),
                       "refreshes": st["refreshes"], "iact": res, "seconds": round(time.time() - t0, 2)}
                rows.append(row)
                print(json.dumps({k: row[k] for k in ("d", "target", "sampler", "accept_rate", "beta")} |
                                 {f: res[f]["tau"] for f in res}), file=sys.stderr, flush=True)
    print(json.dumps({"metric": "integrated autocorrelation time (steps) of DIAM, AM, pCN, RW (Sec. 3.2)",
                      "config": {"P": P, "n_lag": "d/2", "prec": args.cmp_prec.upper(), "warmup_intervals": args.cmp_warmup,
                                 "intervals": args.cmp_intervals, "start": "exact draws of the target"},
                      "rows": rows}), flush=True)


def da_gain(args):
    """Delayed acceptance where the exact target is expensive: the tanh regression with the map carried off
    (carry_map 0), so every exact log-density is a d_y x d product per chain-step on the tensor cores, against the
    screen's 2 (d h + h^2) (h = the hidden width). For each d in --dag-ds (d_y = d / 2, prior N(0, diag(i^-2)),
    P = 256 chains, n_lag = 64, BF16 mode, refresh every interval), the same chains from the same start with and
    without the surrogate: --dag-warmup intervals of burn-in (the surrogate trained every 2 intervals once 4 intervals
    of pairs are in), then --dag-steps timed intervals and the ESS over them, in which it retrains on its own
    schedule (every 20 synchronisations of M = 2 intervals) with the real 0.5-nat gate deciding whether stage 1
    runs. Per d: device ms per interval, acceptance, min-ESS/s, and the screen's state (trainings,
    held-out RMSE, active, stage-1 pass rate, exact evaluations per chain-step). One JSON line."""
    import torch
    import paper_1506_05741_b300 as dm
    import workloads
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    P, nl = 256, 64
    rows = []
    for d in [int(v) for v in args.dag_ds.split(",")]:
        ts = workloads.tanh_regression(d, d // 2, 2000 + d)
        x0 = workloads.start_state(d, P, 5) * np.sqrt(ts.lam)
        C0 = np.diag(ts.lam)
        h = min(512, max(128, (d // 2) // 128 * 128))
        for use in (False, True):
            cfg = dm.default_config(d, P, n_lag=nl, M=2, beta0=min(2.4 / np.sqrt(d), 0.5), seed=41, prec=dm.BF16,
                                    carry_map=0, refresh_delay=0)
            cfg["keep_block_sums"] = 1
            s = dm.Sampler(cfg, ts, x0=x0, C0=C0, stream=stream.cuda_stream)
            if use:
                dc = dm.da_default_config(h1=h, h2=h, first_train_min=4 * P * nl)
                s.da_enable(dc, workloads.mlp_init(d, h, h, seed=11))
            W, K = args.dag_warmup, args.dag_steps
            if use:   # burn-in: 4 intervals of pairs, then a training every 2 intervals (diam_da_train)
                s.run(4 * nl)
                for _ in range((W - 4) // 2):
                    s.da_train()
                    s.run(2 * nl)
                s.run(((W - 4) % 2) * nl)
            else:
                s.run(W * nl)
            mom0 = s.export_moments()
            st0 = s.stats()
            d0 = s.da_stats() if use else None
            dt = time_intervals(s, nl, K, torch, stream)
            mom1 = s.export_moments()
            xs, _ = s.block_sums(W + K)
            table, (min_ess, _, _), plateau, N = ess_sweep(xs[W:W + K], nl, mom0, mom1)
            st = s.stats()
            row = {"d": d, "d_y": d // 2, "surrogate": use, "ms_per_interval": round(dt / K * 1e3, 3),
                   "chain_steps_per_s": round(P * nl * K / dt, 1),
                   "accept_rate": round((st["accepted"] - st0["accepted"]) / max(1, (st["steps"] - st0["steps"]) * P), 4),
                   "min_ess": round(min_ess, 1), "min_ess_per_s": round(min_ess / dt, 2), "ess_plateau": plateau}
            if use:
                ds = s.da_stats()
                tested = ds["stage1_tested"] - d0["stage1_tested"]
                row["da"] = {"hidden": h, "trainings": ds["trainings"], "last_rmse_nats": round(ds["last_rmse"], 3),
                             "active_at_end": ds["active"],
                             "stage1_pass_rate": round((ds["stage1_passed"] - d0["stage1_passed"]) / tested, 4) if tested else None,
                             "exact_evals_per_chain_step": round((ds["exact_evals"] - d0["exact_evals"]) / (K * nl * P), 4)}
            s.close()
            rows.append(row)
            print(json.dumps(row), file=sys.stderr, flush=True)
    print(json.dumps({"metric": "delayed acceptance on an expensive exact target: ms per interval and min-ESS/s with and "
                                "without the surrogate screen",
                      "config": {"workload": "tanh regression, map carried off (a d_y x d product per exact evaluation), "
                                             "P=256, n_lag=64, BF16, refresh every interval, rmse_bound 0.5",
                                 "warmup_intervals": args.dag_warmup, "timed_intervals": args.dag_steps},
                      "rows": rows}), flush=True)


def convergence(args):
    """Sec. 3.3's n_lag experiment on the GPU sampler. Target pi_1 = N(0, (A A^T + I)^-1) of Sec. 3.1 (or, with
    --conv-target dense, N(0, Q diag(1/i) Q^T)) for each d in --conv-ds; chains started from N(0, I) (Algorithm 1's
    x_0); for n_lag in {d/100, d/10, d/4, d/2, d, 2d, 4d, 10d}, the chain-steps (P x steps) and device time until
    the pooled mean is within tol_mean of the truth in the Euclidean norm (the paper's criterion for tuning n_lag,
    TOL = 0.01) and until the pooled covariance is within tol_cov of Sigma in the relative Frobenius norm (its
    stopping criterion elsewhere, TOL = 1e-3), each row capped at --conv-max-s device seconds. The samples to the
    mean criterion are also given relative to n_lag = d, the normalisation of the paper's figure. BF16 mode,
    refresh in order (refresh_delay 0). One JSON line."""
    import torch
    import paper_1506_05741_b300 as dm
    import workloads
    P = args.conv_P
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    out = []
    for d in [int(v) for v in args.conv_ds.split(",")]:
        ts = workloads.paper_targets(d)[1] if args.conv_target == "pi1" else workloads.dense_gaussian(d, 1000 + d)
        nS = float(np.linalg.norm(ts.cov))
        x0 = workloads.start_state(d, P, 3)
        rows = []
        for frac in (0.01, 0.1, 0.25, 0.5, 1.0, 2.0, 4.0, 10.0):
            nl = max(1, int(round(frac * d)))
            cfg = dm.default_config(d, P, n_lag=nl, seed=17, prec=dm.BF16, refresh_delay=0)
            s = dm.Sampler(cfg, ts, x0=x0, stream=stream.cuda_stream)
            chunk = max(nl, (2048 // nl) * nl)   # whole intervals, about 2048 steps a check
            steps, dev_s = 0, 0.0
            hit = {"mean": None, "cov": None}
            while dev_s < args.conv_max_s and (hit["mean"] is None or hit["cov"] is None):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                s.run(chunk)
                e1.record(stream)
                torch.cuda.synchronize()
                dev_s += e0.elapsed_time(e1) / 1e3
                steps += chunk
                m, C, n = s.moments()
                em = float(np.linalg.norm(m - ts.mean))
                ec = float(np.linalg.norm(C - ts.cov)) / nS
                for key, err, tol in (("mean", em, args.conv_tol_mean), ("cov", ec, args.conv_tol_cov)):
                    if hit[key] is None and err <= tol:
                        hit[key] = {"chain_steps": steps * P, "device_s": round(dev_s, 4), "error": round(err, 5)}
            st = s.stats()
            s.close()
            rows.append({"n_lag": nl, "n_lag_over_d": frac, "to_mean_tol": hit["mean"], "to_cov_tol": hit["cov"],
                         "steps_run": steps, "final_mean_error": round(em, 5), "final_cov_error": round(ec, 5),
                         "device_s": round(dev_s, 3), "accept_rate": round(st["accepted"] / max(1, st["steps"] * P), 4),
                         "beta": round(st["beta"], 4), "refreshes": st["refreshes"]})
            print(json.dumps({"d": d, "n_lag": nl, "done": rows[-1]}), file=sys.stderr, flush=True)
        base = next((r["to_mean_tol"] for r in rows if r["n_lag_over_d"] == 1.0), None)
        for r in rows:
            r["samples_to_mean_tol_over_n_lag_d"] = (round(r["to_mean_tol"]["chain_steps"] / base["chain_steps"], 3)
                                                     if r["to_mean_tol"] and base else None)
        out.append({"d": d, "rows": rows})
    print(json.dumps({"metric": "chain-steps and device seconds to convergence (Sec. 3.3, impact of n_lag)",
                      "config": {"workload": f"{'pi_1 of Sec. 3.1' if args.conv_target == 'pi1' else 'dense Gaussian'}"
                                             f", P={P}, BF16 mode, refresh in order, x_0 ~ N(0, I)",
                                 "tol_mean": args.conv_tol_mean, "tol_cov_rel_frobenius": args.conv_tol_cov,
                                 "max_device_s_per_row": args.conv_max_s},
                      "by_d": out}), flush=True)


def config2(args):
    """The dense d = 1024 workload as the paper's multi-chain setting runs it: Sigma = Q diag(1/i) Q^T (Q from the
    QR of a seeded N(0, 1) matrix), P = 128 chains, n_lag = 64, 50 batches of M = 10 intervals (32 000 steps per
    chain), A_0 = Id and x_0 ~ N(0, I) (Algorithm 1's start), beta adaptive, every interval's samples pooled into
    the factor (the batch of M intervals is the reporting unit). Run in the plain FP64 mode and in the FP32 mode
    (the factor quantised to TF32, tensor-core products, one launch per interval, graph-replayed refreshes), and
    in the BF16 mode for comparison. Per mode: chain-steps/s over the 50 batches (CUDA events on the sampler's
    stream, moments read between batches outside the timed spans), the moments' errors against Sigma at batch 1,
    5, 10, 25, 50 (mean: Euclidean; covariance: relative Frobenius), and the PSRF of the second half."""
    import torch
    import paper_1506_05741_b300 as dm
    import workloads
    run = workloads.dense1024()
    ts = run.target
    d, P, nl, M = ts.d, run.P, run.n_lag, run.M
    nS = float(np.linalg.norm(ts.cov))
    x0 = workloads.start_state(d, P, 3)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    modes = {"fp64": dm.FP64, "fp32": dm.FP32, "bf16": dm.BF16}
    out = {}
    for name in args.c2_modes.split(","):
        cfg = dm.default_config(d, P, n_lag=nl, beta0=run.beta0, seed=run.seed, prec=modes[name])
        cfg["keep_block_sums"] = 1
        s = dm.Sampler(cfg, ts, x0=x0, stream=stream.cuda_stream)
        dev_s, traj = 0.0, []
        for b in range(1, args.c2_batches + 1):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            s.run(M * nl)
            s.flush()
            e1.record(stream)
            torch.cuda.synchronize()
            dev_s += e0.elapsed_time(e1) / 1e3
            if b in (1, 5, 10, 25, 50) or b == args.c2_batches:
                m, C, n = s.moments()
                traj.append({"batch": b, "mean_error": round(float(np.linalg.norm(m - ts.mean)), 5),
                             "cov_error": round(float(np.linalg.norm(C - ts.cov)) / nS, 5)})
        st = s.stats()
        nb = args.c2_batches * M
        r = s.psrf(nb // 2, nb - nb // 2)
        s.close()
        steps = args.c2_batches * M * nl
        out[name] = {"chain_steps_per_s": round(steps * P / dev_s, 1), "device_s": round(dev_s, 3),
                     "moments": traj, "accept_rate": round(st["accepted"] / max(1, st["steps"] * P), 4),
                     "beta": round(st["beta"], 5), "refreshes": st["refreshes"],
                     "psrf_max_second_half": round(float(np.max(r)), 4)}
        print(json.dumps({"mode": name, "done": out[name]}), file=sys.stderr, flush=True)
    print(json.dumps({"metric": "chain-steps/s and moment errors, dense d=1024 multi-chain workload",
                      "unit": "chain-steps/s",
                      "config": {"workload": "dense1024: d=1024, Sigma = Q diag(1/i) Q^T, P=128, n_lag=64, "
                                             f"{args.c2_batches} batches of M={M} intervals, A_0 = Id, x_0 ~ N(0, I)",
                                 "moments": "pooled over all chains every interval"},
                      "data": "synthetic", "by_mode": out}), flush=True)


def peaks():
    try:
        with open(PEAKS_FILE) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 50 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "50"],
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


def make_sampler(run, ts, x0, C0, prec, da=False, profile=0, stream=None, keep_sums=0, delay=0):
    import paper_1506_05741_b300 as dm
    import workloads
    cfg = dm.default_config(ts.d, run.P, n_lag=run.n_lag, beta0=run.beta0, seed=run.seed, prec=prec, profile=profile,
                            refresh_delay=delay)
    cfg["keep_block_sums"] = keep_sums
    s = dm.Sampler(cfg, ts, x0=x0, C0=C0, stream=stream)
    if da:
        dc = dm.da_default_config()
        s.da_enable(dc, workloads.mlp_init(ts.d, dc["h1"], dc["h2"], seed=11))
    return s


def rank_max(x, world, device):
    """Max of x over the ranks (timings: the slowest replica sets the whole job's time)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.item()


def time_intervals(s, n_lag, K, torch, stream):
    """Device time of K intervals with CUDA events on the sampler's stream (synchronised on both sides). The
    region opens with every stream idle and closes after the last interval's refresh has finished (flush), so
    it holds exactly the K intervals' refreshes even when they run beside the following interval."""
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s.run(K * n_lag)
    s.flush()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3


def ess_window(xs, n_lag, mom0, mom1, b=1):
    """Batch-means ESS per coordinate over a window of K intervals (eq. (mse): N_eff = N / (1 + 2 Theta)): xs
    (K, P, d) per-interval, per-chain sums; mom0 / mom1 the pooled (mean, M2, n) at the window's ends. The
    window's variance comes from the moment difference (Chan et al.'s pairwise update run backwards); a batch is
    b consecutive intervals of one chain; ESS_i = N s_i^2 / (b n_lag var(batch means)_i), capped at N."""
    (m0, M20, n0), (m1, M21, n1) = mom0, mom1
    N = n1 - n0
    mw = (n1 * m1 - n0 * m0) / N
    delta = mw - m0
    m2w = np.diag(M21) - np.diag(M20) - delta * delta * (n0 * N / n1)
    var = m2w / (N - 1)
    K = xs.shape[0] // b * b
    bm = xs[:K].reshape(K // b, b, *xs.shape[1:]).sum(axis=1) / float(b * n_lag)
    nbm = bm.shape[0] * bm.shape[1]
    vbm = ((bm - mw) ** 2).sum(axis=(0, 1)) / (nbm - 1)
    ess = np.minimum(float(N), N * var / (b * n_lag * np.maximum(vbm, 1e-300)))
    return ess, N


def ess_sweep(xs, n_lag, mom0, mom1):
    """min-ESS over the window for batches of b = 1, 2, 4, ... intervals (at least 4 batches per chain). Batch
    means estimate the IACT only once a batch is much longer than it: the estimate falls as b grows until it
    levels off. Returns the table, the value at the largest b, and whether the last doubling moved it by less
    than 20% (plateau)."""
    K = xs.shape[0]
    table, b, last = {}, 1, None
    while b == 1 or K // b >= 4:   # b = 1 always (a short window has no longer batches)
        ess, N = ess_window(xs, n_lag, mom0, mom1, b)
        table[b] = (float(ess.min()), int(np.argmin(ess)), float(np.median(ess)))
        last = b
        b *= 2
    bl = sorted(table)
    plateau = len(bl) > 1 and abs(table[bl[-1]][0] / table[bl[-2]][0] - 1.0) < 0.2
    return table, table[last], plateau, N


def run_arm(name, run, ts, x0, C0, prec, da, W, K, torch, stream, dm, clocks_index=None, delay=0, K_ess=0):
    """W warm-up intervals, then K timed intervals (chain-steps/s), then, with K_ess > K, the same sampler on to
    K_ess intervals in all, timed too: the ESS window is the K_ess intervals after the warm-up (a batch-size sweep
    needs a window many batches long), min-ESS/s its min-ESS over its device time."""
    s = make_sampler(run, ts, x0, C0, prec, da=da, stream=stream.cuda_stream, keep_sums=1, delay=delay)
    s.run(W * run.n_lag)
    s.profile(reset=True)
    mom0 = s.export_moments()
    l0 = dm.kernel_launches()
    clk = None
    if clocks_index is not None:
        with ClockSampler(clocks_index) as clk:
            dt = time_intervals(s, run.n_lag, K, torch, stream)
    else:
        dt = time_intervals(s, run.n_lag, K, torch, stream)
    launches = dm.kernel_launches() - l0
    Ke = max(K, K_ess)
    dt_ess = dt + (time_intervals(s, run.n_lag, Ke - K, torch, stream) if Ke > K else 0.0)
    mom1 = s.export_moments()
    xs, _ = s.block_sums(W + Ke)
    table, (min_ess, argmin, med), plateau, N = ess_sweep(xs[W:W + Ke], run.n_lag, mom0, mom1)
    bmax = max(table)
    rhat = s.psrf(W, Ke) if run.P > 1 else None   # Sec. 2.4.2 over the ESS window
    st = s.stats()
    rf_cnt, rf_ms = s.profile()["refresh"]
    out = {"chain_steps_per_s": round(run.P * run.n_lag * K / dt, 1), "ms_per_step": round(dt / K * 1e3, 3),
           "timed_intervals": K, "warmup_intervals": W,
           "ess_window_intervals": Ke, "ess_window_s": round(dt_ess, 4), "ess_batch_intervals": bmax,
           "ess_plateau": plateau, "min_ess": round(min_ess, 1), "min_ess_per_s": round(min_ess / dt_ess, 2),
           "median_ess_per_s": round(med / dt_ess, 1), "min_ess_per_chain_step": round(min_ess / N, 6),
           "min_ess_by_batch_intervals": {str(b): round(v[0], 1) for b, v in sorted(table.items())},
           "argmin_coordinate": argmin, "window_samples": int(N),
           "accept_rate": round(st["accepted"] / max(1, st["steps"] * run.P), 4), "beta": round(st["beta"], 5),
           "refreshes": st["refreshes"], "chol_attempts": st["chol_attempts"]}
    if rhat is not None:
        out["psrf_max"] = round(float(rhat.max()), 4)
        out["psrf_frac_within_0.2"] = round(float(np.mean(rhat - 1.0 <= 0.2)), 4)
    if Ke < 8:   # too short for batches of several intervals: no ESS claim
        out["ess_note"] = "window too short for a batch-size sweep; ESS not claimed"
    if rf_cnt:   # refreshes factorised beside the following interval: their device time there
        out["refresh_beside_ms"] = round(rf_ms / rf_cnt, 3)
    if da:
        dst = s.da_stats()
        out["da"] = {"trainings": dst["trainings"], "active": int(dst["active"]),
                     "last_rmse_nats": round(dst["last_rmse"], 4),
                     "stage1_pass_rate": round(dst["stage1_passed"] / max(1, dst["stage1_tested"]), 4),
                     "exact_evals_per_step": round(dst["exact_evals"] / max(1, st["steps"] * run.P), 4)}
    s.close()
    return out, dt, launches, clk


def roofline(prof, run, ts, pk, pk_src, ring):
    """Per-phase achieved rate against its bound, from the profiled intervals; the dominant phase first."""
    d, dy, P, nl = ts.d, ts.d_y, run.P, run.n_lag
    # the interval kernel (one launch walks every chain through the interval's n_lag steps): per step it reads
    # the chain's xi (FP32), W (BF16) and A xi (FP32) rows and writes the FP32 record row and, with the
    # surrogate attached, the BF16 ring row; x, z and A x are read and written once per interval
    step_bytes = (nl * P * (d * (4 + 2 + 4) + dy * 4 + (d * 2 if ring else 0)) + 2 * P * (d * (4 + 4) + dy * 4))
    N = P * nl
    sus = pk.get("bf16_tflops_sustained", pk["bf16_tflops"])
    # algorithmic work per launch of each phase (a launch = one step, or one interval for noise / xi / fold /
    # refresh / rewhiten / train)
    work = {
        # the FP64 Cholesky: the method's own work, d^3 / 3 flops, against the pipe it runs on (the BF16 tensor
        # cores, FP64-accurate by the Ozaki split, around a serial FP64 chain of diagonal blocks); the slices'
        # overhead (28 BF16 products per FP64 product of the rank-64 updates) is reported beside it, not counted
        "refresh": ("tensor", d ** 3 / 3.0, "TFLOP/s", sus),
        # lower-triangular A_n W (2 d^2 N / 2) and the map of the noise, (A A_n) W (2 d_y d N; its lo pass, a
        # precision overhead, is not counted)
        "xi_gemm": ("tensor", float(d) * d * N + 2.0 * dy * d * N, "TFLOP/s", sus),
        # the fold apart from its SYRK: one pass over the interval's FP32 records (read) writing their BF16
        # transpose and tile sums (the per-chain interval sums of x ride along)
        "fold": ("hbm", N * d * (4 + 2), "GB/s", pk["hbm_gbs"]),
        "syrk": ("tensor", float(d) * (d + 1) * N, "TFLOP/s", sus),         # the fold's SYRK, lower half
        "target": ("tensor", 2.0 * dy * d * P * 2, "TFLOP/s", sus),          # A x* with the hi + lo split
        # bytes: propose reads x, z, xi (FP32), writes x*, z* (FP32) and the BF16 hi / lo split of x*
        "propose": ("hbm", P * d * (4 + 4 + 4 + 4 + 4 + 2 + 2), "GB/s", pk["hbm_gbs"]),
        # accept reads x*, z* and writes x, z and the FP32 record row
        "accept": ("hbm", P * d * (4 + 4 + 4 + 4 + 4), "GB/s", pk["hbm_gbs"]),
        "noise": ("hbm", N * d * 2, "GB/s", pk["hbm_gbs"]),                  # BF16 W for the interval
        # the triangular re-solve: its panel products issue 16 tensor-core columns per 4 chains (each chain's
        # solution split into 3 BF16 terms), 2 (d^2 / 2) 16 (P / 4) flops
        "rewhiten": ("tensor", 4.0 * d * d * P, "TFLOP/s", sus),
        "screen": ("tensor", 2.0 * P * (d * 512 + 512 * 512), "TFLOP/s", sus),
        "step": ("hbm", step_bytes, "GB/s", pk["hbm_gbs"]),
    }
    total = sum(ms for k, (_, ms) in prof.items() if k != "syrk") + prof.get("syrk", (0, 0.0))[1]
    table = {}
    for k, (cnt, ms) in prof.items():
        if cnt == 0 or k not in work:
            continue
        bound, units, unit, peak = work[k]
        per = ms / 1e3 / cnt
        ach = units / per / (1e12 if unit == "TFLOP/s" else 1e9)
        table[k] = {"share": round(ms / total, 4), "launch_ms": round(per * 1e3, 4), "bound": bound,
                    "achieved": round(ach, 3), "unit": unit, "peak": peak, "frac": round(ach / peak, 4)}
    # The dominant kernel of the launch list (profiles/launches_tanh4096_bf16.md): tc_gemm_persist_kernel, three
    # wide launches per interval -- the noise product (lower-triangular A_n W: d^2 N flops), its map ((A A_n) W:
    # 2 d_y d N; the lo pass of the two-term operand is a precision overhead, not counted) and the fold's SYRK
    # (lower half, d (d + 1) N). Achieved = their algorithmic flops over their CUDA-event time (phases xi_gemm
    # and syrk), per launch as the average of the three. The refresh is the largest phase but is ~250 launches of
    # three kernels (chol_diag_kernel, trsv_rows_kernel, ozaki_update_kernel), each a smaller share.
    (cx, mx), (cs, ms_) = prof.get("xi_gemm", (0, 0.0)), prof.get("syrk", (0, 0.0))
    if cx and cs:
        per_int = float(d) * d * N + 2.0 * dy * d * N + float(d) * (d + 1) * N
        t_int = (mx / cx + ms_ / cs) / 1e3          # seconds per interval of the three launches
        ach = per_int / t_int / 1e12
        out = {"kernel": "tc_gemm_persist_kernel (noise product, its map, fold SYRK: 3 launches per interval)",
               "bound": "tensor", "achieved": round(ach, 3), "peak": sus, "unit": "TFLOP/s",
               "frac": round(ach / sus, 4), "traffic": gemm_traffic(run, ts), "launch_ms": round(t_int * 1e3 / 3, 4),
               "flops_per_launch": round(per_int / 3), "peak_source": pk_src + " (sustained)", "phases": table}
    else:
        dom = max(table, key=lambda k: table[k]["share"])
        t = table[dom]
        out = {"kernel": dom, "bound": t["bound"], "achieved": t["achieved"], "peak": t["peak"], "unit": t["unit"],
               "frac": t["frac"], "traffic": None, "launch_ms": t["launch_ms"],
               "peak_source": pk_src + (" (sustained)" if t["bound"] == "tensor" else ""), "phases": table}
    if "refresh" in table:   # the slices' overhead, and the same work against the FP64 pipe's nominal rate
        r = table["refresh"]
        r["bf16_issued_tflops"] = round(r["achieved"] * OZ_PRODUCTS, 3)
        r["bf16_issued_note"] = "28 BF16 slice products per FP64 product of the rank-64 updates (Ozaki split)"
        r["fp64_nominal_tflops"] = FP64_PEAK_TFLOPS
        r["frac_of_fp64_nominal"] = round(r["achieved"] / FP64_PEAK_TFLOPS, 3)
    if "refresh" in table:
        out["refresh_note"] = ("the refresh phase: the FP64 Cholesky's d^3/3 flops over its device time, against the "
                               "sustained BF16 peak of the pipe it runs on; a latency-bound chain of 64 diagonal blocks, "
                               "beside the next intervals (refresh_delay 2) in the timed arms")
    return out


# DRAM traffic per launch of tc_gemm_persist_kernel in the benchmark's interval: dram__bytes_read.sum +
# dram__bytes_write.sum from one ncu capture of the benchmark itself (one pass per launch), averaged over the
# noise product (2.266 GB), its map (1.599 GB) and the fold's SYRK (1.272 GB) of one interval
# (profiles/tc_gemm_persist_tanh4096.md), with a digest of the kernel's sources when it was taken: reported only
# while the sources are unchanged.
GEMM_TRAFFIC = {"bytes": 1405800000, "sources_sha16": "99957cd82ff1bade"}


def gemm_traffic(run, ts):
    import hashlib
    h = hashlib.sha256()
    for f in ("tc_gemm.cu", "tc_common.cuh", "tc_gemm.h"):
        with open(os.path.join(ROOT, "paper_1506_05741_b300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    if GEMM_TRAFFIC["bytes"] is None or h.hexdigest()[:16] != GEMM_TRAFFIC["sources_sha16"]:
        return None
    return GEMM_TRAFFIC["bytes"]


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
            "sample": f"{steps} steps x {Ps} chains of tanh4096 (plain FP64 oracle, OpenMP over chains, no "
                      f"surrogate; refresh-free prefix: its amortised Cholesky is ~1.4% of the oracle's per-step "
                      f"work)", "steps_run": steps, "chains": Ps, "seconds": round(dt, 3)}


def main():
    args = parse()
    if args.convergence:
        convergence(args)
        return
    if args.compare:
        compare(args)
        return
    if args.multi:
        multi(args)
        return
    if args.da_gain:
        da_gain(args)
        return
    if args.config2:
        config2(args)
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    cores = os.cpu_count() or 1
    run, ts, x0, C0 = workload(args.P, args.n_lag)
    N = run.P * run.n_lag
    da = not args.no_da
    config = {"workload": f"tanh4096: d={ts.d}, d_y={ts.d_y}, P={run.P}, n_lag={run.n_lag}, BF16 factor/noise/map, "
                          f"FP32 states, FP64-accurate Cholesky refresh every interval"
                          + (f" (used from the interval {1 + args.refresh_delay} after; factorised beside the following ones)"
                             if args.refresh_delay > 0 else "")
                          + (", delayed acceptance with the 4096-512-512-1 MLP surrogate" if da else ""),
              "d": ts.d, "d_y": ts.d_y, "P": run.P, "n_lag": run.n_lag, "delayed_acceptance": da,
              "refresh_delay": args.refresh_delay,
              "step": "one interval: n_lag steps of all chains + moment fold + beta rule + Cholesky refresh",
              "l2": "inputs larger than L2 (per interval: BF16 noise 537 MB, noise product 1074 MB FP32)",
              "parallelism": f"replicas x{world} (chains independent; no data-path collective)"}
    metric = "chain-steps/s and min-ESS/s at d=4096, mixed-prec+DA vs plain FP64, one B300"

    if args.impl == "reference":
        if rank != 0:
            return
        t0 = time.time()
        leg = cpu_leg(run, ts, x0, C0, args.cpu_seconds, cores)
        line = {"impl": "reference", "metric": metric, "value": leg["value"], "unit": "chain-steps/s",
                "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config,
                "cpu_baseline": leg,
                "e2e": {"value": leg["value"], "unit": "chain-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
                # what was timed: leg["steps_run"] oracle steps of leg["chains"] chains (not an interval of P chains)
                "ms_per_step": round(leg["seconds"] / max(1, leg["steps_run"]) * 1e3, 3),
                "ms_per_step_means": f"wall time of one oracle step of {leg['chains']} chains",
                "wall_s": round(time.time() - t0, 2)}
        print(json.dumps(line), flush=True)
        return

    import torch
    import paper_1506_05741_b300 as dm
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    # one non-default stream for the samplers, their CUDA events and their graph replays
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    pk, pk_src = peaks()

    # ---- headline arm (every rank): mixed precision + delayed acceptance
    if world > 1:
        torch.distributed.barrier()
    head, dt, launches, clk = run_arm("mixed_da" if da else "mixed", run, ts, x0, C0, dm.BF16, da, args.warmup,
                                      args.steps, torch, stream, dm, clocks_index=local, delay=args.refresh_delay,
                                      K_ess=args.ess_intervals if rank == 0 else 0)
    dt = rank_max(dt, world, "cuda")
    value = world * N * args.steps / dt
    arms = {("mixed_da" if da else "mixed"): head}

    roof = fp64 = e2e = cpu = None
    if rank == 0:
        # ---- comparison arms on the same workload and start
        msteps = args.steps if args.mixed_steps < 0 else args.mixed_steps
        if da and msteps > 0:
            arms["mixed"], _, _, _ = run_arm("mixed", run, ts, x0, C0, dm.BF16, False, args.warmup, msteps, torch,
                                             stream, dm, delay=args.refresh_delay)
        isteps = args.steps if args.in_order_steps < 0 else args.in_order_steps
        for dly, suffix in ((1, "_delay1"), (0, "_in_order")):   # the same arm with shorter lags
            if dly < args.refresh_delay and isteps > 0:
                name = ("mixed_da" if da else "mixed") + suffix
                arms[name], _, _, _ = run_arm(name, run, ts, x0, C0, dm.BF16, da, args.warmup, isteps, torch, stream,
                                              dm, delay=dly)
        if args.tf32_steps > 0:   # the mixed mode with the factor quantised to TF32 (prec FP32), no surrogate
            arms["mixed_tf32"], _, _, _ = run_arm("mixed_tf32", run, ts, x0, C0, dm.FP32, False, args.warmup,
                                                  args.tf32_steps, torch, stream, dm, delay=args.refresh_delay)
        if args.fp64_steps > 0:
            fw = args.warmup if args.fp64_warmup < 0 else args.fp64_warmup
            arms["fp64"], _, _, _ = run_arm("fp64", run, ts, x0, C0, dm.FP64, False, fw, args.fp64_steps, torch,
                                            stream, dm, delay=args.refresh_delay)
            # the FP64 arm runs the same Markov chain (same proposal, factor rule and random streams; FP64 instead of
            # FP32 rounding), so its ESS per chain-step is the headline's: its min-ESS/s is its throughput times
            # that, and the ratio of the two arms' min-ESS/s is their throughput ratio
            f = arms["fp64"]
            f["min_ess_per_s_same_chain"] = round(f["chain_steps_per_s"] * head["min_ess_per_chain_step"], 2)

        # ---- profile pass: per-phase device time with CUDA events on the same stream
        if not args.no_profile:
            sp = make_sampler(run, ts, x0, C0, dm.BF16, da=da, profile=1, stream=stream.cuda_stream)
            sp.run(args.warmup * run.n_lag)
            sp.profile(reset=True)
            sp.run(max(2, args.steps // 2) * run.n_lag)
            prof = sp.profile()
            sp.close()
            roof = roofline(prof, run, ts, pk, pk_src, da)

        # ---- end to end through the public API with host buffers: init (target, start state and surrogate
        # weights uploaded from host memory), K intervals each followed by a read of log pi, then the pooled
        # moments read back
        if not args.no_e2e:
            torch.cuda.synchronize()
            t0 = time.time()
            se = make_sampler(run, ts, x0, C0, dm.BF16, da=da, stream=stream.cuda_stream, delay=args.refresh_delay)
            for _ in range(args.steps):
                se.run(run.n_lag)
                se.log_pi()
            m, cov, n = se.moments()
            torch.cuda.synchronize()
            te = time.time() - t0
            se.close()
            h2d = ts.A.nbytes + ts.y.nbytes + ts.lam.nbytes + x0.nbytes + C0.nbytes
            if da:
                h2d += 8 * (512 * ts.d + 512 + 512 * 512 + 512 + 512 + 1)
            d2h_final = m.nbytes + cov.nbytes
            e2e = {"value": round(N * args.steps / te, 1), "unit": "chain-steps/s",
                   "h2d_bytes_per_step": int(h2d / args.steps), "d2h_bytes_per_step": int(run.P * 8 + d2h_final / args.steps),
                   "includes": "diam_init from host arrays, K intervals each with a log-pi read, final moments read; refresh delay as the headline arm"}

        if not args.no_cpu:
            cpu = cpu_leg(run, ts, x0, C0, args.cpu_seconds, cores)

    if rank == 0:
        ess_ratio = None
        if "fp64" in arms and arms["fp64"].get("min_ess_per_s_same_chain", 0) > 0:
            ess_ratio = round(head["min_ess_per_s"] / arms["fp64"]["min_ess_per_s_same_chain"], 2)
        line = {"metric": metric, "value": round(value, 1), "unit": "chain-steps/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 3),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
                "data": "synthetic", "config": config, "min_ess_per_s": head["min_ess_per_s"],
                "min_ess_per_s_vs_fp64": ess_ratio, "arms": arms, "roofline": roof, "cpu_baseline": cpu,
                "e2e": e2e, "gpu_launches": int(launches), "clocks": clk.summary() if clk else None}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
