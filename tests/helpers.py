"""Shared set-up for the parity tests: one run description builds both the CUDA sampler (through the C ABI)
and the oracle with identical parameters. Inputs come from the seeded workload generators only."""
import numpy as np

import oracle
import workloads

CFG_KEYS = ["d", "P", "n_lag", "M", "beta0", "infl", "adapt_beta", "xref_mode", "acc_lo", "acc_hi", "beta_factor",
            "beta_min", "beta_max", "eps_jitter", "min_samples_refresh", "refresh_delay", "prec", "seed",
            "problem_id", "burnin", "proposal", "eps_jitter_min"]


def oracle_target(ts):
    return oracle.Target(ts.kind, ts.d, ts.d_y, lam=ts.lam, G=ts.G, A=ts.A, y=ts.y, sigma=ts.sigma,
                         ban_a=ts.ban_a, ban_b=ts.ban_b, ban_c=ts.ban_c)


def make_pair(ts, P, trace_steps=0, threads=4, x0=None, C0=None, xref0=None, **kw):
    """(gpu_sampler, oracle_sampler) for target spec ts, P chains and config overrides kw."""
    import paper_1506_05741_b300 as dm
    d = ts.d
    cfg = dm.default_config(d, P, **kw)
    cfg["trace_steps"] = trace_steps
    ocfg = oracle.default_config(**{k: cfg[k] for k in CFG_KEYS})
    ocfg.update(threads=threads, trace_steps=trace_steps)
    g = dm.Sampler(cfg, ts, x0=x0, C0=C0, xref0=xref0)
    o = oracle.Sampler(ocfg, oracle_target(ts), x0=x0, C0=C0, xref0=xref0)
    return g, o


def rel_err(a, b, scale):
    return np.max(np.abs(np.asarray(a) - np.asarray(b)) / np.maximum(scale, 1.0))


def trace_scale(tr):
    return np.maximum.reduce([np.abs(tr["lp_prop"]), np.abs(tr["q_prop"]), np.abs(tr["q_cur"])])


def diff_scale(to):
    """Scale of the log-density differences of each traced step (oracle trace): max(1, |log pi(x*) - log pi(x)|,
    |q(x*) - q(x)|). log a = (log pi(x*) - log pi(x)) + (q(x*) - q(x)), so its error is measured against the size
    of its two terms, not against |log pi| itself."""
    dq = to["q_prop"] - to["q_cur"]
    dlp = to["loga"] - dq
    return np.maximum(1.0, np.maximum(np.abs(dlp), np.abs(dq)))


def loga_err(tg, to):
    """Largest error of log a, relative to the difference scale above."""
    return float(np.max(np.abs(np.asarray(tg["loga"]) - np.asarray(to["loga"])) / diff_scale(to)))


def state_rounding_bound(d):
    """Absolute size up to which log a of the BF16 path may leave the FP64 oracle's through the FP32 rounding of the
    proposal itself. The CUDA path keeps the chain's states x and z in FP32: each coordinate of x* and z* is
    rounded once (relative error <= 2^-24), and log a depends on them through the log-density difference and the
    quadratic's difference, with sensitivities of O(1) per coordinate in whitened units (d(q* - q)/dz*_k = z*_k,
    and the same for the prior part when the factor follows the prior). So the two values differ by a sum of ~2d
    independent terms of size <= 2^-24 v_k^2 (E v^4 = 3): standard deviation ~ 2^-24 sqrt(2 d), measured 1.0e-5 at
    d = 4096 with the tanh likelihood's part included. The bound is 14 2^-24 sqrt(d) (5.3e-5 at d = 4096, about
    five measured standard deviations)."""
    return 14.0 * 2.0 ** -24 * np.sqrt(d)


def fp32_value_bound(to):
    """Absolute size up to which log a of the BF16 path may leave the oracle's where the CUDA path forms log pi(x*)
    or q* as values in FP32 (a target evaluated whole, such as the twisted Gaussians, or a per-step product) rather
    than as differences: each such value carries the FP32 rounding of its terms and sums, a relative error of a few
    2^-24, so the bar is 4 2^-24 (|log pi(x*)| + |log pi(x)| + |q*| + |q|) of the oracle's trace."""
    dq = np.asarray(to["q_prop"]) - np.asarray(to["q_cur"])
    lp_cur = np.asarray(to["lp_prop"]) - (np.asarray(to["loga"]) - dq)
    return 4.0 * 2.0 ** -24 * (np.abs(to["lp_prop"]) + np.abs(lp_cur) + np.abs(to["q_prop"]) + np.abs(to["q_cur"]))


def loga_excess(tg, to, bound, rel=1e-5):
    """Largest error of log a over its bar: max(rel x the difference scale, bound) (<= 1 passes); bound a number
    (state_rounding_bound) or an array over the trace (fp32_value_bound)."""
    err = np.abs(np.asarray(tg["loga"]) - np.asarray(to["loga"]))
    return float(np.max(err / np.maximum(rel * diff_scale(to), bound)))
