"""Parity at the sizes the benchmark runs: the tanh regression of the headline workload (d = 4096,
d_y = 2048, prior N(0, diag(i^-2)), A 2048 x 4096), in BF16 mode, through whole intervals, so that every step
runs in the one-launch interval kernel (one block walks its chain through the n_lag steps). The oracle runs
its BF16 mode on the same rounded factor, noise and map (FP64 states and sums), so the two agree to the level
of the CUDA path's FP32 states and sums.

Bars (Algorithm 1's test, eq. (accept)): identical accept decisions; log pi(x*) within 1e-5 of |log pi|; and
log a within 1e-5 of the size of its two terms, max(1, |log pi(x*) - log pi(x)|, |q(x*) - q(x)|) (the
log-density differences the test decides on), or within the FP32-state bound 14 2^-24 sqrt(d) where that is
larger (helpers.state_rounding_bound: the chain's x* and z* are FP32, one rounding per coordinate, while the
oracle's are FP64; measured standard deviation of the difference 1.0e-5 at d = 4096, 5.3e-5 bound).

The full-size case runs the benchmark's launch configuration (P = 512, n_lag = 128) and checks sampled chains
against the oracle run on those chains alone: with beta fixed and no refresh in the window the chains are
independent, and the oracle's chain0 field gives its chain p the random streams of chain chain0 + p.

The noise product and the fold's SYRK are also checked at their full shapes, M = K = 4096, N = 65536 and
M = N = 4096, K = 65536, against FP64 products of the same BF16 operands."""
import ctypes

import numpy as np
import pytest

import oracle
import workloads
from helpers import CFG_KEYS, diff_scale, loga_excess, oracle_target, state_rounding_bound

pytestmark = pytest.mark.gpu
TOL = 1e-5


def _headline(P, nl):
    run = workloads.tanh4096(P=P, n_lag=nl)
    ts = run.target
    x0 = workloads.start_state(ts.d, P, 1) * np.sqrt(ts.lam)   # the benchmark's start
    return run, ts, x0, np.diag(ts.lam)


def _gpu(run, ts, x0, C0, steps, profile=0, prec=None):
    import paper_1506_05741_b300 as dm
    cfg = dm.default_config(ts.d, run.P, n_lag=run.n_lag, beta0=run.beta0, seed=run.seed,
                            prec=dm.BF16 if prec is None else prec, adapt_beta=0, min_samples_refresh=10 ** 12,
                            profile=profile)
    cfg["trace_steps"] = steps
    g = dm.Sampler(cfg, ts, x0=x0, C0=C0)
    g.run(steps)
    return g, cfg


def _oracle(cfg, ts, x0, C0, steps, chain0, n):
    ocfg = oracle.default_config(**{k: cfg[k] for k in CFG_KEYS})
    ocfg.update(P=n, chain0=chain0, threads=n, trace_steps=steps)
    o = oracle.Sampler(ocfg, oracle_target(ts), x0=x0[chain0:chain0 + n], C0=C0)
    o.run(steps)
    return o.trace()


def _check(tg, to, cols):
    sub = {k: v[:, cols] for k, v in tg.items()}
    assert np.array_equal(sub["acc"], to["acc"]), np.argwhere(sub["acc"] != to["acc"])[:5]
    lp_err = np.max(np.abs(sub["lp_prop"] - to["lp_prop"]) / np.maximum(1.0, np.abs(to["lp_prop"])))
    assert lp_err <= TOL, lp_err
    ex = loga_excess(sub, to, state_rounding_bound(4096))
    assert ex <= 1.0, (ex, np.unravel_index(np.argmax(np.abs(sub["loga"] - to["loga"]) / diff_scale(to)),
                                            to["loga"].shape))
    return ex


def test_interval_kernel_at_d4096_matches_oracle():
    """Eight chains, n_lag 16, two whole intervals (32 steps, two launches of the interval kernel)."""
    run, ts, x0, C0 = _headline(8, 16)
    steps = 2 * run.n_lag
    g, cfg = _gpu(run, ts, x0, C0, steps, profile=1)
    assert g.profile()["step"][0] == 2          # one launch per whole interval
    tg = g.trace(steps)
    to = _oracle(cfg, ts, x0, C0, steps, 0, run.P)
    _check(tg, to, slice(0, run.P))
    assert 0 < tg["acc"].mean() < 1
    g.close()


def test_fp32_mode_interval_kernel_at_d4096_matches_oracle():
    """The same two whole intervals with the factor quantised to TF32 (prec FP32: the noise product's second K
    pass for the factor's lo term, the map A A_n from both terms) against the oracle's FP32 mode."""
    import paper_1506_05741_b300 as dm
    run, ts, x0, C0 = _headline(8, 16)
    steps = 2 * run.n_lag
    g, cfg = _gpu(run, ts, x0, C0, steps, profile=1, prec=dm.FP32)
    assert g.profile()["step"][0] == 2          # one launch per whole interval
    L, Lq, _, _ = g.factor()
    assert np.array_equal(Lq, oracle.round_tf32(L))                 # TF32, not BF16
    tg = g.trace(steps)
    to = _oracle(cfg, ts, x0, C0, steps, 0, run.P)
    _check(tg, to, slice(0, run.P))
    assert 0 < tg["acc"].mean() < 1
    g.close()


def test_full_size_interval_sampled_chains_match_oracle():
    """The benchmark's launch configuration: P = 512, n_lag = 128, two whole intervals (256 steps); chains 0, 1,
    300 and 511 against the oracle."""
    run, ts, x0, C0 = _headline(512, 128)
    steps = 2 * run.n_lag
    g, cfg = _gpu(run, ts, x0, C0, steps)
    tg = g.trace(steps)
    g.close()
    for c0, n in ((0, 2), (300, 1), (511, 1)):
        to = _oracle(cfg, ts, x0, C0, steps, c0, n)
        _check(tg, to, slice(c0, c0 + n))


def _gemm_f64_check(M, N, K, a_lower):
    """D = B A^T from the tcgen05 GEMM (BN = 256, the benchmark's tile) against the FP64 product of the same
    BF16 operands, within the FP32 accumulation bound 2 K 2^-24 (|B| |A|^T) entrywise."""
    import torch
    import paper_1506_05741_b300 as dm
    l = dm.lib()
    f = l.diam_op_gemm_bf16_tile
    P, I32 = ctypes.c_void_p, ctypes.c_int32
    f.argtypes = [I32, I32, I32, P, I32, P, P, I32, I32, ctypes.c_float, P, I32, I32, P]
    f.restype = ctypes.c_int
    g = torch.Generator(device="cuda").manual_seed(M + N + K)
    A = torch.randn(M, K, device="cuda", generator=g)
    if a_lower:
        A = torch.tril(A)
    A = A.to(torch.bfloat16)
    B = torch.randn(N, K, device="cuda", generator=g).to(torch.bfloat16)
    D = torch.empty(N, M, dtype=torch.float32, device="cuda")
    assert f(M, N, K, A.view(torch.int16).data_ptr(), K, B.view(torch.int16).data_ptr(), None, K, a_lower, 1.0,
             D.data_ptr(), M, 256, None) == 0
    Ad, Aa = A.double(), A.double().abs()
    worst = 0.0
    for n0 in range(0, N, 8192):
        Bd = B[n0:n0 + 8192].double()
        ref = Bd @ Ad.T
        bound = 2 * K * 2.0 ** -24 * (Bd.abs() @ Aa.T) + 1e-30
        worst = max(worst, ((D[n0:n0 + 8192].double() - ref).abs() / bound).max().item())
    assert worst <= 1.0, worst
    return worst


def test_noise_product_at_full_shape():
    """xi = A_n W for one interval of the benchmark: A_n 4096 x 4096 lower triangular (K blocks past each
    128-row tile skipped), W for P n_lag = 65536 proposals."""
    _gemm_f64_check(4096, 65536, 4096, 1)


def test_fold_product_at_full_shape():
    """The fold's SYRK shape: the interval's 65536 records (K) of 4096 coordinates against themselves."""
    _gemm_f64_check(4096, 4096, 65536, 0)
