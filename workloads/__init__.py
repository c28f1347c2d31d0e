"""Seeded synthetic workloads for the DIAM hot path.

This module only builds inputs: target data (the arrays that define log pi) and run parameters. It holds
none of the sampler's arithmetic and draws with numpy's PCG64 generator, never with the sampler's Philox
streams, so both the CUDA path and the CPU oracle can take their inputs from here.

Workloads (the kinds of target of the paper's experiments, Sec. 3.1, at the sizes of the runs below):
  diag64     Gaussian N(0, diag(i^-2)), d = 64, one chain.
  dense1024  Gaussian with covariance Q diag(i^-1) Q^T, Q from the QR factorisation of a seeded
             N(0, 1) matrix; log pi = -|G x|^2 / 2 with G = diag(sqrt(i)) Q^T. d = 1024, P = 128.
  tanh4096   Bayesian regression: prior N(0, diag(i^-2)), y = tanh(A x*) + 0.05 eps, A (2048 x 4096)
             N(0, 1/4096) in FP32, x* from the prior. P = 256, n_lag = 128.
  banana     pi ~ exp(-x1^2/200 - (x2 + 0.1 x1^2 - 10)^2 / 2 - sum_{i>=3} x_i^2 / (2 lambda_i)), lambda_i = 1/i.
  multi64    64 problems, d log-uniform in [256, 8192]: even ones dense Gaussians, odd ones bananas.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

TARGET_DIAG, TARGET_DENSE, TARGET_TANH, TARGET_BANANA, TARGET_REF = 0, 1, 2, 3, 4


@dataclass
class TargetSpec:
    kind: int
    d: int
    d_y: int = 0
    lam: np.ndarray | None = None      # d, variances lambda_i (prior / diagonal)
    G: np.ndarray | None = None        # d_y x d
    A: np.ndarray | None = None        # d_y x d
    y: np.ndarray | None = None        # d_y
    sigma: float = 0.0
    ban_a: float = 100.0
    ban_b: float = 0.1
    ban_c: float = 10.0
    cov: np.ndarray | None = None      # exact covariance when known (for checks)
    mean: np.ndarray | None = None


@dataclass
class RunSpec:
    name: str
    target: TargetSpec
    P: int
    n_lag: int
    M: int = 10
    beta0: float = 0.3
    n_steps: int = 0
    seed: int = 0
    extra: dict = field(default_factory=dict)


def diag_gaussian(d: int, power: float = 2.0) -> TargetSpec:
    lam = np.arange(1, d + 1, dtype=np.float64) ** (-power)
    return TargetSpec(TARGET_DIAG, d, lam=lam, cov=np.diag(lam), mean=np.zeros(d))


def dense_gaussian(d: int, seed: int) -> TargetSpec:
    """Sigma = Q diag(i^-1) Q^T with Q from QR of a seeded N(0,1) d x d FP64 matrix."""
    rng = np.random.default_rng(seed)
    Z = rng.standard_normal((d, d))
    Q, _ = np.linalg.qr(Z)
    i = np.arange(1, d + 1, dtype=np.float64)
    G = np.sqrt(i)[:, None] * Q.T
    cov = (Q * (1.0 / i)) @ Q.T
    return TargetSpec(TARGET_DENSE, d, d_y=d, G=np.ascontiguousarray(G), cov=cov, mean=np.zeros(d))


def tanh_regression(d: int, d_y: int, seed: int, sigma: float = 0.05) -> TargetSpec:
    rng = np.random.default_rng(seed)
    A32 = (rng.standard_normal((d_y, d), dtype=np.float32) * np.float32(1.0 / math.sqrt(d)))
    lam = np.arange(1, d + 1, dtype=np.float64) ** -2.0
    xstar = rng.standard_normal(d) * np.sqrt(lam)
    eps = rng.standard_normal(d_y)
    A = A32.astype(np.float64)
    y = np.tanh(A @ xstar) + sigma * eps
    return TargetSpec(TARGET_TANH, d, d_y=d_y, lam=lam, A=A, y=y, sigma=sigma)


def banana(d: int, a: float = 100.0, b: float = 0.1, c: float = 10.0) -> TargetSpec:
    lam = 1.0 / np.arange(1, d + 1, dtype=np.float64)
    var = lam.copy()
    var[0] = a
    if d > 1:
        var[1] = 1.0 + b * b * 2.0 * a * a
    return TargetSpec(TARGET_BANANA, d, lam=lam, ban_a=a, ban_b=b, ban_c=c, mean=np.zeros(d),
                      cov=np.diag(var))


def diag64() -> RunSpec:
    return RunSpec("diag64", diag_gaussian(64), P=1, n_lag=100, beta0=0.3, n_steps=20000, seed=0)


def dense1024(d: int = 1024, P: int = 128) -> RunSpec:
    return RunSpec("dense1024", dense_gaussian(d, 1002), P=P, n_lag=64, M=10, beta0=min(2.4 / math.sqrt(d), 0.5),
                   n_steps=50 * 10 * 64, seed=2)


def tanh4096(d: int = 4096, d_y: int = 2048, P: int = 256, n_lag: int = 128) -> RunSpec:
    return RunSpec("tanh4096", tanh_regression(d, d_y, 1003), P=P, n_lag=n_lag, M=10,
                   beta0=min(2.4 / math.sqrt(d), 0.5), n_steps=20 * 10 * n_lag, seed=3)


def multi64(n_problems: int = 64, d_lo: int = 256, d_hi: int = 8192):
    """Problem sizes d_j = round(exp(U(ln d_lo, ln d_hi))) from seed 7; even j dense, odd j banana."""
    rng = np.random.default_rng(7)
    ds = np.rint(np.exp(rng.uniform(math.log(d_lo), math.log(d_hi), n_problems))).astype(int)
    specs = []
    for j, d in enumerate(ds):
        t = dense_gaussian(int(d), 7000 + j) if j % 2 == 0 else banana(int(d))
        specs.append(RunSpec(f"multi{j}", t, P=32, n_lag=64, M=10, beta0=min(2.4 / math.sqrt(d), 0.5), seed=7 + j))
    return specs


def multi_sizes(n_problems: int = 64, d_lo: int = 256, d_hi: int = 8192):
    rng = np.random.default_rng(7)
    return np.rint(np.exp(rng.uniform(math.log(d_lo), math.log(d_hi), n_problems))).astype(int)


def start_state(d: int, P: int, seed: int, scale: np.ndarray | float = 1.0) -> np.ndarray:
    """A seeded over-dispersed starting state (P x d)."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((P, d)) * scale


def spd_matrix(d: int, seed: int, cond: float = 1e3) -> np.ndarray:
    """A seeded symmetric positive definite matrix with eigenvalues log-spaced in [1/cond, 1]."""
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((d, d)))
    ev = np.logspace(0, -math.log10(cond), d)
    return (Q * ev) @ Q.T


def mlp_init(d: int, h1: int = 512, h2: int = 512, seed: int = 4) -> dict:
    """Seeded initial weights of the surrogate network (He-scaled normal, zero biases), FP64."""
    rng = np.random.default_rng(seed)
    return {"W1": rng.standard_normal((h1, d)) * math.sqrt(2.0 / d), "b1": np.zeros(h1),
            "W2": rng.standard_normal((h2, h1)) * math.sqrt(2.0 / h1), "b2": np.zeros(h2),
            "w3": rng.standard_normal(h2) * math.sqrt(1.0 / h2), "b3": np.zeros(())}
