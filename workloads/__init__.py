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
  paper_targets  the six test targets pi_1 .. pi_6 of Sec. 3.1 at any d (Gaussians built from a standard normal
             matrix, and the two twisted Gaussians with their closed-form moments).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

TARGET_DIAG, TARGET_DENSE, TARGET_TANH, TARGET_BANANA, TARGET_REF, TARGET_TWIST = 0, 1, 2, 3, 4, 6


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
    umean: np.ndarray | None = None    # twisted target: exact mean and variance of each u_j = (G x)_j
    uvar: np.ndarray | None = None


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


def dense_gaussian(d: int, seed: int, with_cov: bool = True) -> TargetSpec:
    """Sigma = Q diag(i^-1) Q^T with Q from QR of a seeded N(0,1) d x d FP64 matrix (with_cov = False leaves
    Sigma itself out: the sampler needs only G)."""
    rng = np.random.default_rng(seed)
    Z = rng.standard_normal((d, d))
    Q, _ = np.linalg.qr(Z)
    i = np.arange(1, d + 1, dtype=np.float64)
    G = np.sqrt(i)[:, None] * Q.T
    cov = (Q * (1.0 / i)) @ Q.T if with_cov else None
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


def paper_targets(d: int, seed: int = 31, b5: float = 0.3, b6: float = 2.0, sigma2_4: float | None = None) -> dict:
    """pi_1 .. pi_6 of Sec. 3.1 (keys 1 .. 6). A (d x r) standard normal, B = A A^T:
    pi_1 = N(0, (B + I)^-1), r = d;  pi_2 = N(0, (B / d + I)^-1), r = d;  pi_3 = N(0, (B + I)^-1), r = d / 10;
    pi_4 = N(0, V diag[(sigma^-2 n^-4 + 1)^-1] V^T), V the eigenvectors of pi_1's covariance ordered from its
    smallest eigenvalue (sigma^2 = sigma2_4, default 1 / d^2, a condition number O(d^2));
    pi_5, pi_6 = pi_1 o V o phi o V^T with phi(w)_j = w_j + b_{j-1} w_{j-1}^2 for the even (1-based) j <= d / 10,
    b_i = b sigma_i^-2 / sqrt(d), b = b5 (mildly twisted) or b6 (strongly twisted).
    The Gaussians are dense targets, log pi = -|G x|^2 / 2 with G^T G their precision (G from its Cholesky
    factor); the twisted ones are TARGET_TWIST: u = G x with G = V^T, log pi = -sum_j (u_j + c_j u_{j-1}^2)^2
    / (2 lam_j), lam = the eigenvalues sigma_j^2 of pi_1's covariance and c_j the twist coefficients (in y).
    Their exact moments: E u_j = -c_j sigma_{j-1}^2, var u_j = sigma_j^2 + 2 c_j^2 sigma_{j-1}^4 (mean 0, variance
    sigma_j^2 where c_j = 0)."""
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((d, d))
    A3 = rng.standard_normal((d, max(1, d // 10)))
    eye = np.eye(d)

    def gauss(prec):
        cov = np.linalg.inv(prec)
        return TargetSpec(TARGET_DENSE, d, d_y=d, G=np.ascontiguousarray(np.linalg.cholesky(prec).T),
                          cov=0.5 * (cov + cov.T), mean=np.zeros(d))

    B = A @ A.T
    out = {1: gauss(B + eye), 2: gauss(B / d + eye), 3: gauss(A3 @ A3.T + eye)}
    sig2, V = np.linalg.eigh(out[1].cov)              # ascending: v_1 belongs to the smallest eigenvalue
    n = np.arange(1, d + 1, dtype=np.float64)
    s2 = sigma2_4 if sigma2_4 is not None else 1.0 / d ** 2
    prec4 = n ** -4.0 / s2 + 1.0
    out[4] = TargetSpec(TARGET_DENSE, d, d_y=d, G=np.ascontiguousarray(np.sqrt(prec4)[:, None] * V.T),
                        cov=(V / prec4) @ V.T, mean=np.zeros(d))
    for key, b in ((5, b5), (6, b6)):
        c = np.zeros(d)
        for j in range(1, d // 10, 2):                # 0-based j = 1, 3, ...: the 1-based even indices <= d / 10
            c[j] = b / sig2[j - 1] / math.sqrt(d)
        umean = np.zeros(d)
        uvar = sig2.copy()
        tw = c != 0
        umean[1:][tw[1:]] = -c[1:][tw[1:]] * sig2[:-1][tw[1:]]
        uvar[1:][tw[1:]] += 2.0 * c[1:][tw[1:]] ** 2 * sig2[:-1][tw[1:]] ** 2
        out[key] = TargetSpec(TARGET_TWIST, d, d_y=d, G=np.ascontiguousarray(V.T), lam=sig2.copy(), y=c,
                              umean=umean, uvar=uvar)
    return out


def diag64() -> RunSpec:
    return RunSpec("diag64", diag_gaussian(64), P=1, n_lag=100, beta0=0.3, n_steps=20000, seed=0)


def dense1024(d: int = 1024, P: int = 128) -> RunSpec:
    return RunSpec("dense1024", dense_gaussian(d, 1002), P=P, n_lag=64, M=10, beta0=min(2.4 / math.sqrt(d), 0.5),
                   n_steps=50 * 10 * 64, seed=2)


def tanh4096(d: int = 4096, d_y: int = 2048, P: int = 256, n_lag: int = 128) -> RunSpec:
    return RunSpec("tanh4096", tanh_regression(d, d_y, 1003), P=P, n_lag=n_lag, M=10,
                   beta0=min(2.4 / math.sqrt(d), 0.5), n_steps=20 * 10 * n_lag, seed=3)


def multi64(n_problems: int = 64, d_lo: int = 256, d_hi: int = 8192, with_cov: bool = True):
    """Problem sizes d_j = round(exp(U(ln d_lo, ln d_hi))) from seed 7; even j dense, odd j banana."""
    rng = np.random.default_rng(7)
    ds = np.rint(np.exp(rng.uniform(math.log(d_lo), math.log(d_hi), n_problems))).astype(int)
    specs = []
    for j, d in enumerate(ds):
        t = dense_gaussian(int(d), 7000 + j, with_cov=with_cov) if j % 2 == 0 else banana(int(d))
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
