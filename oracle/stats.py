"""Diagnostics for the oracle's chains: batch-means ESS and the PSRF of Sec. 2.4.2.

TEST INFRASTRUCTURE (see ``oracle/__init__.py``). Plain numpy, written from the definitions.
"""
from __future__ import annotations

import numpy as np


def batch_means(series: np.ndarray, n_batches: int = 20):
    """Batch means of a (T, P) series: the T steps of each chain split into n_batches equal batches.

    Returns (means (n_batches, P), batch length). Trailing steps that do not fill a batch are dropped.
    """
    T = series.shape[0]
    b = T // n_batches
    s = series[: b * n_batches]
    return s.reshape(n_batches, b, *series.shape[1:]).mean(axis=1), b


def ess_batch_means(series: np.ndarray, n_batches: int = 20) -> float:
    """Effective sample size N_eff = N / (1 + 2 Theta) (eq. (mse)), with the integrated autocorrelation
    time estimated by batch means pooled over chains: tau = b * var(batch means) / var(series)."""
    series = np.asarray(series, np.float64)
    if series.ndim == 1:
        series = series[:, None]
    T, P = series.shape
    mu = series.mean()
    var = ((series - mu) ** 2).sum() / (T * P - 1)
    bm, b = batch_means(series, n_batches)
    var_bm = ((bm - mu) ** 2).sum() / (bm.size - 1)
    if var <= 0 or var_bm <= 0:
        return float(T * P)
    tau = b * var_bm / var
    return float(min(T * P, T * P / max(tau, 1e-300)))


def mean_and_se(series: np.ndarray, n_batches: int = 20):
    """Pooled mean of a (T, P) series and its batch-means standard error."""
    series = np.asarray(series, np.float64)
    if series.ndim == 1:
        series = series[:, None]
    bm, _ = batch_means(series, n_batches)
    mu = bm.mean()
    se = bm.std(ddof=1) / np.sqrt(bm.size)
    return float(mu), float(se)


def psrf(chain_mean: np.ndarray, chain_var: np.ndarray, n: int) -> np.ndarray:
    """Potential scale reduction factor sqrt(R_i) of eq. (winco), (btwco), (psrf).

    chain_mean, chain_var: (P, d) per-chain sample mean m^p and within-chain variance (C^p)_ii with the
    1/n normalisation of eq. (sampcov); n = M K n_lag samples per chain.
    """
    P = chain_mean.shape[0]
    m_glob = chain_mean.mean(axis=0)
    B = n / (P - 1) * ((chain_mean - m_glob) ** 2).sum(axis=0)
    W = n / ((n - 1) * P) * chain_var.sum(axis=0)
    R = (n - 1) / n + (P + 1) / (P * n) * B / W
    return np.sqrt(R)
