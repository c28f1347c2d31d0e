"""FP64 reference of the delayed-acceptance surrogate: an MLP d -> h1 -> h2 -> 1 with GELU (exact erf form),
its gradient of the mean squared error, and one Adam step (Kingma & Ba 2015).

TEST INFRASTRUCTURE (see ``oracle/__init__.py``). The surrogate is not in the paper; it screens proposals as
the first stage of a two-stage (delayed-acceptance) Metropolis-Hastings test (Christen & Fox 2005), with
the exact target as the second stage, so the chain still targets pi exactly.

Parameters: W1 (h1 x d), b1 (h1), W2 (h2 x h1), b2 (h2), w3 (h2), b3 (scalar). Input x is the normalised
state u = (x - shift) * scale (per coordinate); output s = mu + sigma * (w3 . H2 + b3).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

SQRT1_2 = 1.0 / math.sqrt(2.0)
INV_SQRT_2PI = 1.0 / math.sqrt(2.0 * math.pi)


def gelu(z):
    return 0.5 * z * (1.0 + erf(z * SQRT1_2))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z * SQRT1_2)) + z * INV_SQRT_2PI * np.exp(-0.5 * z * z)


def forward(params, U):
    """U: (B, d) normalised inputs. Returns the network output (B,) and the cache for backward."""
    W1, b1, W2, b2, w3, b3 = (params[k] for k in ("W1", "b1", "W2", "b2", "w3", "b3"))
    Z1 = U @ W1.T + b1
    H1 = gelu(Z1)
    Z2 = H1 @ W2.T + b2
    H2 = gelu(Z2)
    out = H2 @ w3 + b3
    return out, (U, Z1, H1, Z2, H2)


def loss_and_grads(params, U, target):
    """L = mean((out - target)^2) / 2 and its gradient with respect to every parameter."""
    out, (U, Z1, H1, Z2, H2) = forward(params, U)
    B = U.shape[0]
    r = out - target
    L = 0.5 * float(np.mean(r * r))
    ds = r / B
    g = {}
    g["w3"] = H2.T @ ds
    g["b3"] = np.array(ds.sum())
    dH2 = np.outer(ds, params["w3"])
    dZ2 = dH2 * gelu_grad(Z2)
    g["W2"] = dZ2.T @ H1
    g["b2"] = dZ2.sum(axis=0)
    dH1 = dZ2 @ params["W2"]
    dZ1 = dH1 * gelu_grad(Z1)
    g["W1"] = dZ1.T @ U
    g["b1"] = dZ1.sum(axis=0)
    return L, g


def adam_step(params, grads, m, v, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (bias-corrected first and second moments), in place; t is the 1-based step count."""
    for k in params:
        m[k] = beta1 * m[k] + (1.0 - beta1) * grads[k]
        v[k] = beta2 * v[k] + (1.0 - beta2) * grads[k] * grads[k]
        mh = m[k] / (1.0 - beta1 ** t)
        vh = v[k] / (1.0 - beta2 ** t)
        params[k] = params[k] - lr * mh / (np.sqrt(vh) + eps)
    return params
