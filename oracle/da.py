"""FP64 reference of delayed acceptance (two-stage Metropolis-Hastings, Christen & Fox 2005) for the DIAM
proposal with a surrogate screen: the rule the library's BF16 screen applies, written plainly for small cases.

TEST INFRASTRUCTURE (see ``oracle/__init__.py``). The surrogate is not in the paper. This reference covers the
screen with a fixed factor and beta (no refresh, no training): the part the two-stage rule adds to Algorithm 1.

Per chain p and step t, with the oracle's random streams (oracle.normals, oracle.uniform):
  x* = x_ref + rho (x - x_ref) + beta alpha Lq W,   q(v) = |Lq^{-1}(v - x_ref)|^2 / (2 alpha^2)      (eq. (diamnl))
  s(v) = the target's exact O(d) terms at v + mu + sigma * net(v)     (the network estimates the linear-map terms)
  stage 1: log a1 = s(x*) - s(x) + q(x*) - q(x); pass iff log u1 < log a1, u1 = uniform(tag 3)
  stage 2 (passed proposals only): log a2 = log pi(x*) - log pi(x) - s(x*) + s(x); accept iff log u2 < log a2,
           u2 = uniform(tag 1)
The stage-1 screen and the stage-2 correction make the pair a Metropolis-Hastings kernel for pi whatever s is.

The network is evaluated as the library's tensor cores see it: input bf16((v - shift) * scale) (shift 0, scale 1
for a screen that runs from the start), weights W1, W2 rounded to BF16 from their FP32 values, biases and w3 in
FP32, hidden activations GELU (exact erf form) rounded to BF16, sums in FP64 (the library's are FP32: the values
agree to FP32 rounding of the sums, the BF16 roundings they feed agree except at rounding boundaries).
"""
from __future__ import annotations

import numpy as np

from . import forward_sub, normals, round_bf16, uniform
from .mlp import gelu

TAG_U, TAG_UDA = 1, 3


def bf16(a):
    return round_bf16(np.asarray(a, np.float64))


def f32(a):
    return np.asarray(a, np.float64).astype(np.float32).astype(np.float64)


class Screen:
    """The surrogate network as the screen evaluates it (weights from their FP64 values, as uploaded)."""

    def __init__(self, w, mu=0.0, sigma=1.0):
        self.W1 = bf16(f32(w["W1"]))
        self.W2 = bf16(f32(w["W2"]))
        self.b1, self.b2, self.w3 = f32(w["b1"]), f32(w["b2"]), f32(w["w3"])
        self.b3 = float(np.float32(np.ravel(w["b3"])[0]))
        self.mu, self.sigma = mu, sigma

    def net(self, v):
        u = bf16(f32(v))
        h1 = bf16(gelu(self.W1 @ u + self.b1))
        h2 = bf16(gelu(self.W2 @ h1 + self.b2))
        return self.mu + self.sigma * (float(self.w3 @ h2) + self.b3)


def run(target, od_terms, screen, x0, Lq, xref, beta, infl, seed, problem_id, steps, chain0=0):
    """Two-stage chains for steps steps from x0 (P x d) with the fixed factor Lq (the quantised one) and x_ref.
    target(v) = log pi(v); od_terms(v) = the exact O(d) terms of log pi in s. Returns the per-step trace:
    stage-1 pass, acceptance, log a1, log a2 (NaN where stage 1 rejected), |log u - log a| margins."""
    P, d = x0.shape
    rho = np.sqrt(1.0 - beta * beta)
    ba = beta * infl
    X = np.array(x0, np.float64)
    Lq = np.asarray(Lq, np.float64)

    def q(v):
        z = forward_sub(Lq, v - xref)
        return 0.5 * float(z @ z) / (infl * infl)

    lp = np.array([target(x) for x in X])
    qc = np.array([q(x) for x in X])
    s = np.array([od_terms(x) + screen.net(x) for x in X])
    out = {k: np.zeros((steps, P)) for k in ("loga1", "loga2", "m1", "m2")}
    out["pass1"] = np.zeros((steps, P), bool)
    out["acc"] = np.zeros((steps, P), bool)
    for t in range(steps):
        for p in range(P):
            W = bf16(normals(seed, problem_id, t, chain0 + p, d).astype(np.float64))
            xp = xref + rho * (X[p] - xref) + ba * (Lq @ W)
            qp = q(xp)
            sp = od_terms(xp) + screen.net(xp)
            a1 = sp - s[p] + qp - qc[p]
            l1 = np.log(uniform(seed, problem_id, TAG_UDA, t, chain0 + p))
            out["loga1"][t, p], out["m1"][t, p] = a1, abs(l1 - a1)
            out["loga2"][t, p], out["m2"][t, p] = np.nan, np.inf
            if not (np.isfinite(a1) and l1 < a1):
                continue
            out["pass1"][t, p] = True
            lpp = target(xp)
            a2 = lpp - lp[p] - sp + s[p]
            l2 = np.log(uniform(seed, problem_id, TAG_U, t, chain0 + p))
            out["loga2"][t, p], out["m2"][t, p] = a2, abs(l2 - a2)
            if np.isfinite(lpp) and l2 < a2:
                out["acc"][t, p] = True
                X[p], lp[p], qc[p], s[p] = xp, lpp, qp, sp
    out["x"] = X
    return out
