"""Pins of the delayed-acceptance reference (oracle/da.py) against what the two-stage rule fixes (Christen & Fox
2005; the screen is not in the paper, its proposal is Algorithm 1's):

- with a surrogate equal to log pi itself, stage 2's ratio is exactly 0, so every proposal the screen passes is
  accepted, and stage 1's ratio is Algorithm 1's log a (eq. (accept)), the same number the main oracle computes
  for the same state and noise;
- with a surrogate that is wrong (a random network, a mis-scaled density), the two-stage chain still samples the
  target: coordinate means and variances of a small Gaussian within 4 batch-means standard errors;
- a surrogate that is a constant passes every proposal whose q-difference allows it (stage 1 sees only q), and
  stage 2 is then the whole Metropolis-Hastings ratio."""
import numpy as np

import oracle
from oracle import da
import workloads


def _zero_net(d, h=4):
    return {"W1": np.zeros((h, d)), "b1": np.zeros(h), "W2": np.zeros((h, h)), "b2": np.zeros(h),
            "w3": np.zeros(h), "b3": np.zeros(())}


def _diag_setup(d, P, seed):
    ts = workloads.diag_gaussian(d)
    target = oracle.Target(ts.kind, d, 0, lam=ts.lam)
    x0 = workloads.start_state(d, P, seed) * np.sqrt(ts.lam)
    C0 = np.diag(ts.lam * np.linspace(0.6, 1.4, d))   # a factor that is not the target's: log a != 0
    Lq = oracle.round_bf16(oracle.cholesky(C0))
    return ts, target, x0, C0, Lq


def test_exact_surrogate_reduces_stage_one_to_algorithm_1():
    d, P, beta, seed = 16, 4, 0.5, 9
    ts, target, x0, C0, Lq = _diag_setup(d, P, 2)
    exact = lambda v: -0.5 * float(np.sum(v * v / ts.lam))     # s = log pi: the O(d) terms are all of it
    ref = da.run(target.logpi, exact, da.Screen(_zero_net(d)), x0, Lq, np.zeros(d), beta, 1.0, seed, 0, 40)
    passed = ref["pass1"]
    assert passed.any() and not passed.all()
    assert np.all(np.abs(ref["loga2"][passed]) <= 1e-10)        # log pi(x*) - log pi(x) - s(x*) + s(x), rounding
    assert np.array_equal(ref["acc"], passed)                   # log u2 < 0 always
    cfg = oracle.default_config(d=d, P=P, n_lag=1000, beta0=beta, adapt_beta=0, prec=oracle.BF16, seed=seed,
                                trace_steps=1, min_samples_refresh=10 ** 9, xref_mode=0)
    o = oracle.Sampler(cfg, target, x0=x0, C0=C0)
    o.run(1)
    np.testing.assert_allclose(ref["loga1"][0], o.trace()["loga"][0], rtol=0, atol=1e-10)


def test_two_stage_chain_keeps_the_target_with_a_wrong_surrogate():
    d, P, beta, seed, steps = 3, 8, 0.6, 5, 5000
    ts, target, x0, C0, Lq = _diag_setup(d, P, 3)
    rng = np.random.default_rng(0)
    h = 6
    w = {"W1": rng.standard_normal((h, d)), "b1": rng.standard_normal(h) * 0.1, "W2": rng.standard_normal((h, h)) * 0.5,
         "b2": np.zeros(h), "w3": rng.standard_normal(h), "b3": np.zeros(())}
    half = lambda v: -0.25 * float(np.sum(v * v / ts.lam))      # half the true log-density, plus the network
    # the reference returns the final states: run it in batches of 200 steps (fresh random streams per batch, the
    # same kernel) and keep the states at the batch ends, about independent draws once the chains have mixed
    X, p1, acc = [], [], []
    x = x0.copy()
    for t in range(0, steps, 200):
        r = da.run(target.logpi, half, da.Screen(w), x, Lq, np.zeros(d), beta, 1.0, seed + 1 + t, 0, 200)
        x = r["x"]
        X.append(x.copy())
        p1.append(r["pass1"].mean())
        acc.append(r["acc"].mean())
    assert 0.05 < np.mean(p1) < 0.95 and 0.05 < np.mean(acc) < 0.95   # both stages decide something
    X = np.array(X[3:])                                          # (batches, P, d) states at batch ends
    for k in range(d):
        for f, truth in ((X[..., k], 0.0), (X[..., k] ** 2, ts.lam[k])):
            m, se = f.mean(), f.std(ddof=1) / np.sqrt(f.size)
            assert abs(m - truth) <= 4 * se + 1e-12, (k, m, truth, se)


def test_constant_surrogate_screens_on_q_alone():
    d, P, beta, seed = 8, 4, 0.4, 11
    ts, target, x0, C0, Lq = _diag_setup(d, P, 4)
    ref = da.run(target.logpi, lambda v: 0.0, da.Screen(_zero_net(d)), x0, Lq, np.zeros(d), beta, 1.0, seed, 0, 30)
    cfg = oracle.default_config(d=d, P=P, n_lag=1000, beta0=beta, adapt_beta=0, prec=oracle.BF16, seed=seed,
                                trace_steps=1, min_samples_refresh=10 ** 9, xref_mode=0)
    o = oracle.Sampler(cfg, target, x0=x0, C0=C0)
    o.run(1)
    tr = o.trace()
    dq = tr["q_prop"][0] - tr["q_cur"][0]
    np.testing.assert_allclose(ref["loga1"][0], dq, rtol=0, atol=1e-10)         # s(x*) - s(x) = 0
    p1 = ref["pass1"][0]
    np.testing.assert_allclose(ref["loga2"][0][p1], (tr["loga"][0] - dq)[p1], rtol=0, atol=1e-10)
