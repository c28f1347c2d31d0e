"""Delayed acceptance (two-stage Metropolis-Hastings with a BF16 MLP surrogate trained on the GPU).

- The training kernels' loss and gradients against the FP64 oracle network (oracle/mlp.py), fed the same
  BF16-rounded weights and inputs; the CUDA side also rounds its hidden activations and backward signals
  to BF16, so agreement is normwise to ~1e-2.
- A run that fills the ring, trains, screens: counters are consistent and the surrogate error is finite.
- Exactness: on a Gaussian target the two-stage chain still samples the target (moments within 4
  batch-means standard errors of the known covariance)."""
import numpy as np
import pytest

import oracle
from oracle import mlp, stats
import workloads

pytestmark = pytest.mark.gpu


def _sampler(ts, P, **kw):
    import paper_1506_05741_b300 as dm
    cfg = dm.default_config(ts.d, P, prec=dm.BF16, **kw)
    return dm, cfg


def test_training_gradients_match_oracle_network():
    import paper_1506_05741_b300 as dm
    ts = workloads.tanh_regression(256, 128, 21)
    cfg = dm.default_config(256, 64, prec=dm.BF16, n_lag=16, seed=1)
    s = dm.Sampler(cfg, ts)
    w = workloads.mlp_init(256, 128, 128, seed=5)
    w["b1"] = np.random.default_rng(1).standard_normal(128) * 0.05
    w["b3"] = np.array([0.2])
    s.da_enable(dm.da_default_config(h1=128, h2=128, batch=128, ring=1000), w)
    U = np.random.default_rng(2).standard_normal((128, 256))
    t = np.random.default_rng(3).standard_normal(128)
    loss, g = s.da_grad(U, t)
    # the oracle with exactly the weights and inputs the tensor cores see
    q = {k: np.asarray(v, np.float64) for k, v in w.items()}
    q["W1"] = oracle.round_bf16(q["W1"].astype(np.float32).astype(np.float64))
    q["W2"] = oracle.round_bf16(q["W2"].astype(np.float32).astype(np.float64))
    for k in ("b1", "b2", "w3"):
        q[k] = q[k].astype(np.float32).astype(np.float64)
    q["b3"] = np.array(float(np.float32(w["b3"][0])))
    Uq = oracle.round_bf16(U)
    L, go = mlp.loss_and_grads(q, Uq, t)
    assert abs(loss - L) <= 1e-2 * L
    for k in ("W1", "b1", "W2", "b2", "w3", "b3"):
        a, b = np.ravel(g[k]), np.ravel(go[k])
        assert np.linalg.norm(a - b) <= 3e-2 * np.linalg.norm(b), (k, np.linalg.norm(a - b) / np.linalg.norm(b))


def test_adam_kernel_matches_oracle_adam():
    """The training's Adam kernel (diam_da_adam_step: FP32 masters and moments) against the oracle's adam_step
    (FP64) over five steps with seeded gradients (rounded to FP32, as uploaded) and non-default lr, beta1, beta2
    and eps: the weights' changes agree to FP32 accuracy, so a swapped beta, an off-by-one bias-correction
    exponent or a misplaced eps would show."""
    import paper_1506_05741_b300 as dm
    d, h1, h2 = 192, 128, 128
    ts = workloads.tanh_regression(d, 64, 23)
    s = dm.Sampler(dm.default_config(d, 8, prec=dm.BF16, n_lag=8, seed=1), ts)
    w = workloads.mlp_init(d, h1, h2, seed=7)
    lr, b1, b2, eps = 3e-3, 0.8, 0.95, 1e-4
    s.da_enable(dm.da_default_config(h1=h1, h2=h2, batch=128, ring=1000, lr=lr, beta1=b1, beta2=b2, adam_eps=eps), w)
    f32 = lambda a: np.asarray(a, np.float64).astype(np.float32).astype(np.float64)
    params = {k: f32(v) for k, v in w.items()}
    w0 = {k: v.copy() for k, v in params.items()}
    m = {k: np.zeros_like(v) for k, v in params.items()}
    v = {k: np.zeros_like(v) for k, v in params.items()}
    rng = np.random.default_rng(8)
    for t in range(1, 6):
        grads = {k: f32(rng.standard_normal(np.shape(params[k])) * 10.0 ** rng.uniform(-3, 0)) for k in params}
        s.da_adam_step(grads)
        mlp.adam_step(params, grads, m, v, t, lr=lr, beta1=b1, beta2=b2, eps=eps)
    got = s.da_weights()
    for k in params:
        dg = np.ravel(got[k]) - np.ravel(w0[k])
        do = np.ravel(params[k]) - np.ravel(w0[k])
        # |dW| ~ 5 lr; FP32 rounding of the weights themselves (|W| <= ~1) and of the update's terms
        assert np.max(np.abs(dg - do)) <= 1e-5 * lr * 5 + 2e-7 * np.max(np.abs(np.ravel(w0[k])) + 1.0), k
        assert np.max(np.abs(do)) > 0.3 * lr    # the steps did move the weights
    s.close()


def test_two_stage_decisions_match_oracle():
    """The screen (stage 1) and the exact test (stage 2) of delayed acceptance against the FP64 reference of the
    two-stage rule (oracle/da.py), with stage 1 on from the start (screen_from_start, the given network, no
    training) and a fixed factor and beta: tanh regression d = 192, d_y = 64, eight chains, 64 steps. Every stage-1
    pass and every final decision agree (only a decision whose log u lies within 5e-3 of its log a on the oracle's
    side may go the other way, the network's BF16 roundings may differ there, and then ends that chain's
    comparison); the stage-2 log ratios agree to
    2e-3 of max(1, |log a2|) (the same BF16 roundings, and FP32 sums of the network and of the map terms)."""
    import paper_1506_05741_b300 as dm
    from oracle import da
    d, dy, P, steps = 192, 64, 8, 64
    ts = workloads.tanh_regression(d, dy, 24)
    x0 = workloads.start_state(d, P, 3) * np.sqrt(ts.lam)
    C0 = np.diag(ts.lam)
    cfg = dm.default_config(d, P, prec=dm.BF16, n_lag=16, seed=13, beta0=0.3, adapt_beta=0, min_samples_refresh=10 ** 12)
    cfg["trace_steps"] = steps
    s = dm.Sampler(cfg, ts, x0=x0, C0=C0)
    w = workloads.mlp_init(d, 128, 128, seed=7)
    s.da_enable(dm.da_default_config(h1=128, h2=128, batch=128, ring=4096, first_train_min=10 ** 9,
                                     retrain_every=10 ** 6, screen_from_start=1), w)
    s.run(steps)
    tg = s.trace(steps)
    st = s.da_stats()
    s.close()
    target = oracle.Target(ts.kind, d, dy, lam=ts.lam, A=oracle.round_bf16(ts.A), y=ts.y, sigma=ts.sigma)
    od = lambda v: -0.5 * float(np.sum(v * v / ts.lam))
    Lq = oracle.round_bf16(oracle.cholesky(C0))
    ref = da.run(target.logpi, od, da.Screen(w), x0, Lq, np.zeros(d), 0.3, 1.0, 13, 0, steps)
    pass_g = np.isfinite(tg["loga"])
    # s enters both ratios: the network's hidden activations are rounded to BF16 from FP32 pre-activations on the
    # GPU and from FP64 ones here, so an activation that lies at a rounding boundary can round the other way,
    # moving s by about |w3_o| 2^-8 |H_o| (~2e-4) per such activation; a margin of 5e-3 covers a few of them
    tie = 5e-3
    compared = 0
    for p in range(P):
        for t in range(steps):
            near = ref["m1"][t, p] < tie or ref["m2"][t, p] < tie
            same = pass_g[t, p] == ref["pass1"][t, p] and tg["acc"][t, p] == ref["acc"][t, p]
            if near and not same:
                break                                # a near tie decided the other way: the chains part here
            assert pass_g[t, p] == ref["pass1"][t, p], (t, p)
            assert tg["acc"][t, p] == ref["acc"][t, p], (t, p)
            if ref["pass1"][t, p]:
                assert abs(tg["loga"][t, p] - ref["loga2"][t, p]) <= 2e-3 * max(1.0, abs(ref["loga2"][t, p])), (t, p)
            compared += 1
    assert compared >= 0.9 * P * steps
    assert 0.05 < ref["pass1"].mean() < 1.0 and ref["acc"].sum() > 0    # both stages decide something
    assert st["stage1_tested"] == P * steps and st["stage1_passed"] == int(pass_g.sum())


def test_delayed_acceptance_trains_and_screens():
    import paper_1506_05741_b300 as dm
    ts = workloads.tanh_regression(256, 128, 22)
    P = 128
    cfg = dm.default_config(256, P, prec=dm.BF16, n_lag=16, M=2, seed=3, beta0=0.2)
    x0 = workloads.start_state(256, P, 4) * np.sqrt(ts.lam)
    s = dm.Sampler(cfg, ts, x0=x0, C0=np.diag(ts.lam))
    s.da_enable(dm.da_default_config(h1=128, h2=128, batch=256, ring=20000, first_train_min=4000, train_steps=100,
                                     retrain_every=4, rmse_bound=1e9), workloads.mlp_init(256, 128, 128, seed=6))
    s.run(16 * 40)
    st = s.da_stats()
    base = s.stats()
    assert st["trainings"] >= 2
    assert np.isfinite(st["last_rmse"]) and st["active"] == 1
    assert 0 < st["stage1_passed"] <= st["stage1_tested"]
    assert st["exact_evals"] < base["steps"] * P           # screening skipped some exact evaluations
    assert st["ring_filled"] == min(20000, st["exact_evals"])
    assert base["accepted"] > 0 and base["nonfinite"] == 0


def test_delayed_acceptance_keeps_the_target():
    """Dense Gaussian target: with stage 1 on (an imperfect surrogate), the chain's mean and variance along
    coordinates stay within 4 batch-means standard errors of the exact covariance."""
    import paper_1506_05741_b300 as dm
    d, P = 64, 256
    ts = workloads.dense_gaussian(d, 31)
    cfg = dm.default_config(d, P, prec=dm.BF16, n_lag=32, M=2, seed=5, beta0=0.5, adapt_beta=0,
                            min_samples_refresh=10 ** 12, xref_mode=0)
    cfg["keep_block_sums"] = 1
    x0 = workloads.start_state(d, P, 9) @ np.linalg.cholesky(ts.cov).T
    s = dm.Sampler(cfg, ts, x0=x0, C0=1.5 * ts.cov)
    s.da_enable(dm.da_default_config(h1=128, h2=128, batch=256, ring=20000, first_train_min=2000, train_steps=100,
                                     retrain_every=1000, rmse_bound=1e9), workloads.mlp_init(d, 128, 128, seed=7))
    s.run(32 * 8)             # fill the ring and train once (stage 1 on from then on)
    assert s.da_stats()["active"] == 1
    nb0 = s.stats()["steps"] // 32
    s.run(32 * 60)
    xs, _ = s.block_sums(200)
    xs = xs[nb0:] / 32.0      # per-interval, per-chain means
    st = s.da_stats()
    assert st["stage1_passed"] < st["stage1_tested"]
    chi2 = 0.0
    for i in range(0, d, 7):
        bm = xs[:, :, i]
        mu = bm.mean()
        se = bm.std(ddof=1) / np.sqrt(bm.size)
        chi2 += (mu / se) ** 2
        assert abs(mu) < 4.5 * se
    # variance of the coordinate from the batch means of x is not available; check the pooled covariance
    m, cov, n = s.moments()
    rel = np.abs(np.diag(cov) - np.diag(ts.cov)) / np.diag(ts.cov)
    assert np.median(rel) < 0.1


def test_trained_surrogate_saves_exact_evaluations():
    """What the network gains: on the same tanh-regression target, seed and start, the two-stage sampler
    with the trained surrogate spends fewer exact log-density evaluations per accepted move than the plain
    sampler, and screens out a real share of the proposals, while its acceptance per proposal stays within a
    factor of two of the plain chain's."""
    import paper_1506_05741_b300 as dm
    d, P, nl = 256, 128, 16
    ts = workloads.tanh_regression(d, 128, 23)
    x0 = workloads.start_state(d, P, 5) * np.sqrt(ts.lam)

    def sampler():
        cfg = dm.default_config(d, P, prec=dm.BF16, n_lag=nl, M=2, seed=7, beta0=0.2)
        return dm.Sampler(cfg, ts, x0=x0, C0=np.diag(ts.lam))

    plain = sampler()
    plain.run(nl * 60)
    sp = plain.stats()
    evals_plain = sp["steps"] * P
    per_acc_plain = evals_plain / max(1, sp["accepted"])

    two = sampler()
    two.da_enable(dm.da_default_config(h1=128, h2=128, batch=256, ring=20000, first_train_min=4000, train_steps=300,
                                       retrain_every=2, rmse_bound=1e9), workloads.mlp_init(d, 128, 128, seed=8))
    two.run(nl * 20)                 # fill the ring; trainings every 2 synchronisations
    s0, d0 = two.stats(), two.da_stats()
    two.run(nl * 40)
    s1, d1 = two.stats(), two.da_stats()
    assert d1["active"] == 1 and d1["trainings"] >= 2
    evals = d1["exact_evals"] - d0["exact_evals"]
    acc = s1["accepted"] - s0["accepted"]
    tested = d1["stage1_tested"] - d0["stage1_tested"]
    passed = d1["stage1_passed"] - d0["stage1_passed"]
    per_acc_two = evals / max(1, acc)
    assert passed < 0.9 * tested                       # stage 1 screens out a real share
    assert per_acc_two < per_acc_plain                 # fewer exact evaluations per accepted move
    assert acc / (40 * nl * P) > 0.5 * sp["accepted"] / (60 * nl * P)
    plain.close()
    two.close()


def test_inactive_surrogate_leaves_the_chain_unchanged():
    """Until the surrogate passes its error bound, the screen is off: the chain with the network attached (its
    ring filled by every step) is bit for bit the chain without it, and every proposal counts as an exact
    evaluation that went to the ring."""
    import paper_1506_05741_b300 as dm
    d, P, nl = 256, 64, 16
    ts = workloads.tanh_regression(d, 128, 24)
    x0 = workloads.start_state(d, P, 6) * np.sqrt(ts.lam)

    def sampler():
        cfg = dm.default_config(d, P, prec=dm.BF16, n_lag=nl, M=2, seed=9, beta0=0.2)
        return dm.Sampler(cfg, ts, x0=x0, C0=np.diag(ts.lam))

    plain = sampler()
    plain.run(nl * 12 + 5)
    two = sampler()
    two.da_enable(dm.da_default_config(h1=128, h2=128, batch=256, ring=3000, first_train_min=2000, train_steps=20,
                                       retrain_every=2, rmse_bound=1e-9), workloads.mlp_init(d, 128, 128, seed=10))
    two.run(nl * 12 + 5)
    xa, la, sa = plain.state()
    xb, lb, sb = two.state()
    assert np.array_equal(xa, xb) and np.array_equal(la, lb) and sa == sb
    st = two.da_stats()
    steps = two.stats()["steps"]
    assert st["active"] == 0 and st["trainings"] >= 1
    assert st["exact_evals"] == steps * P and st["ring_filled"] == min(3000, steps * P)
    plain.close()
    two.close()
