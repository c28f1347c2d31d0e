"""FP64 CUDA path vs the FP64 oracle, through the C ABI.

Bars: the noise draws are bit-exact; the proposals' log-densities and the chain states agree to 1e-12
relative (to max(1, |log pi(x*)|, |q(x*)|, |q(x)|)) while both sides run on the starting factor, and past the
first refresh to the forward error of the FP64 Cholesky factorisation, d u cond(C_n) (two factorisations of
the same C_n in different orders); every accept decision is identical; moments and
factors agree to 1e-10 / 1e-9 (they pass through an FP64 Cholesky of C_n). The proposal-density quadratic
q and log a are compared at Q_TOL = 5e-12 (or 4 d u cond(A_n) if larger): the CUDA path carries
z = A_n^{-1}(x - x_ref) by its recursion while the oracle solves by forward substitution every step, and
each side carries the triangular solve's forward error, bounded by about d u cond(A_n) (Higham,
"Accuracy and Stability of Numerical Algorithms", Thm 8.5). Sizes are small enough for the oracle (seconds) but
span several 64-wide tiles with ragged tails (d = 96, 130, 200), odd chain counts and refreshes."""
import ctypes

import numpy as np
import pytest

import oracle
import workloads
from helpers import make_pair, rel_err, trace_scale

pytestmark = pytest.mark.gpu
TOL = 1e-12
Q_TOL = 5e-12
U = 2.0 ** -53
U_EPS = U


def _torch():
    import torch
    return torch


def _lib():
    import paper_1506_05741_b300 as dm
    l = dm.lib()
    P, I32, I64, U32, U64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint64
    l.diam_op_normals.argtypes = [U64, U32, I64, I32, I32, I32, I32, I32, P, P]
    l.diam_op_cholesky_f64.argtypes = [I32, P, I32, P, P]
    l.diam_op_trsm_lower_f64.argtypes = [I32, I32, P, I32, P, I32, P]
    for f in (l.diam_op_normals, l.diam_op_cholesky_f64, l.diam_op_trsm_lower_f64):
        f.restype = ctypes.c_int
    return l


def test_noise_draws_are_bit_exact():
    torch = _torch()
    l = _lib()
    d, P, S, ld = 103, 5, 3, 104
    out = torch.zeros(S * P * ld, dtype=torch.float32, device="cuda")
    assert l.diam_op_normals(77, 3, 40, S, P, d, ld, 0, out.data_ptr(), None) == 0
    torch.cuda.synchronize()
    g = out.cpu().numpy().reshape(S, P, ld)
    for s in range(S):
        for p in range(P):
            want = oracle.normals(77, 3, 40 + s, p, d)
            assert np.array_equal(g[s, p, :d].view(np.uint32), want.view(np.uint32))
            assert np.all(g[s, p, d:] == 0)
    # BF16 kind: the FP32 draw rounded to nearest even
    outb = torch.zeros(S * P * ld, dtype=torch.int16, device="cuda")
    assert l.diam_op_normals(77, 3, 40, S, P, d, ld, 2, outb.data_ptr(), None) == 0
    torch.cuda.synchronize()
    bits = outb.cpu().numpy().view(np.uint16).reshape(S, P, ld).astype(np.uint32) << 16
    vals = bits.view(np.float32).astype(np.float64)
    for s in range(S):
        for p in range(P):
            assert np.array_equal(vals[s, p, :d], oracle.round_bf16(oracle.normals(77, 3, 40 + s, p, d)))


@pytest.mark.parametrize("d", [1, 5, 64, 65, 130, 300])
def test_cholesky_matches_oracle(d):
    torch = _torch()
    l = _lib()
    Cm = workloads.spd_matrix(d, 500 + d, cond=1e6)
    A = torch.from_numpy(Cm.copy()).cuda()
    info = ctypes.c_int32(-1)
    assert l.diam_op_cholesky_f64(d, A.data_ptr(), d, ctypes.byref(info), None) == 0
    assert info.value == 0
    L = A.cpu().numpy()
    ref = oracle.cholesky(Cm)
    assert np.max(np.abs(L - ref)) <= 1e-11 * np.max(np.abs(ref))
    assert np.all(np.triu(L, 1) == 0)


@pytest.mark.parametrize("d", [130, 300, 1000])
def test_tensor_core_cholesky_matches_oracle(d):
    """The Ozaki-split tensor-core trailing update keeps the factorisation FP64-accurate."""
    torch = _torch()
    l = _lib()
    l.diam_op_cholesky_f64_tc.argtypes = [ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]
    l.diam_op_cholesky_f64_tc.restype = ctypes.c_int
    Cm = workloads.spd_matrix(d, 700 + d, cond=1e6)
    A = torch.from_numpy(Cm.copy()).cuda()
    info = ctypes.c_int32(-1)
    assert l.diam_op_cholesky_f64_tc(d, A.data_ptr(), d, ctypes.byref(info), None) == 0
    assert info.value == 0
    L = A.cpu().numpy()
    ref = oracle.cholesky(Cm)
    assert np.max(np.abs(L - ref)) <= 1e-11 * np.max(np.abs(ref))
    assert np.linalg.norm(L @ L.T - Cm) / np.linalg.norm(Cm) < 1e-14


def test_tensor_core_cholesky_large_reconstructs():
    torch = _torch()
    l = _lib()
    l.diam_op_cholesky_f64_tc.argtypes = [ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]
    d = 4096
    Cm = workloads.spd_matrix(d, 11, cond=1e5)
    A = torch.from_numpy(Cm.copy()).cuda()
    info = ctypes.c_int32(-1)
    assert l.diam_op_cholesky_f64_tc(d, A.data_ptr(), d, ctypes.byref(info), None) == 0 and info.value == 0
    Cg = torch.from_numpy(Cm).cuda()
    assert (torch.linalg.norm(A @ A.T - Cg) / torch.linalg.norm(Cg)).item() < 1e-14
    B = torch.from_numpy(Cm.copy()).cuda()
    assert l.diam_op_cholesky_f64(d, B.data_ptr(), d, ctypes.byref(info), None) == 0 and info.value == 0
    assert (torch.abs(A - B).max() / torch.abs(B).max()).item() < 1e-12


def test_cholesky_reports_indefinite_and_large_reconstructs():
    torch = _torch()
    l = _lib()
    bad = np.eye(70)
    bad[40, 40] = -1.0
    A = torch.from_numpy(bad).cuda()
    info = ctypes.c_int32(0)
    assert l.diam_op_cholesky_f64(70, A.data_ptr(), 70, ctypes.byref(info), None) == 0
    assert info.value == 41
    d = 2048
    Cm = workloads.spd_matrix(d, 9, cond=1e4)
    A = torch.from_numpy(Cm.copy()).cuda()
    assert l.diam_op_cholesky_f64(d, A.data_ptr(), d, ctypes.byref(info), None) == 0 and info.value == 0
    L = A
    Cg = torch.from_numpy(Cm).cuda()
    assert (torch.linalg.norm(L @ L.T - Cg) / torch.linalg.norm(Cg)).item() < 1e-14


def test_trsm_matches_forward_substitution():
    torch = _torch()
    l = _lib()
    d, rows = 200, 7
    Lm = np.linalg.cholesky(workloads.spd_matrix(d, 3, cond=1e4))
    B = np.random.default_rng(0).standard_normal((rows, d))
    Lg = torch.from_numpy(Lm).cuda()
    Bg = torch.from_numpy(B.copy()).cuda()
    assert l.diam_op_trsm_lower_f64(d, rows, Lg.data_ptr(), d, Bg.data_ptr(), d, None) == 0
    torch.cuda.synchronize()
    Y = Bg.cpu().numpy()
    for r in range(rows):
        want = oracle.forward_sub(Lm, B[r])
        assert np.max(np.abs(Y[r] - want)) <= 1e-12 * max(1.0, np.max(np.abs(want)))


@pytest.mark.parametrize("d,rows", [(200, 7), (1000, 300), (4096, 256)])
def test_tensor_core_trsm_matches_forward_substitution(d, rows):
    """Block updates on the tensor cores (Ozaki split) keep the re-solve FP64-accurate: ragged row and
    column tiles, and the 4096 x 256 shape of the refresh's re-solve."""
    torch = _torch()
    l = _lib()
    f = l.diam_op_trsm_lower_f64_tc
    I32, P = ctypes.c_int32, ctypes.c_void_p
    f.argtypes = [I32, I32, P, I32, P, I32, P]
    f.restype = ctypes.c_int
    Lm = np.linalg.cholesky(workloads.spd_matrix(d, 5 + d, cond=1e4))
    B = np.random.default_rng(d).standard_normal((rows, d))
    B[0] *= 1e-6                                   # rows of very different scale
    Lg = torch.from_numpy(Lm).cuda()
    Bg = torch.from_numpy(B.copy()).cuda()
    assert f(d, rows, Lg.data_ptr(), d, Bg.data_ptr(), d, None) == 0
    Y = Bg.cpu().numpy()
    check = range(rows) if d <= 1000 else (0, 1, 77, rows - 1)
    for r in check:
        want = oracle.forward_sub(Lm, B[r])
        assert np.max(np.abs(Y[r] - want)) <= 1e-12 * np.max(np.abs(want))


def _q_tol(o):
    L, _, _ = o.factor()
    return max(Q_TOL, 4 * L.shape[0] * U * np.linalg.cond(L))


def _refresh_tol(o):
    """After a refresh the two sides run on factors from two FP64 Cholesky factorisations of the same C_n in
    different orders; they agree to the factorisation's forward error, about d u cond(C_n) = d u cond(A_n)^2
    (Higham, "Accuracy and Stability of Numerical Algorithms", Sec. 10.1), and the proposals, states and
    log-densities from then on agree to that level."""
    L, _, _ = o.factor()
    return max(TOL, 4 * L.shape[0] * U * np.linalg.cond(L) ** 2)


def _compare(g, o, steps, tol=TOL, q_tol=None, first_factor_steps=None):
    """tol bounds log pi(x*) and the states while both sides run on the starting factor (the first
    first_factor_steps steps: n_lag (1 + refresh_delay), before any refreshed factor is in use); past them the
    bound is _refresh_tol. q_tol bounds q(x*), q(x), log a. The CUDA path carries z = A_n^{-1}(x - x_ref) by the
    z recursion while the oracle solves by forward substitution, so their difference is the substitution's
    forward error, proportional to cond(A_n) eps."""
    if q_tol is None:
        q_tol = _q_tol(o)
    k0 = steps if first_factor_steps is None else min(steps, first_factor_steps)
    late = max(tol, _refresh_tol(o)) if k0 < steps else tol
    q_tol = max(q_tol, late)
    tg, to = g.trace(steps), o.trace()
    assert np.array_equal(tg["acc"], to["acc"]), np.argwhere(tg["acc"] != to["acc"])[:5]
    sc = trace_scale(to)
    assert rel_err(tg["lp_prop"][:k0], to["lp_prop"][:k0], sc[:k0]) <= tol, \
        rel_err(tg["lp_prop"][:k0], to["lp_prop"][:k0], sc[:k0])
    if k0 < steps:
        assert rel_err(tg["lp_prop"][k0:], to["lp_prop"][k0:], sc[k0:]) <= late, \
            (rel_err(tg["lp_prop"][k0:], to["lp_prop"][k0:], sc[k0:]), late)
    for k in ("q_prop", "q_cur", "loga"):
        assert rel_err(tg[k], to[k], sc) <= q_tol, (k, rel_err(tg[k], to[k], sc))
    xg, lpg, st = g.state()
    xo, lpo = o.state()
    assert np.max(np.abs(xg - xo)) <= late * max(1.0, np.max(np.abs(xo)))
    # the current log pi is one of the traced values: same scale as the trace (q is its natural size)
    assert rel_err(lpg, lpo, np.maximum(np.abs(lpo), sc.max(axis=0))) <= late
    co = o.counts()
    assert st["accepted"] == co["accepted"] and st["refreshes"] == co["refreshes"]
    assert st["n"] == co["n"]
    mg, cg, n = g.moments()
    mo, cmo = o.moments()
    assert n == co["n"]
    assert np.max(np.abs(mg - mo)) <= 1e-11 * max(1.0, np.max(np.abs(mo)))
    assert np.max(np.abs(cg - cmo)) <= 1e-10 * np.max(np.abs(cmo))
    Lg, Lqg, xrg, bg = g.factor()
    Lo, Lqo, xro = o.factor()
    assert np.max(np.abs(Lg - Lo)) <= 1e-9 * np.max(np.abs(Lo))
    assert abs(bg - o.beta) <= 1e-15 * o.beta
    return tg


def test_diag64_single_chain_matches_oracle():
    """The diag64 workload (d = 64, lambda_i = i^-2, P = 1, n_lag = 100, x_0 = 0, A_0 = Id, beta = 0.3), all of its
    2e4 steps."""
    run = workloads.diag64()
    steps = 20000
    g, o = make_pair(run.target, run.P, trace_steps=steps, n_lag=run.n_lag, beta0=run.beta0, seed=run.seed)
    g.run(steps)
    o.run(steps)
    # starting at A_0 = Id the chain is stuck for thousands of steps and the adapted factor is far worse
    # conditioned than the target: q's bound grows with cond(A_n) (see the module docstring)
    tg = _compare(g, o, steps, first_factor_steps=run.n_lag)
    assert o.counts()["refreshes"] > 0 and tg["acc"].sum() > 100


@pytest.mark.parametrize("P,steps", [(128, 128), (4, 157 * 64)])
def test_dense1024_prefix_matches_oracle(P, steps):
    """The dense1024 workload (d = 1024, Sigma = Q diag(1/i) Q^T, n_lag = 64, seed 2): all 128 chains over two
    intervals (a refresh between them), and four chains over the first 1e4 steps (157 whole intervals, a refresh
    at each; the moments fold whole intervals)."""
    run = workloads.dense1024(P=P)
    ts = run.target
    x0 = workloads.start_state(ts.d, P, 3) @ np.linalg.cholesky(ts.cov).T
    g, o = make_pair(ts, P, trace_steps=steps, threads=8, n_lag=run.n_lag, beta0=run.beta0, seed=run.seed, x0=x0,
                     C0=ts.cov)
    g.run(steps)
    o.run(steps)
    tg = _compare(g, o, steps, first_factor_steps=run.n_lag)
    assert o.counts()["refreshes"] >= (1 if steps == 128 else 100) and 0 < tg["acc"].mean() < 1


@pytest.mark.parametrize("kind", ["dense", "tanh", "banana", "twisted5", "twisted6", "pi4"])
def test_small_targets_match_oracle(kind):
    """Small cases of every target kind, including the test targets of Sec. 3.1: pi_4 (a dense target of
    condition number d^2) and the twisted pi_5, pi_6 (u = V^T x through the FP64 product, then the twisted
    terms)."""
    if kind == "dense":
        ts, P = workloads.dense_gaussian(96, 11), 5
    elif kind == "tanh":
        ts, P = workloads.tanh_regression(130, 70, 12), 7
    elif kind.startswith("twisted"):
        ts, P = workloads.paper_targets(100)[int(kind[-1])], 5
    elif kind == "pi4":
        ts, P = workloads.paper_targets(100)[4], 5
    else:
        ts, P = workloads.banana(70), 3
    steps, nl = 320, 16
    if ts.uvar is not None:      # the Gaussian with the twisted target's exact first two moments
        C0 = (ts.G.T * ts.uvar) @ ts.G
    else:
        C0 = ts.cov if ts.cov is not None else np.diag(ts.lam)
    tol = TOL
    if kind in ("twisted5", "twisted6", "pi4"):
        # u = G x is an ill-conditioned sum here (G's rows up to 1e2 against states of 1e-2 along v_1): two FP64
        # summation orders differ by up to d u sum_k |G_mk x_k| per row each (Higham, Sec. 3.1), and log pi to first
        # order by 2 d u kappa relative, kappa = sum_m |dlog pi / du_m| sum_k |G_mk x_k| / |log pi| (taken over the
        # starting states, with a factor 8 for the spread of the states along the run)
        X = workloads.start_state(ts.d, P, 5) @ np.linalg.cholesky(C0).T
        U, Ua = X @ ts.G.T, np.abs(X) @ np.abs(ts.G.T)
        if ts.uvar is None:          # -|u|^2 / 2
            grad, lp = -U, -0.5 * np.sum(U * U, axis=1)
        else:                        # -sum_j (u_j + c_j u_{j-1}^2)^2 / (2 lam_j)
            ph = U.copy()
            ph[:, 1:] += ts.y[1:] * U[:, :-1] ** 2
            gph = -ph / ts.lam
            grad = gph.copy()
            grad[:, :-1] += gph[:, 1:] * 2.0 * ts.y[1:] * U[:, :-1]
            lp = -0.5 * np.sum(ph * ph / ts.lam, axis=1)
        kappa = np.max(np.sum(np.abs(grad) * Ua, axis=1) / np.abs(lp))
        tol = max(TOL, 16 * ts.d * U_EPS * kappa)
    x0 = workloads.start_state(ts.d, P, 5) @ np.linalg.cholesky(C0).T
    # eps_jitter 1e-3 keeps every refresh well conditioned (few samples per dimension early on), so the
    # two FP64 factorisations agree to rounding instead of to cond(C_n) * rounding
    g, o = make_pair(ts, P, trace_steps=steps, n_lag=nl, beta0=0.25, seed=21, min_samples_refresh=40, x0=x0,
                     C0=C0, eps_jitter=1e-3)
    g.run(100)
    g.run(steps - 100)      # a run that stops mid-interval and resumes
    o.run(steps)
    _compare(g, o, steps, tol=tol)
    assert o.counts()["refreshes"] >= 5


def test_refresh_delay_burnin_and_inflation_match_oracle():
    ts, P = workloads.dense_gaussian(200, 4), 3
    steps = 240
    x0 = workloads.start_state(200, P, 8) @ np.linalg.cholesky(ts.cov).T
    g, o = make_pair(ts, P, trace_steps=steps, n_lag=20, beta0=0.3, seed=5, min_samples_refresh=30,
                     refresh_delay=2, burnin=50, infl=1.2, x0=x0, C0=ts.cov, eps_jitter=1e-3)
    g.run(steps)
    o.run(steps)
    _compare(g, o, steps)


def test_reference_gaussian_accepts_every_proposal_on_gpu():
    d, P = 150, 4
    ts = workloads.TargetSpec(workloads.TARGET_REF, d)
    import paper_1506_05741_b300 as dm
    cfg = dm.default_config(d, P, n_lag=20, beta0=0.4, min_samples_refresh=20, infl=1.3, seed=3, eps_jitter=1e-3)
    cfg["trace_steps"] = 200
    g = dm.Sampler(cfg, ts, x0=workloads.start_state(d, P, 1))
    g.run(200)
    tr = g.trace(200)
    assert tr["acc"].all()
    assert np.abs(tr["loga"]).max() < 1e-9
    assert g.stats()["refreshes"] >= 5


def test_checkpoint_resume_is_bit_identical():
    ts, P = workloads.tanh_regression(96, 30, 2), 4
    import paper_1506_05741_b300 as dm
    cfg = dm.default_config(96, P, n_lag=10, beta0=0.3, seed=9, min_samples_refresh=20)
    cfg["keep_block_sums"] = 1
    a = dm.Sampler(cfg, ts)
    a.run(95)
    blob = a.save()
    a.run(105)
    b = dm.Sampler(cfg, ts)
    b.load(blob)
    b.run(105)
    xa, lpa, sa = a.state()
    xb, lpb, sb = b.state()
    assert np.array_equal(xa, xb) and np.array_equal(lpa, lpb) and sa == sb
    ma, ca, na = a.moments()
    mb, cb, nb = b.moments()
    assert np.array_equal(ma, mb) and np.array_equal(ca, cb) and na == nb
    xs_a, _ = a.block_sums(20)
    xs_b, _ = b.block_sums(20)
    assert np.array_equal(xs_a, xs_b)


def test_moment_merge_equals_pooled_samples():
    """eq. (mom2g), (mom1g): merging exported moments gives the moments of all samples pooled."""
    ts, P = workloads.diag_gaussian(40, 1.0), 2
    x0 = workloads.start_state(40, P, 3) * np.sqrt(ts.lam)
    kw = dict(n_lag=10, beta0=0.4, min_samples_refresh=10, eps_jitter=1e-3, x0=x0, C0=ts.cov)
    ga, oa = make_pair(ts, P, seed=1, **kw)
    gb, ob = make_pair(ts, P, seed=2, **kw)
    oa.run(100, record=True)
    ob.run(100, record=True)
    ga.run(100)
    gb.run(100)
    mb, M2b, nb = gb.export_moments()
    ga.sync_moments(mb, M2b, nb)
    m, cov, n = ga.moments()
    X = np.concatenate([oa.trajectory().reshape(-1, 40), ob.trajectory().reshape(-1, 40)])
    assert n == X.shape[0]
    assert np.max(np.abs(m - X.mean(0))) < 1e-11
    assert np.max(np.abs(cov - np.cov(X.T, bias=True))) < 1e-10 * np.max(np.abs(cov))


@pytest.mark.parametrize("prec", [0, 2])
def test_graph_replay_equals_eager_launches(prec):
    """Whole intervals replay one captured CUDA graph; the chains are bit-identical to eager launches."""
    import paper_1506_05741_b300 as dm
    ts, P = workloads.tanh_regression(128, 64, 3), 6
    out = []
    for graphs in (0, 1):
        cfg = dm.default_config(128, P, n_lag=8, beta0=0.3, seed=4, prec=prec, graphs=graphs, min_samples_refresh=20)
        s = dm.Sampler(cfg, ts, x0=workloads.start_state(128, P, 1) * np.sqrt(ts.lam), C0=np.diag(ts.lam))
        s.run(5)      # partial interval (eager), then whole intervals
        s.run(3 + 8 * 5)
        out.append((s.state(), s.moments()))
    (xa, la, sa), (ma, ca, na) = out[0]
    (xb, lb, sb), (mb, cb, nb) = out[1]
    assert np.array_equal(xa, xb) and np.array_equal(la, lb) and sa == sb
    assert np.array_equal(ma, mb) and np.array_equal(ca, cb) and na == nb


def test_psrf_matches_oracle_chains():
    """The device PSRF (Sec. 2.4.2) over a window of completed intervals equals eq. (winco)-(psrf) evaluated
    by the oracle's statistics on the oracle's own recorded trajectory (FP64 mode: the same chains)."""
    from oracle import stats
    d, P, nl = 48, 6, 16
    ts = workloads.dense_gaussian(d, 12)
    x0 = workloads.start_state(d, P, 2) * 3.0   # over-dispersed starts
    g, o = make_pair(ts, P, n_lag=nl, beta0=0.4, seed=9, min_samples_refresh=40, x0=x0, C0=ts.cov,
                     keep_block_sums=1)
    g.run(8 * nl)
    o.run(8 * nl, record=True)
    traj = o.trajectory()            # post-step states, (steps, P, d)
    for first, count in [(2, 6), (0, 8), (7, 1)]:
        win = traj[first * nl:(first + count) * nl]
        mean = win.mean(axis=0)
        var = ((win - mean) ** 2).mean(axis=0)
        want = stats.psrf(mean, var, count * nl)
        got = g.psrf(first, count)
        assert np.max(np.abs(got - want) / want) <= 1e-10, (first, count)
