"""BF16 (mixed-precision) CUDA path: the tcgen05 GEMM against torch's FP32-accumulated BF16 product, and the
sampler against the oracle run in its BF16 mode (same rounded factor A_q, same rounded noise W_q, same
rounded linear map). The CUDA side keeps FP32 states and FP32 accumulation, so agreement is to the FP32
level: log-densities and proposal quadratics within 1e-5 of max(1, |log pi|, |q|); log a within 1e-5 of
max(1, |log pi(x*) - log pi(x)|, |q* - q|), or within the FP32 rounding of the values it is formed from
(helpers.fp32_value_bound) where that is larger; accept decisions identical over the compared steps."""
import ctypes

import numpy as np
import pytest

import oracle
import workloads
from helpers import fp32_value_bound, loga_excess, make_pair, rel_err, trace_scale

pytestmark = pytest.mark.gpu
TOL = 1e-5


def _gemm(M, N, K, A, B, B2=None, a_lower=0, scale=1.0, bn=128):
    import torch
    import paper_1506_05741_b300 as dm
    l = dm.lib()
    f = l.diam_op_gemm_bf16_tile
    P, I32 = ctypes.c_void_p, ctypes.c_int32
    f.argtypes = [I32, I32, I32, P, I32, P, P, I32, I32, ctypes.c_float, P, I32, I32, P]
    f.restype = ctypes.c_int
    D = torch.zeros(N, M, dtype=torch.float32, device="cuda")
    rc = f(M, N, K, A.data_ptr(), A.shape[1], B.data_ptr(), None if B2 is None else B2.data_ptr(), B.shape[1],
           a_lower, scale, D.data_ptr(), M, bn, None)
    assert rc == 0, rc
    return D


@pytest.mark.parametrize("bn", [32, 64, 128, 256])
@pytest.mark.parametrize("M,N,K", [(128, 128, 64), (300, 200, 192), (130, 257, 128), (256, 32, 4096)])
def test_tc_gemm_matches_torch(M, N, K, bn):
    import torch
    g = torch.Generator(device="cuda").manual_seed(M + N + K)
    A = torch.randn(M, K, device="cuda", generator=g).to(torch.bfloat16)
    B = torch.randn(N, K, device="cuda", generator=g).to(torch.bfloat16)
    D = _gemm(M, N, K, A.view(torch.int16), B.view(torch.int16), scale=0.5, bn=bn)
    ref = 0.5 * (B.float() @ A.float().T)
    assert (D - ref).abs().max().item() <= 1e-5 * ref.abs().max().item() + 1e-6


def test_tc_gemm_second_operand_and_lower_triangle():
    import torch
    g = torch.Generator(device="cuda").manual_seed(7)
    M = K = 320
    N = 192
    A = torch.tril(torch.randn(M, K, device="cuda", generator=g)).to(torch.bfloat16)
    B = torch.randn(N, K, device="cuda", generator=g).to(torch.bfloat16)
    B2 = (torch.randn(N, K, device="cuda", generator=g) * 1e-3).to(torch.bfloat16)
    D = _gemm(M, N, K, A.view(torch.int16), B.view(torch.int16), B2.view(torch.int16), a_lower=1)
    ref = (B.float() + B2.float()) @ A.float().T
    assert (D - ref).abs().max().item() <= 1e-5 * ref.abs().max().item()


def _bf16_pair(ts, P, steps, **kw):
    import oracle as _o
    return make_pair(ts, P, trace_steps=steps, prec=_o.BF16, **kw)


@pytest.mark.parametrize("kind", ["tanh", "dense", "diag", "tanh_vec", "dense_vec", "tanh4096", "twisted", "banana",
                                  "banana_odd"])
def test_bf16_steps_match_oracle_bf16_mode(kind):
    """The map-carrying targets run as one fused launch per step: scalar element layout for d or d_y not a
    multiple of 4 (tanh, dense), 16-byte vectors otherwise (tanh_vec, dense_vec, with d past one element
    group per thread), and the chain's rows staged in shared memory by bulk copies (the vector cases; at
    d = 4096 they fill the 48 KB the kernel is set up for). The O(d) targets take the same fused kernels (diag;
    banana with d a multiple of 4, its head's two coordinates in one thread) or the per-step kernels (banana_odd)."""
    if kind == "tanh":
        ts, P = workloads.tanh_regression(200, 130, 31), 6
    elif kind == "dense":
        ts, P = workloads.dense_gaussian(150, 32), 5
    elif kind == "tanh_vec":
        ts, P = workloads.tanh_regression(2052, 132, 35), 4
    elif kind == "dense_vec":
        ts, P = workloads.dense_gaussian(160, 36), 5
    elif kind == "tanh4096":
        ts, P = workloads.tanh_regression(4096, 2048, 40), 3
    elif kind == "twisted":    # pi_6 of Sec. 3.1: the map through the tensor-core product, the twist in FP64
        ts, P = workloads.paper_targets(128)[6], 5
    elif kind == "banana":
        ts, P = workloads.banana(120), 4
    elif kind == "banana_odd":
        ts, P = workloads.banana(70), 3
    else:
        ts, P = workloads.diag_gaussian(100), 3
    d = ts.d
    steps = 6 if d > 2048 else 12
    C0 = np.diag(np.linspace(0.5, 1.5, d) * (ts.lam if ts.lam is not None else np.full(d, 0.01)))
    x0 = workloads.start_state(d, P, 4, scale=np.sqrt(np.diag(C0)))
    g, o = _bf16_pair(ts, P, steps, n_lag=8, beta0=0.3, seed=13, C0=C0, x0=x0, min_samples_refresh=10 ** 9)
    g.run(steps)
    o.run(steps)
    tg, to = g.trace(steps), o.trace()
    assert np.array_equal(tg["acc"], to["acc"])
    sc = trace_scale(to)
    for k in ("lp_prop", "q_prop", "q_cur"):   # values: against their own size
        assert rel_err(tg[k], to[k], sc) <= TOL, (k, rel_err(tg[k], to[k], sc))
    # log a: against the size of its two differences, or the FP32 rounding of the values they come from
    assert loga_excess(tg, to, fp32_value_bound(to)) <= 1.0, loga_excess(tg, to, fp32_value_bound(to))
    L, Lq, xr, _ = g.factor()
    Lo, Lqo, xro = o.factor()
    assert np.array_equal(Lq, Lqo) and np.array_equal(xr, xro)


@pytest.mark.parametrize("kind", ["tanh", "dense_vec", "diag"])
def test_fp32_factor_mode_matches_oracle(kind):
    """prec FP32: the factor quantised to TF32 (two BF16 terms, the second as an extra tensor-core K pass in the
    noise product and in A A_n), W and the map BF16, z solved by the FP64-accurate triangular solve; against the
    oracle's same mode over two intervals on the initial factor (C0's Cholesky factor quantised to TF32)."""
    import oracle as _o
    if kind == "tanh":
        ts, P = workloads.tanh_regression(256, 128, 61), 6
    elif kind == "dense_vec":
        ts, P = workloads.dense_gaussian(160, 62), 5
    else:
        ts, P = workloads.diag_gaussian(100), 4
    d, nl = ts.d, 8
    steps = 2 * nl
    C0 = np.diag(np.linspace(0.5, 1.5, d) * (ts.lam if ts.lam is not None else np.full(d, 0.01)))
    x0 = workloads.start_state(d, P, 6, scale=np.sqrt(np.diag(C0)))
    g, o = make_pair(ts, P, trace_steps=steps, prec=_o.FP32, n_lag=nl, beta0=0.3, seed=17, C0=C0, x0=x0,
                     min_samples_refresh=10 ** 9)
    L0, Lq0, _, _ = g.factor()
    assert np.array_equal(Lq0, _o.round_tf32(L0))                   # TF32, not BF16
    assert not np.array_equal(Lq0, _o.round_bf16(L0))
    g.run(steps)
    o.run(steps)
    tg, to = g.trace(steps), o.trace()
    assert np.array_equal(tg["acc"], to["acc"])
    sc = trace_scale(to)
    for k in ("lp_prop", "q_prop", "q_cur"):
        assert rel_err(tg[k], to[k], sc) <= TOL, (k, rel_err(tg[k], to[k], sc))
    assert loga_excess(tg, to, fp32_value_bound(to)) <= 1.0, loga_excess(tg, to, fp32_value_bound(to))
    g.close()


def test_bf16_refresh_and_moments_track_oracle():
    """One interval (64 steps of 16 chains: K = 1024 samples) folded by the BF16 tensor-core SYRK against the
    oracle's FP64 sums. The mean comes from the FP32 records: FP32 accuracy. The centred second moment multiplies
    the records rounded to BF16 (8-bit significand, round to nearest even: |delta| <= u = 2^-8 relative each)
    with FP32 accumulation: elementwise |dC_ij| <= (2u + u^2 + K 2^-24) sum_k |x_ik x_jk| / K in the worst
    case. The roundings are unbiased and independent across samples (relative standard deviation at most
    u / sqrt(3) each), so dC_ij has standard deviation at most u sqrt(2/3) sqrt(E[x_i^2 x_j^2] / K), with
    E[x_i^2 x_j^2] = C_ii C_jj + 2 C_ij^2 for a Gaussian; the largest of the 8515 entries is checked at 6 of
    them (~4 expected)."""
    ts, P, nl = workloads.dense_gaussian(130, 41), 16, 64
    g, o = _bf16_pair(ts, P, nl, n_lag=nl, beta0=0.3, seed=3, min_samples_refresh=10 ** 9,
                      x0=workloads.start_state(130, P, 2) @ np.linalg.cholesky(ts.cov).T, C0=ts.cov)
    g.run(nl)
    o.run(nl, record=True)
    assert np.array_equal(g.trace(nl)["acc"], o.trace()["acc"])
    mg, cg, n = g.moments()
    mo, co = o.moments()
    K = o.counts()["n"]
    assert n == K == nl * P
    assert np.max(np.abs(mg - mo)) <= 1e-5 * max(1e-3, np.max(np.abs(mo)))
    x0 = workloads.start_state(130, P, 2) @ np.linalg.cholesky(ts.cov).T
    X = o.trajectory().reshape(-1, 130) - x0.mean(axis=0)            # the records about the fold's centre
    u = 2.0 ** -8
    worst = (2 * u + u * u + K * 2.0 ** -24) * (np.abs(X).T @ np.abs(X)) / K
    X0 = o.trajectory().reshape(-1, 130) - mo
    worst = np.maximum(worst, (2 * u + u * u + K * 2.0 ** -24) * (np.abs(X0).T @ np.abs(X0)) / K)
    assert np.all(np.abs(cg - co) <= worst)
    var = np.diag(co)
    sd = u * np.sqrt(2.0 / 3.0) * np.sqrt((np.outer(var, var) + 2 * co * co) / K)
    assert np.max(np.abs(cg - co) / sd) <= 6.0, np.max(np.abs(cg - co) / sd)


@pytest.mark.parametrize("delay", [1, 2])
def test_refresh_delay_applies_the_factor_where_the_oracle_does(delay):
    """refresh_delay = 1 or 2 in BF16 mode (graphs on, so each factorisation runs on its own streams beside the
    following intervals). The factor built from interval 0's moments drives the chains from interval 1 + delay
    on: up to there decisions and log-densities follow the oracle, and both re-whiten exactly at step
    (1 + delay) n_lag (q of the current states stops being carried from the accepted proposals). Past that step
    the two factors come from differently rounded moments (BF16 records with FP32 accumulation against FP64),
    so the trajectories are not compared further."""
    ts, P, nl = workloads.tanh_regression(256, 128, 37), 8, 16
    steps = (2 + delay) * nl
    x0 = workloads.start_state(256, P, 5) * np.sqrt(ts.lam)
    g, o = _bf16_pair(ts, P, steps, n_lag=nl, beta0=0.3, seed=21, min_samples_refresh=30, refresh_delay=delay,
                      x0=x0, C0=np.diag(ts.lam))
    g.run(steps)
    o.run(steps)
    tg, to = g.trace(steps), o.trace()
    k = (1 + delay) * nl
    assert np.array_equal(tg["acc"][:k], to["acc"][:k])
    sc = trace_scale(to)[:k]
    for key in ("lp_prop", "q_prop", "q_cur"):
        assert rel_err(tg[key][:k], to[key][:k], sc) <= TOL, (key, rel_err(tg[key][:k], to[key][:k], sc))
    head, ohead = {key: v[:k] for key, v in tg.items()}, {key: v[:k] for key, v in to.items()}
    assert loga_excess(head, ohead, fp32_value_bound(ohead)) <= 1.0
    for tr in (tg, to):
        carried = np.where(tr["acc"], tr["q_prop"], tr["q_cur"])   # q of each step's outcome
        assert np.array_equal(tr["q_cur"][1:k], carried[:k - 1])   # no factor change before step 2 n_lag
        assert np.all(np.abs(tr["q_cur"][k] - carried[k - 1]) > 1e-6 * np.abs(carried[k - 1]))   # re-whitened
    assert g.stats()["refreshes"] == o.counts()["refreshes"] == 2 + delay


@pytest.mark.parametrize("mode", ["bf16", "fp32"])
@pytest.mark.parametrize("delay", [1, 2])
def test_refresh_beside_the_next_interval_equals_refresh_in_order(delay, mode):
    """The overlapped refreshes (graphs on; with delay 2 two are in flight) and the in-order ones (graphs off)
    give bit-identical chains, in BF16 mode and in the FP32 mode (the factor rounded to TF32)."""
    import paper_1506_05741_b300 as dm
    ts, P = workloads.tanh_regression(192, 64, 38), 6
    out = []
    for graphs in (0, 1):
        cfg = dm.default_config(192, P, n_lag=8, beta0=0.3, seed=6, prec=dm.BF16 if mode == "bf16" else dm.FP32,
                                graphs=graphs,
                                min_samples_refresh=20, refresh_delay=delay)
        s = dm.Sampler(cfg, ts, x0=workloads.start_state(192, P, 2) * np.sqrt(ts.lam), C0=np.diag(ts.lam))
        s.run(8 * 12 + 3)
        out.append((s.state(), s.moments(), s.stats()["refreshes"]))
        s.close()
    (xa, la, sa), (ma, ca, na), ra = out[0]
    (xb, lb, sb), (mb, cb, nb), rb = out[1]
    assert np.array_equal(xa, xb) and np.array_equal(la, lb) and sa == sb
    assert np.array_equal(ma, mb) and np.array_equal(ca, cb) and na == nb
    assert ra == rb >= 8


def test_reading_log_pi_between_intervals_leaves_refreshes_beside_them():
    """With refresh_delay 2 two factorisations run beside the intervals; reading log pi after every interval
    (diam_get_state with lp only) neither waits for them nor changes anything: the chains, log pi and the
    moments are bit-identical to a run that reads nothing in between, and the same refreshes happen."""
    import paper_1506_05741_b300 as dm
    ts, P, nl = workloads.tanh_regression(192, 64, 38), 6, 8
    out = []
    for read in (False, True):
        cfg = dm.default_config(192, P, n_lag=nl, beta0=0.3, seed=6, prec=dm.BF16, min_samples_refresh=20,
                                refresh_delay=2)
        s = dm.Sampler(cfg, ts, x0=workloads.start_state(192, P, 2) * np.sqrt(ts.lam), C0=np.diag(ts.lam))
        lps = []
        for _ in range(12):
            s.run(nl)
            if read:
                lps.append(s.log_pi())
        s.flush()
        out.append((s.state(), s.moments(), s.stats()["refreshes"], lps))
        s.close()
    (xa, la, sa), (ma, ca, na), ra, _ = out[0]
    (xb, lb, sb), (mb, cb, nb), rb, lps = out[1]
    assert np.array_equal(xa, xb) and np.array_equal(la, lb) and sa == sb
    assert np.array_equal(ma, mb) and np.array_equal(ca, cb) and na == nb
    assert ra == rb >= 8
    assert np.array_equal(lps[-1], lb)   # the last read is the final state's log pi


def test_bf16_interval_sums_equal_the_states_summed():
    """BF16 mode forms each interval's per-chain sums of x from the interval's records in the fold's pass
    (blocks of 32 chains: P = 40 leaves a partial block); they equal the states read back after every step
    and summed on the host, FP32-close, for intervals inside, across and past the burn-in."""
    import paper_1506_05741_b300 as dm
    d, P, nl = 96, 40, 8
    ts = workloads.tanh_regression(d, 48, 39)
    cfg = dm.default_config(d, P, n_lag=nl, beta0=0.4, seed=8, prec=dm.BF16, burnin=nl + 3, min_samples_refresh=30)
    cfg["keep_block_sums"] = 1
    s = dm.Sampler(cfg, ts, x0=workloads.start_state(d, P, 3) * np.sqrt(ts.lam), C0=np.diag(ts.lam))
    want = np.zeros((4, P, d))
    for t in range(4 * nl):
        s.run(1)
        x, _, _ = s.state()
        want[t // nl] += x
    s.run(3)   # a partial interval is not reported
    xs, _ = s.block_sums(10)
    assert xs.shape[0] == 4
    scale = np.abs(want).max()
    assert np.max(np.abs(xs - want)) <= 1e-5 * scale
    s.close()


def test_bf16_reference_gaussian_accepts_almost_every_proposal():
    d, P = 256, 8
    import paper_1506_05741_b300 as dm
    ts = workloads.TargetSpec(workloads.TARGET_REF, d)
    cfg = dm.default_config(d, P, n_lag=32, beta0=0.5, min_samples_refresh=64, seed=4, prec=2)
    cfg["trace_steps"] = 256
    g = dm.Sampler(cfg, ts, x0=workloads.start_state(d, P, 6))
    g.run(256)
    tr = g.trace(256)
    assert tr["acc"].mean() > 0.999
    assert np.abs(tr["loga"]).max() < 1e-3
    assert g.stats()["refreshes"] >= 3


@pytest.mark.parametrize("delay", [0, 2])
def test_multi_problem_run_equals_each_problem_alone(delay):
    """Problems of uneven d (dense Gaussians and bananas, BF16 mode) run together; each result equals the
    same problem run alone, bit for bit (refresh_delay 2: each factorisation beside the next intervals, on the
    problem's own streams, as the benchmark runs them)."""
    import paper_1506_05741_b300 as dm
    ds = [72, 200, 131, 64, 256, 97]
    targets, cfgs = [], []
    for j, d in enumerate(ds):
        targets.append(workloads.dense_gaussian(d, 900 + j) if j % 2 == 0 else workloads.banana(d))
        cfgs.append(dm.default_config(d, 8, n_lag=16, seed=50 + j, problem_id=j, prec=dm.BF16, min_samples_refresh=40,
                                      refresh_delay=delay))
    m = dm.MultiSampler(cfgs, targets)
    m.run(16 * 4 + 5)
    for j in range(len(ds)):
        s = dm.Sampler(cfgs[j], targets[j])
        s.run(16 * 4 + 5)
        xa, la, sa = m.views[j].state()
        xb, lb, sb = s.state()
        assert np.array_equal(xa, xb) and np.array_equal(la, lb) and sa == sb
        s.close()
    assert all(v.stats()["n"] == 16 * 4 * 8 for v in m.views)   # every problem folded its four intervals
    m.close()


def test_multi_problem_larger_problem_first():
    """Two dense Gaussians whose whole-interval kernels need more than the default 48 KB of shared memory, the
    larger created first: the kernel's shared-memory limit is a property of the kernel, shared by both
    problems, so the later, smaller problem must not lower it below what the first one launches with."""
    import paper_1506_05741_b300 as dm
    ds = [3600, 3200]
    targets = [workloads.dense_gaussian(d, 950 + j) for j, d in enumerate(ds)]
    cfgs = [dm.default_config(d, 4, n_lag=16, seed=60 + j, problem_id=j, prec=dm.BF16, min_samples_refresh=10 ** 9)
            for j, d in enumerate(ds)]
    m = dm.MultiSampler(cfgs, targets)
    m.run(2 * 16)
    for j in range(len(ds)):
        s = dm.Sampler(cfgs[j], targets[j])
        s.run(2 * 16)
        xa, la, _ = m.views[j].state()
        xb, lb, _ = s.state()
        assert np.array_equal(xa, xb) and np.array_equal(la, lb)
        s.close()
    m.close()


@pytest.mark.parametrize("prec", [0, 2])
def test_initial_log_density_after_upload(prec):
    """log pi of the starting states, for several samplers created one after another in one process (each
    reuses freed device memory): the target's arrays reach the device before the first kernel that reads them
    (every copy is ordered on the sampler's stream)."""
    import paper_1506_05741_b300 as dm
    d, dy, P = 2048, 1024, 64
    ts = workloads.tanh_regression(d, dy, 77)
    x0 = workloads.start_state(d, P, 3) * np.sqrt(ts.lam)
    A = oracle.round_bf16(ts.A) if prec == 2 else ts.A
    X = x0.astype(np.float32).astype(np.float64) if prec == 2 else x0
    want = -0.5 * np.sum(X * X / ts.lam, axis=1) - np.sum((ts.y - np.tanh(X @ A.T)) ** 2, axis=1) / (2 * ts.sigma ** 2)
    tol = 1e-5 if prec == 2 else 1e-12
    for _ in range(3):
        s = dm.Sampler(dm.default_config(d, P, n_lag=16, prec=prec), ts, x0=x0, C0=np.diag(ts.lam))
        lp = s.log_pi()
        s.close()
        assert np.max(np.abs(lp - want) / np.abs(want)) <= tol


def test_bf16_psrf_matches_the_states_read_back():
    """BF16 mode forms the PSRF's per-chain terms in the fold's pass over the records (sum and scatter about the
    interval mean, FP32); the device PSRF over a window equals eq. (winco)-(psrf) evaluated on the states read
    back after every step, to FP32 accuracy."""
    from oracle import stats
    import paper_1506_05741_b300 as dm
    d, P, nl = 64, 40, 8
    ts = workloads.tanh_regression(d, 32, 41)
    cfg = dm.default_config(d, P, n_lag=nl, beta0=0.4, seed=10, prec=dm.BF16, min_samples_refresh=30)
    cfg["keep_block_sums"] = 1
    s = dm.Sampler(cfg, ts, x0=workloads.start_state(d, P, 4) * 2.0 * np.sqrt(ts.lam), C0=np.diag(ts.lam))
    states = []
    for _ in range(6 * nl):
        s.run(1)
        states.append(s.state()[0])
    traj = np.array(states)
    for first, count in [(1, 5), (0, 6)]:
        win = traj[first * nl:(first + count) * nl]
        mean = win.mean(axis=0)
        var = ((win - mean) ** 2).mean(axis=0)
        want = stats.psrf(mean, var, count * nl)
        got = s.psrf(first, count)
        assert np.max(np.abs(got - want) / want) <= 1e-4, (first, count, np.max(np.abs(got - want) / want))
    s.close()


@pytest.mark.parametrize("mode", ["bf16", "fp32"])
def test_bf16_rewhitening_matches_fp64_solve(mode):
    """After a refresh, BF16 mode re-solves z = Lq^{-1}(x - x_ref) in FP32 (the states' precision): q of every
    chain at the interval start agrees with the FP64 forward substitution on the same factor and states to
    1e-5 relative (it is ~1e-6; the states themselves are FP32). The FP32 mode (the factor rounded to TF32, its
    products from two BF16 terms, z re-solved by the FP64-accurate triangular solve) to the same bar, with the
    refreshed factor rounded to TF32."""
    import scipy.linalg as sl
    import paper_1506_05741_b300 as dm
    import oracle as _o
    d, P, nl = 512, 8, 16
    ts = workloads.tanh_regression(d, 256, 42)
    cfg = dm.default_config(d, P, n_lag=nl, beta0=0.3, seed=12, prec=dm.BF16 if mode == "bf16" else dm.FP32,
                            min_samples_refresh=30)
    cfg["trace_steps"] = 5 * nl + 1
    s = dm.Sampler(cfg, ts, x0=workloads.start_state(d, P, 5) * np.sqrt(ts.lam), C0=np.diag(ts.lam))
    s.run(4 * nl)
    x, _, _ = s.state()
    s.run(1)                               # the interval start applies the new factor and re-whitens
    L, Lq, xr, _ = s.factor()
    assert s.stats()["refreshes"] >= 3
    assert np.array_equal(Lq, _o.round_bf16(L) if mode == "bf16" else _o.round_tf32(L))
    z = sl.solve_triangular(Lq, (x - xr).T, lower=True)
    q64 = 0.5 * np.sum(z * z, axis=0)
    qg = s.trace(4 * nl + 1)["q_cur"][4 * nl]
    assert np.max(np.abs(qg - q64) / q64) <= 1e-5
    s.close()


@pytest.mark.parametrize("mode", ["bf16", "fp32"])
def test_bf16_dense1024_chain_matches_closed_form_moments(mode):
    """The dense1024 target (d = 1024, Sigma = Q diag(1/i) Q^T) in BF16 mode (and in the FP32 mode: the factor
    quantised to TF32), P = 128, n_lag = 64, from exact
    draws of the target, with a fixed factor near Sigma (its eigenvalues scaled by seeded factors in [0.7, 1.4],
    so the quantised proposal is not reversible for the target and the test of eq. (accept) does the work), beta
    0.4, 400 intervals. The chains' states at the interval ends (second half, 25600 draws), rotated to Sigma's
    eigenbasis y = Q^T x: the coordinates of v_1 and v_d, their squares and |x|^2 within 4 batch-means standard
    errors of the closed forms (mean 0, variance lambda_i, E|x|^2 = tr Sigma), and the chi^2 aggregates of all
    1024 standardised means and second moments below their 99.9% quantile. (The adaptive run from A_0 = Id is
    far from Sigma after 2e4 steps, see the design notes: its first refreshes come from stuck, degenerate
    samples.)"""
    import scipy.stats
    from oracle import stats
    import paper_1506_05741_b300 as dm
    run = workloads.dense1024()
    ts = run.target
    d, P, nl, K = ts.d, run.P, run.n_lag, 400
    lam, Q = np.linalg.eigh(ts.cov)
    sfac = np.exp(np.random.default_rng(5).uniform(np.log(0.7), np.log(1.4), d))
    C0 = (Q * (lam * sfac)) @ Q.T
    x0 = workloads.start_state(d, P, 3) @ np.linalg.cholesky(ts.cov).T
    cfg = dm.default_config(d, P, n_lag=nl, beta0=0.4, seed=run.seed, prec=dm.BF16 if mode == "bf16" else dm.FP32,
                            adapt_beta=0, xref_mode=0, min_samples_refresh=10 ** 12)
    s = dm.Sampler(cfg, ts, x0=x0, C0=C0)
    Y = np.zeros((K, P, d), np.float32)
    for k in range(K):
        s.run(nl)
        Y[k] = s.state()[0] @ Q
    s.close()
    h = Y[K // 2:].astype(np.float64)
    zm = np.array([stats.mean_and_se(h[:, :, i]) for i in range(d)])
    zv = np.array([stats.mean_and_se(h[:, :, i] ** 2) for i in range(d)])
    for i in (0, d - 1):
        assert abs(zm[i, 0]) <= 4 * zm[i, 1]
        assert abs(zv[i, 0] - lam[i]) <= 4 * zv[i, 1]
    m2, se2 = stats.mean_and_se((h ** 2).sum(axis=2))
    assert abs(m2 - lam.sum()) <= 4 * se2
    q = scipy.stats.chi2.ppf(0.999, d)
    assert np.sum((zm[:, 0] / zm[:, 1]) ** 2) < q
    assert np.sum(((zv[:, 0] - lam) / zv[:, 1]) ** 2) < q
