"""Failure paths, all injected on the host (no GPU fault, trap or hang is provoked):
  - moments made indefinite by an imported external M2 (diam_sync_moments): the refresh rule's retries all fail,
    the refresh is skipped and counted (DIAM_ENOTSPD is not fatal) and the factor in use stays as it was;
  - a user log-density callback (DIAM_T_CALLBACK) computing the dense Gaussian in torch on the sampler's stream:
    the chain equals the oracle's on the same target;
  - a callback that returns NaN or -inf for some proposals: those proposals are rejected and counted in
    diam_stats.nonfinite;
  - a callback that fails: diam_run_batch returns DIAM_ETARGET and the context refuses further work
    (DIAM_ESTATE)."""
import ctypes

import numpy as np
import pytest

import oracle
import workloads
from helpers import CFG_KEYS

pytestmark = pytest.mark.gpu


class _Dev:
    """A device buffer seen by torch through the CUDA array interface (no copy)."""

    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"shape": shape, "typestr": typestr, "data": (int(ptr), False),
                                         "version": 3, "strides": None, "stream": None}


class _CallbackTarget:
    """log pi(x) = -|G x|^2 / 2 evaluated by a callback, optionally poisoned: proposals with x_0 > cut get NaN,
    those with x_0 < -cut get -inf; fail_after > 0 makes the call number fail_after return DIAM_ETARGET."""
    kind = 5

    def __init__(self, G, cut=None, fail_after=0):
        import torch
        self.Gt = torch.from_numpy(np.ascontiguousarray(G)).cuda()
        self.cut, self.fail_after, self.calls = cut, fail_after, 0
        self.fn = self._call

    def _call(self, user, X, d, P, prec, lp_out, stream):
        import torch
        self.calls += 1
        if self.fail_after and self.calls >= self.fail_after:
            return 6
        with torch.cuda.stream(torch.cuda.ExternalStream(stream)):
            Xt = torch.as_tensor(_Dev(X, (P, d), "<f8" if prec == 0 else "<f4"), device="cuda").double()
            lp = -0.5 * ((Xt @ self.Gt.T) ** 2).sum(dim=1)
            if self.cut is not None:
                lp = torch.where(Xt[:, 0] > self.cut, torch.full_like(lp, float("nan")), lp)
                lp = torch.where(Xt[:, 0] < -self.cut, torch.full_like(lp, float("-inf")), lp)
            torch.as_tensor(_Dev(lp_out, (P,), "<f8"), device="cuda").copy_(lp)
        return 0


def test_indefinite_moments_skip_the_refresh_and_keep_the_factor():
    import paper_1506_05741_b300 as dm
    d, P, nl = 24, 4, 20
    ts = workloads.dense_gaussian(d, 5)
    cfg = dm.default_config(d, P, n_lag=nl, beta0=0.4, seed=2, min_samples_refresh=30)
    s = dm.Sampler(cfg, ts, x0=workloads.start_state(d, P, 1) @ np.linalg.cholesky(ts.cov).T, C0=ts.cov)
    s.run(3 * nl)                                   # refreshes at the ends of intervals 0, 1, 2
    st0 = s.stats()
    assert st0["refreshes"] == 3 and st0["notspd"] == 0
    _, _, n = s.moments()
    s.sync_moments(np.zeros(d), -1e3 * n * np.eye(d), 10)    # host-injected fault: an indefinite scatter
    s.run(nl)                                       # interval 3 runs on interval 2's factor; its refresh fails
    L3 = s.factor()[0]
    st = s.stats()
    assert st["notspd"] == 1 and st["refreshes"] == 3
    assert st["chol_attempts"] == st0["chol_attempts"] + 4          # the first try and its three retries
    s.run(nl)                                       # no new factor was queued: interval 4 keeps it
    assert np.array_equal(s.factor()[0], L3)
    assert s.stats()["notspd"] == 2
    s.close()


def _callback_pair(G, P, steps, **kw):
    import paper_1506_05741_b300 as dm
    d = G.shape[1]
    cfg = dm.default_config(d, P, n_lag=16, beta0=0.35, seed=44, min_samples_refresh=30, eps_jitter=1e-3)
    cfg["trace_steps"] = steps
    x0 = workloads.start_state(d, P, 4) * 0.05      # inside the poisoned callback's finite region
    C0 = np.linalg.inv(G.T @ G)                     # the target's covariance: a factor the chains move with
    cb = _CallbackTarget(G, **kw)
    g = dm.Sampler(cfg, cb, x0=x0, C0=C0)
    ocfg = oracle.default_config(**{k: cfg[k] for k in CFG_KEYS})
    ocfg.update(trace_steps=steps, threads=2)
    o = oracle.Sampler(ocfg, oracle.Target(oracle.T_DENSE, d, G.shape[0], G=G), x0=x0, C0=C0)
    return g, o, cb


def test_callback_target_matches_oracle():
    ts = workloads.dense_gaussian(40, 6)
    steps = 160
    g, o, cb = _callback_pair(ts.G, 5, steps)
    g.run(steps)
    o.run(steps)
    tg, to = g.trace(steps), o.trace()
    assert np.array_equal(tg["acc"], to["acc"])
    sc = np.maximum.reduce([np.abs(to["lp_prop"]), np.abs(to["q_prop"]), np.abs(to["q_cur"]), np.ones_like(to["q_cur"])])
    assert np.max(np.abs(tg["lp_prop"] - to["lp_prop"]) / sc) <= 1e-12
    assert np.max(np.abs(tg["loga"] - to["loga"]) / sc) <= 1e-10
    assert g.stats()["refreshes"] >= 3 and cb.calls >= steps
    g.close()


def test_callback_nan_and_minus_inf_proposals_are_rejected_and_counted():
    ts = workloads.dense_gaussian(40, 6)
    steps = 160
    g, _, cb = _callback_pair(ts.G, 5, steps, cut=0.25)
    g.run(steps)
    tr = g.trace(steps)
    bad = ~np.isfinite(tr["lp_prop"])
    assert np.isnan(tr["lp_prop"]).any() and np.isneginf(tr["lp_prop"]).any()
    assert not np.any(tr["acc"] & bad)              # never accepted
    assert g.stats()["nonfinite"] == int(bad.sum())
    x, lp, _ = g.state()
    assert np.all(np.isfinite(lp)) and np.all(np.abs(x[:, 0]) <= 0.25 + 1e-12)
    g.close()


@pytest.mark.parametrize("prec", [0, 2])
def test_callback_failure_stops_the_run(prec):
    import paper_1506_05741_b300 as dm
    ts = workloads.dense_gaussian(32, 7)
    cfg = dm.default_config(32, 4, n_lag=8, beta0=0.3, seed=1, prec=prec)
    cb = _CallbackTarget(ts.G, fail_after=10)
    s = dm.Sampler(cfg, cb)                         # call 1: log pi of the starting states
    with pytest.raises(dm.DiamError) as e:
        s.run(40)
    assert e.value.status == 6                       # DIAM_ETARGET
    with pytest.raises(dm.DiamError) as e2:
        s.run(1)
    assert e2.value.status == 7                      # DIAM_ESTATE: the context refuses further work
    s.close()


def test_bounded_device_wait_reports_timeout_and_leaves_the_device_usable():
    """The bounded wait (diam_op_wait_flag) on a flag that nothing sets gives up after its short runtime limit
    with DIAM_ETIMEOUT instead of hanging; nothing is left in flight (the device synchronises), the same wait
    succeeds once the flag is set, and a sampler still runs afterwards."""
    import torch
    import paper_1506_05741_b300 as dm
    l = dm.lib()
    f = l.diam_op_wait_flag
    f.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p]
    f.restype = ctypes.c_int
    flag = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert f(flag.data_ptr(), 1, 2_000_000, None) == 5            # DIAM_ETIMEOUT after ~1 ms of clock
    torch.cuda.synchronize()                                       # nothing left running
    flag.fill_(1)
    torch.cuda.synchronize()
    assert f(flag.data_ptr(), 1, 2_000_000, None) == 0
    assert f(flag.data_ptr(), 1, -1, None) == 1                   # DIAM_EINVAL: a negative limit
    ts = workloads.dense_gaussian(32, 3)
    s = dm.Sampler(dm.default_config(32, 4, n_lag=8, seed=5), ts, C0=ts.cov)
    s.run(24)
    assert s.stats()["steps"] == 24
    s.close()
