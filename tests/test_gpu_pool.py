"""A pool of two samplers sharing one factor (Sec. 2.4.1 across processes or GPUs), driven through the library:
each runs in its own host thread, and at every interval end its hook (diam_set_interval_hook) exports the
increment (diam_export_increment), waits for the other's and imports it (diam_sync_moments), before the refresh.
Both then refresh from the moments of both samplers' samples, each counted once (eq. (mom2g), (mom1g))."""
import threading

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", [0, 2])
def test_two_samplers_pool_their_moments_before_every_refresh(prec):
    import paper_1506_05741_b300 as dm
    d, P, nl, K = 48, 6, 16, 5
    ts = workloads.dense_gaussian(d, 21)
    members = []
    for j in range(2):
        cfg = dm.default_config(d, P, n_lag=nl, beta0=0.4, seed=30 + j, prec=prec, min_samples_refresh=40)
        cfg["keep_block_sums"] = 1
        members.append(dm.Sampler(cfg, ts, x0=workloads.start_state(d, P, 9 + j) @ np.linalg.cholesky(ts.cov).T,
                                  C0=ts.cov))
    box = [None, None]
    bar = threading.Barrier(2, timeout=120)

    def hook_for(j):
        def hook(k):
            box[j] = members[j].export_increment()
            bar.wait()
            m, M2, n = box[1 - j]
            bar.wait()                       # both have read before either box is overwritten
            members[j].sync_moments(m, M2, n)
        return hook

    for j in range(2):
        members[j].set_interval_hook(hook_for(j))
    errs = []

    def run(j):
        try:
            members[j].run(K * nl)
        except BaseException as e:           # pragma: no cover - reported below
            errs.append(e)
            bar.abort()

    th = [threading.Thread(target=run, args=(j,)) for j in range(2)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    assert not errs, errs
    (ma, Ca, na), (mb, Cb, nb) = members[0].moments(), members[1].moments()
    assert na == nb == 2 * K * nl * P                     # every sample of both samplers, once
    tot = sum(members[j].block_sums(K)[0].sum(axis=(0, 1)) for j in range(2))
    scale = np.abs(tot / na).max()
    assert np.max(np.abs(ma - tot / na)) <= (1e-10 if prec == 0 else 1e-5) * scale
    assert np.max(np.abs(ma - mb)) <= 1e-12 * scale
    assert np.max(np.abs(Ca - Cb)) <= 1e-10 * np.abs(Ca).max()
    La, Lb = members[0].factor()[0], members[1].factor()[0]
    assert members[0].stats()["refreshes"] >= 2
    assert np.max(np.abs(La - Lb)) <= 1e-8 * np.abs(La).max()   # one factor for the pool (merge order aside)
    for s in members:
        s.close()
