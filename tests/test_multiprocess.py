"""The N > 1 host paths on CPU with gloo (world size 2): the exchange step of a pooled multi-process sampler
(every member's increment gathered and imported into every other member, pool.synchronise) and the bench's
cross-rank timing reduction. The samplers here are numpy stand-ins with the semantics of diam_export_increment
and diam_sync_moments (the library calls need a GPU; tests/test_gpu_pool.py drives them)."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _merge(a, b):
    """Moments of two disjoint sample sets, each as (mean, M2, n) (plain definition via the pooled sums)."""
    (ma, Ma, na), (mb, Mb, nb) = a, b
    if na == 0:
        return mb.copy(), Mb.copy(), nb
    if nb == 0:
        return ma.copy(), Ma.copy(), na
    n = na + nb
    S1 = na * ma + nb * mb
    S2 = Ma + na * np.outer(ma, ma) + Mb + nb * np.outer(mb, mb)   # raw second moments
    m = S1 / n
    return m, S2 - n * np.outer(m, m), n


def _moments(X):
    if X.shape[0] == 0:
        return np.zeros(X.shape[1]), np.zeros((X.shape[1], X.shape[1])), 0
    m = X.mean(axis=0)
    return m, (X - m).T @ (X - m), X.shape[0]


class _Member:
    """Stand-in sampler: fold(X) adds local samples; the two pooling calls behave as the library's."""

    def __init__(self, d):
        self.mom = (np.zeros(d), np.zeros((d, d)), 0)
        self.snap = self.mom

    def fold(self, X):
        self.mom = _merge(self.mom, _moments(X))

    def export_increment(self):
        (m, M2, n), (m0, M20, n0) = self.mom, self.snap
        ni = n - n0
        if ni == 0:
            return np.zeros_like(m), np.zeros_like(M2), 0
        mi = (n * m - n0 * m0) / ni
        dl = m0 - mi
        return mi, M2 - M20 - np.outer(dl, dl) * (n0 * ni / n), ni

    def sync_moments(self, m=None, M2=None, n=0):
        if n:
            self.mom = _merge(self.mom, (np.asarray(m), np.asarray(M2), n))
        self.snap = self.mom


def _samples(rank, k, d=6):
    rng = np.random.default_rng(1000 * rank + k)
    n = 20 + 13 * rank + 7 * k                 # uneven sample counts per rank and interval
    return rng.standard_normal((n, d)) * np.arange(1, d + 1) + rank


def _worker(rank, world, port):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_1506_05741_b300 import pool
        import bench
        s = _Member(6)
        for k in range(4):                     # four intervals, a synchronisation after each
            s.fold(_samples(rank, k))
            pool.synchronise(s)
            allX = np.concatenate([_samples(r, j) for j in range(k + 1) for r in range(world)])
            m, M2, n = s.mom
            assert n == allX.shape[0]           # every sample of every rank counted once
            assert np.allclose(m, allX.mean(axis=0), rtol=1e-12, atol=1e-12)
            assert np.allclose(M2, (allX - allX.mean(axis=0)).T @ (allX - allX.mean(axis=0)), rtol=1e-10, atol=1e-9)
        # the slowest replica sets the job's time
        assert bench.rank_max(1.5 + rank, world, "cpu") == 1.5 + (world - 1)
    finally:
        dist.destroy_process_group()


def test_two_ranks_pool_increments_and_reduce_timings():
    mp.spawn(_worker, args=(2, _free_port()), nprocs=2, join=True)


def test_increment_run_backwards_recovers_the_new_samples():
    """The stand-in's increment (the library's formula: the pairwise update run backwards) gives the moments of
    exactly the samples folded since the last synchronisation."""
    rng = np.random.default_rng(5)
    A = rng.standard_normal((300, 4)) @ rng.standard_normal((4, 4)) + 3.0
    B = rng.standard_normal((41, 4)) * 2.0 - 1.0
    s = _Member(4)
    s.fold(A)
    s.sync_moments()
    s.fold(B)
    m, M2, n = s.export_increment()
    mb, Mb, nb = _moments(B)
    assert n == nb and np.allclose(m, mb, rtol=1e-11) and np.allclose(M2, Mb, rtol=1e-9, atol=1e-9)
