"""The N > 1 host paths on CPU with gloo (world size 2): the exchange step of a pooled multi-process
sampler (every rank's moments gathered and merged) and the bench's cross-rank timing reduction."""
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


def _samples(rank, d=7):
    rng = np.random.default_rng(100 + rank)
    n = 50 + 37 * rank                       # uneven sample counts per rank
    return rng.standard_normal((n, d)) * np.arange(1, d + 1) + rank


def _worker(rank, world, port):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_1506_05741_b300 import pool
        import bench
        X = _samples(rank)
        m = X.mean(axis=0)
        M2 = (X - m).T @ (X - m)
        mean, M2p, n = pool.pooled_moments(m, M2, X.shape[0])
        allX = np.concatenate([_samples(r) for r in range(world)])
        want_m = allX.mean(axis=0)
        want_M2 = (allX - want_m).T @ (allX - want_m)
        assert n == allX.shape[0]
        assert np.allclose(mean, want_m, rtol=1e-13, atol=1e-13)
        assert np.allclose(M2p, want_M2, rtol=1e-12, atol=1e-10)
        # the slowest replica sets the job's time
        assert bench.rank_max(1.5 + rank, world, "cpu") == 1.5 + (world - 1)
    finally:
        dist.destroy_process_group()


def test_two_ranks_pool_moments_and_reduce_timings():
    mp.spawn(_worker, args=(2, _free_port()), nprocs=2, join=True)


def test_merge_moments_matches_pooled_samples_in_any_split():
    from paper_1506_05741_b300 import pool
    rng = np.random.default_rng(5)
    X = rng.standard_normal((300, 4)) @ rng.standard_normal((4, 4)) + 3.0
    cuts = [0, 1, 40, 41, 200, 300]
    parts = []
    for a, b in zip(cuts[:-1], cuts[1:]):
        Y = X[a:b]
        m = Y.mean(axis=0)
        parts.append((m, (Y - m).T @ (Y - m), Y.shape[0]))
    parts.append((np.zeros(4), np.zeros((4, 4)), 0))   # an empty rank
    mean, M2, n = pool.merge_moments(parts)
    assert n == 300
    assert np.allclose(mean, X.mean(axis=0), rtol=1e-13)
    Xc = X - X.mean(axis=0)
    assert np.allclose(M2, Xc.T @ Xc, rtol=1e-12)
