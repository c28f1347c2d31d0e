"""Pooling of moments across processes (the one exchange step of a pooled multi-GPU sampler).

Each process exports its sampler's moments in mergeable form (mean, centred sum M2, sample count n; see
``Sampler.export_moments``); ``allgather_moments`` collects them from every rank of a torch.distributed group
and ``merge_moments`` combines them with the pairwise update of Chan, Golub and LeVeque (1979), the same
combination the library applies inside ``diam_sync_moments`` (the merge of eq. (mom2g)/(mom1g) with sample
counts as weights). Host-side numpy/torch only: the merged moments are handed back to a sampler through
``Sampler.sync_moments``.
"""
from __future__ import annotations

import numpy as np


def merge_moments(parts):
    """Combine [(mean, M2, n), ...] into one (mean, M2, n); parts with n = 0 are skipped."""
    mean, M2, n = None, None, 0
    for m_b, M2_b, n_b in parts:
        if n_b <= 0:
            continue
        m_b = np.asarray(m_b, np.float64)
        M2_b = np.asarray(M2_b, np.float64)
        if n == 0:
            mean, M2, n = m_b.copy(), M2_b.copy(), int(n_b)
            continue
        tot = n + n_b
        delta = m_b - mean
        M2 = M2 + M2_b + np.outer(delta, delta) * (n * n_b / tot)
        mean = mean + delta * (n_b / tot)
        n = tot
    return mean, M2, n


def allgather_moments(mean, M2, n, group=None):
    """Every rank's (mean, M2, n), in rank order, gathered over the default (or given) process group."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    d = int(np.asarray(mean).shape[0])
    flat = torch.from_numpy(np.concatenate([np.asarray(mean, np.float64).ravel(),
                                            np.asarray(M2, np.float64).ravel(), [float(n)]]))
    out = [torch.empty_like(flat) for _ in range(world)]
    dist.all_gather(out, flat, group=group)
    parts = []
    for t in out:
        a = t.numpy()
        parts.append((a[:d], a[d:d + d * d].reshape(d, d), int(round(a[-1]))))
    return parts


def pooled_moments(mean, M2, n, group=None):
    """The moments of the samples of every rank together (the same on every rank)."""
    return merge_moments(allgather_moments(mean, M2, n, group))
