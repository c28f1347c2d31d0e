"""Pooling of moments across processes: the one exchange step of a pooled multi-GPU sampler.

A pool of samplers (one per process or GPU) shares one proposal factor built from the moments of every
member's samples (eq. (mom2g), (mom1g) of Sec. 2.4.1, with sample counts as weights). At every synchronisation
each member exports the moments of the samples it folded since the last one (``Sampler.export_increment``,
``diam_export_increment``), the members gather them over a torch.distributed group, and each member imports every
other member's increment into its own moments (``Sampler.sync_moments``, ``diam_sync_moments``). Each sample is
then counted once in every member's moments, and the merge arithmetic is the library's: this module only moves
arrays between processes.

``attach`` makes the synchronisation run at every interval end, after the interval's fold and before the refresh
that uses the moments (``Sampler.set_interval_hook``), so every member refreshes from the pooled moments.
"""
from __future__ import annotations

import numpy as np


def allgather_increments(sampler, group=None):
    """Every member's (mean, M2, n) increment, in rank order, gathered over the default (or given) group."""
    import torch
    import torch.distributed as dist
    mean, M2, n = sampler.export_increment()
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


def synchronise(sampler, group=None):
    """One synchronisation of the pool: import every other member's increment (the local one is already in)."""
    import torch.distributed as dist
    rank = dist.get_rank(group)
    parts = allgather_increments(sampler, group)
    imported = False
    for r, (m, M2, n) in enumerate(parts):
        if r != rank and n > 0:
            sampler.sync_moments(m, M2, n)
            imported = True
    if not imported:
        sampler.sync_moments()   # still a synchronisation point: the next increment counts from here


def attach(sampler, group=None):
    """Synchronise the pool at every interval end, before the refresh (all members must run the same steps)."""
    sampler.set_interval_hook(lambda interval: synchronise(sampler, group))
