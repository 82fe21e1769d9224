"""Combining independent replicas (one process per GPU) of a KPM run.

The stochastic trace averages over all random vectors (Eq. (munr)).  Ranks
that ran disjoint sets of vectors (realisation index s = rank, so rank k uses
the counters (s R + r) N + i of the same generator) combine by the
vector-weighted mean of their moments, mu = sum_k w_k mu_k / sum_k w_k with w_k
the number of vectors of rank k: one all-reduce of M + 1 doubles after the
compute, no exchange on the data path.
"""
from __future__ import annotations

import numpy as np


def combine_moments(mu_local, n_vectors: int, group=None) -> np.ndarray:
    """Vector-weighted mean of the moments of all ranks of `group` (host arrays)."""
    import torch
    import torch.distributed as dist

    buf = np.concatenate([np.asarray(mu_local, dtype=np.float64) * float(n_vectors),
                          [float(n_vectors)]])
    t = torch.from_numpy(buf)
    if dist.get_backend(group) == "nccl":
        t = t.cuda()
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    t = t.cpu().numpy()
    return t[:-1] / t[-1]
