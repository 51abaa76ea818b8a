"""Placement of independent fits on ranks (one process per GPU).

A sweep of independent fits shards without any exchange between ranks: each rank
fits whole problems on its own GPU.  The fits are placed by greedy longest-processing-
time first (LPT), the paper's load balancing of configurations over processes
(Sec. III): fits in descending estimated cost, each to the rank with the least work
so far.  Ties go to the lower fit index and the lower rank, so every rank computes
the same placement without communicating.
"""
from typing import List, Sequence


def lpt_assign(costs: Sequence[float], n_ranks: int) -> List[List[int]]:
    """Fit indices per rank, by greedy LPT on ``costs``."""
    if n_ranks < 1:
        raise ValueError("n_ranks must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i))
    loads = [0.0] * n_ranks
    out: List[List[int]] = [[] for _ in range(n_ranks)]
    for i in order:
        r = min(range(n_ranks), key=lambda k: (loads[k], k))
        out[r].append(i)
        loads[r] += float(costs[i])
    return out


def fit_cost(n_rows: int, n_sparse: int) -> float:
    """Estimated work of one fit: its QR, 2 N M^2 (the dominant term at sweep sizes)."""
    return 2.0 * float(n_rows) * float(n_sparse) ** 2
