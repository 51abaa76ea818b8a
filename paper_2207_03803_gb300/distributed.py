"""The fit of one problem over several GPUs: the row-block distribution of the paper's
Sec. III-B as a TSQR over torch.distributed ranks.

Each rank assembles the configurations placed on it and factors its own data rows
(``gap_tsqr_local``); the ranks exchange their [R_g | Q_g^T b_g] blocks and residual
tails in one all-gather; every rank then factors the stack [R_1 z_1; ...; R_G z_G; U 0]
(``gap_tsqr_merge``) and solves, so all hold the same weights.  The blocks move as device
tensors through NCCL between GPUs (gloo serves CPU tensors); the exchange carries
G x M x (M + 1) numbers, independent of the rows.
"""
from __future__ import annotations

import numpy as np


def place_configurations(rows_per_cfg, world: int):
    """Configurations to ranks by greedy longest-processing-time on their design rows (the
    paper's load balancing, Sec. III-B): heaviest first, each to the least loaded rank,
    ties to the lower rank and the lower configuration.  Returns one sorted index array
    per rank."""
    rows = np.asarray(rows_per_cfg, dtype=np.int64)
    order = sorted(range(len(rows)), key=lambda a: (-int(rows[a]), a))
    load = [0] * world
    parts = [[] for _ in range(world)]
    for a in order:
        r = min(range(world), key=lambda k: (load[k], k))
        parts[r].append(a)
        load[r] += int(rows[a])
    return [np.array(sorted(p), dtype=np.int64) for p in parts]


def exchange_blocks(Rz, tail2: float, group=None):
    """All-gather of every rank's [R_g | z_g] block ([M, M + 1]) and residual tail: the
    stacked blocks [G, M, M + 1] in rank order and the sum of the tails, on every rank."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    blocks = [torch.empty_like(Rz) for _ in range(world)]
    dist.all_gather(blocks, Rz.contiguous(), group=group)
    t = torch.tensor([float(tail2)], dtype=torch.float64, device=Rz.device)
    tails = [torch.empty_like(t) for _ in range(world)]
    dist.all_gather(tails, t, group=group)
    return torch.stack(blocks).contiguous(), float(sum(x.item() for x in tails))


def fit_row_blocks(ctx, local_problem, c_out, group=None) -> dict:
    """One rank's part of the fit: assemble and factor this rank's rows, exchange, merge,
    solve.  ``ctx`` is an FP64 context on this rank's GPU, ``local_problem`` its
    configurations (the sparse set and hyperparameters the same on every rank), ``c_out``
    a device tensor [M] for the weights.  Returns the solve report (the residual norm is
    the whole fit's)."""
    import torch
    ctx.assemble(local_problem)
    M = c_out.shape[0]
    Rz = torch.empty((M, M + 1), dtype=torch.float64, device=c_out.device)
    tail2 = ctx.tsqr_local(Rz)
    stack, tails = exchange_blocks(Rz, tail2, group)
    ctx.tsqr_merge(stack, tails)
    return ctx.solve(c_out)
