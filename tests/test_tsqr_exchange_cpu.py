"""The exchange step of the fit over several GPUs (the row-block distribution of Sec.
III-B as a TSQR), run as two gloo processes on the CPU.

Each rank holds the configurations that greedy LPT places on it, factors their data rows
[Sigma^{-1/2} K_g | b_g] on its own (the oracle's Householder QR stands in for the
GPU's gap_tsqr_local here), and the product's ``exchange_blocks`` all-gathers the
[R_g | z_g] blocks and residual tails.  Every rank then factors the stack with U and
solves: both ranks must hold the same weights, equal to the oracle's fit of the whole
problem, with the whole fit's residual norm.  ``gap_tsqr_local`` and ``gap_tsqr_merge``
themselves are checked on the GPU against the same oracle fit."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import gapgen  # noqa: E402
import oracle  # noqa: E402
from paper_2207_03803_gb300.distributed import exchange_blocks, place_configurations  # noqa: E402


def _problem():
    r = gapgen.Recipe(n_cfg=14, atoms=(3, 12), d=11, n_sparse=(16,), zeta=3, delta=1.0, neighbours=(1, 6),
                      seed=91)
    p = gapgen.make_problem(r)
    return p, oracle.targets(p)


def _block_rows(p, cfgs):
    """Design-matrix rows of the given configurations: their energy rows, then the force
    rows of their atoms."""
    rows = [int(A) for A in cfgs]
    for A in cfgs:
        for a in range(p.cfg_ptr[A], p.cfg_ptr[A + 1]):
            rows += [p.n_cfg + 3 * a + al for al in range(3)]
    return np.array(rows, dtype=np.int64)


def test_configuration_placement_is_lpt():
    rows = [10, 3, 7, 7, 1]
    parts = place_configurations(rows, 2)
    assert [[int(a) for a in x] for x in parts] == [[0, 1, 4], [2, 3]]  # loads 14 and 14
    p, _ = _problem()
    sizes = 1 + 3 * np.diff(p.cfg_ptr)
    parts = place_configurations(sizes, 3)
    assert sorted(int(a) for q in parts for a in q) == list(range(p.n_cfg))
    loads = [int(sizes[q].sum()) for q in parts]
    assert max(loads) <= 4.0 / 3.0 * max(sum(loads) / 3, sizes.max())


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    p, y = _problem()
    M = p.n_sparse
    D = oracle.design(p)
    b = y / oracle.sigma(p)
    mine = place_configurations(1 + 3 * np.diff(p.cfg_ptr), world)[rank]
    rows = _block_rows(p, mine)
    QR, _ = oracle.householder_qr(np.hstack([D[rows], b[rows, None]]))
    top = np.triu(QR[:M + 1])
    Rz = np.ascontiguousarray(top[:M])                  # [R_g | z_g]
    tail2 = float(top[M, M]) ** 2 if len(rows) > M else 0.0
    stack, tails = exchange_blocks(torch.from_numpy(Rz), tail2)
    U = oracle.cholesky_upper(oracle.kmm(p))
    S = np.vstack([stack.numpy().reshape(world * M, M + 1), np.hstack([U, np.zeros((M, 1))])])
    QS, _ = oracle.householder_qr(S)
    c = oracle.back_substitution(np.triu(QS[:M, :M]), QS[:M, M])
    res = np.sqrt(QS[M, M] ** 2 + tails)
    q.put((rank, c, res, len(rows)))
    dist.destroy_process_group()


def test_row_blocks_exchange_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    res = sorted((q.get(timeout=300) for _ in range(2)), key=lambda x: x[0])
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    (_, c0, r0, n0), (_, c1, r1, n1) = res
    p, y = _problem()
    assert n0 + n1 == p.n_rows and min(n0, n1) > p.n_sparse
    assert np.array_equal(c0, c1)  # every rank merges the same stack
    c_or, _ = oracle.fit(p, y)
    assert np.linalg.norm(c0 - c_or) < 1e-9 * np.linalg.norm(c_or)
    A, _ = oracle.stacked_matrix(p)
    bb = np.concatenate([y / oracle.sigma(p), np.zeros(p.n_sparse)])
    assert abs(r0 - np.linalg.norm(bb - A @ c_or)) < 1e-9 * np.linalg.norm(bb)
