"""The row-block (TSQR) reading of the distributed solve of Sec. III-B, checked on the
CPU with the oracle's own Householder QR: the data rows of [A | b] cut into blocks,
each block factored on its own, and the stack [R_1 z_1; ...; R_G z_G; U 0] factored
once more gives the normal matrix, the weights, |R| and the residual norm of the
one-matrix QR (the solution does not depend on which process holds which rows).
These pin the algebra that libgap's "tsqr_shards" factorisation runs on the GPU."""
import numpy as np
import pytest

import gapgen
import oracle


def _problem():
    r = gapgen.Recipe(n_cfg=9, atoms=(3, 12), d=11, n_sparse=(17,), zeta=3, delta=1.0, neighbours=(0, 6),
                      n_species=1, absval=True, seed=77)
    p = gapgen.make_problem(r)
    y = oracle.targets(p)
    return p, y


def _blocks(n, g):
    cuts = np.linspace(0, n, g + 1).round().astype(int)
    return [(int(a), int(b)) for a, b in zip(cuts[:-1], cuts[1:])]


def _tsqr(A_data, b_data, U, g):
    """R (M x M), z = (Q^T b)[:M] and the residual norm from G row blocks."""
    M = U.shape[0]
    stack, tails = [], []
    for a, b in _blocks(A_data.shape[0], g):
        QR, _ = oracle.householder_qr(np.hstack([A_data[a:b], b_data[a:b, None]]))
        top = np.triu(QR[:M + 1])  # R_g with Q_g^T b_g in column M; entry (M, M) = +-|tail_g|
        stack.append(top[:M])
        tails.append(top[M, M] if b - a > M else 0.0)
    stack.append(np.hstack([U, np.zeros((M, 1))]))
    S = np.vstack(stack)
    QR, _ = oracle.householder_qr(S)
    R = np.triu(QR[:M, :M])
    z = QR[:M, M]
    res = np.sqrt(QR[M, M] ** 2 + np.sum(np.square(tails)))
    return R, z, res, S


@pytest.mark.parametrize("g", [1, 2, 5])
def test_tsqr_stack_gives_the_one_matrix_solution(g):
    p, y = _problem()
    M = p.n_sparse
    A, U = oracle.stacked_matrix(p)
    b = np.concatenate([y / oracle.sigma(p), np.zeros(M)])
    N = p.n_rows
    assert N >= g * (M + 1)  # every block tall
    R, z, res, S = _tsqr(A[:N], b[:N], U, g)
    # the stack keeps A^T A and A^T b of [A | b] (only b^T b loses the block tails, which
    # the residual norm below accounts for)
    Ab = np.hstack([A, b[:, None]])
    G_s, G_a = (S.T @ S)[:M], (Ab.T @ Ab)[:M]
    assert np.abs(G_s - G_a).max() < 1e-12 * np.abs(G_a).max()
    # R agrees with the one-matrix QR up to the signs of its rows
    QR1, _ = oracle.householder_qr(A)
    R1 = np.triu(QR1[:M])
    assert np.linalg.norm(np.abs(R) - np.abs(R1)) < 1e-11 * np.linalg.norm(R1)
    # same weights as the oracle's fit, same residual norm as the direct evaluation
    c = oracle.back_substitution(R, z)
    c_or, _ = oracle.fit(p, y)
    assert np.linalg.norm(c - c_or) < 1e-9 * np.linalg.norm(c_or)
    assert abs(res - np.linalg.norm(b - A @ c_or)) < 1e-9 * res


def test_tsqr_of_a_permuted_row_order_is_the_same():
    """Configurations may go to any process: permuting the data rows before the cut
    changes the blocks, not the result."""
    p, y = _problem()
    M, N = p.n_sparse, p.n_rows
    A, U = oracle.stacked_matrix(p)
    b = y / oracle.sigma(p)
    perm = np.random.default_rng(5).permutation(N)
    R0, z0, res0, _ = _tsqr(A[:N], b, U, 3)
    R1, z1, res1, _ = _tsqr(A[:N][perm], b[perm], U, 3)
    c0, c1 = oracle.back_substitution(R0, z0), oracle.back_substitution(R1, z1)
    assert np.linalg.norm(c0 - c1) < 1e-9 * np.linalg.norm(c0)
    assert abs(res0 - res1) < 1e-9 * res0
