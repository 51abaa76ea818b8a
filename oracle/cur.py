"""ORACLE -- test infrastructure only.

Plain FP64 numpy statement of the CUR choice of the sparse set (the cur_points option
of Secs. III-A and III-C, which cite Mahoney and Drineas, PNAS 106 (2009) 697).  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may use it; the GPU
library never does, and the two share no code.

Per species, the descriptor rows X of its atoms (atom order) are scored by their rank-k
leverage (Mahoney and Drineas, Eq. 3: the squared row norms of the k leading singular
vectors, divided by k), with the singular vectors taken from a randomised range finder
(Halko, Martinsson and Tropp, SIAM Rev. 53 (2011) 217: Alg. 4.4, power iterations with
a re-orthonormalisation after every product, then Alg. 5.1, the SVD of the small matrix
Q^T X).  The sparse points are drawn without replacement with probabilities
proportional to the scores by the key method of Efraimidis and Spirakis (IPL 97 (2006)
181): keep the m largest log(u_i) / pi_i.  Library steps: numpy's QR for orth, numpy's
symmetric eigensolver for the small SVD, a stable sort for the keys.
"""
from __future__ import annotations

import numpy as np


def range_basis(X: np.ndarray, omega: np.ndarray, power_iters: int) -> np.ndarray:
    """Orthonormal basis of range(X omega) after ``power_iters`` power iterations,
    Q <- orth(X X^T Q) (Halko et al., Alg. 4.4)."""
    Q, _ = np.linalg.qr(X @ omega)
    for _ in range(power_iters):
        Q, _ = np.linalg.qr(X @ (X.T @ Q))
    return Q


def leverage(X: np.ndarray, omega: np.ndarray, k: int, power_iters: int) -> np.ndarray:
    """Rank-k leverage scores pi_i = |U_k[i, :]|^2 / k of the rows of X, with U_k the k
    leading left singular vectors of Q Q^T X (Halko et al., Alg. 5.1: B = Q^T X,
    B B^T = W diag(lambda) W^T, U = Q W)."""
    Q = range_basis(X, omega, power_iters)
    B = Q.T @ X
    lam, W = np.linalg.eigh(B @ B.T)
    order = np.argsort(-lam, kind="stable")[:k]
    Uk = Q @ W[:, order]
    return (Uk * Uk).sum(axis=1) / k


def draw(pi: np.ndarray, u: np.ndarray, m: int) -> np.ndarray:
    """m distinct positions drawn without replacement with probabilities proportional
    to pi: the m largest keys log(u_i) / pi_i (-inf where pi_i = 0), ties to the lower
    position; returned ascending."""
    with np.errstate(divide="ignore"):
        key = np.where(pi > 0, np.log(u) / np.where(pi > 0, pi, 1.0), -np.inf)
    order = np.lexsort((np.arange(len(pi)), -key))  # key descending, then position
    return np.sort(order[:m])


def select_cur(X, atom_species, n_select, k, l, power_iters, omega, u):
    """The CUR sparse set of every species: (selected atom indices, species after
    species, ascending within each; leverage scores per atom, NaN for species with no
    sparse points)."""
    X = np.asarray(X, dtype=np.float64)
    n = X.shape[0]
    assert omega.shape == (X.shape[1], l) and 1 <= k <= l
    species = np.zeros(n, dtype=np.int64) if atom_species is None else np.asarray(atom_species)
    lev = np.full(n, np.nan)
    out = []
    for t, m in enumerate(n_select):
        if m == 0:
            continue
        atoms = np.nonzero(species == t)[0]
        pi = leverage(X[atoms], omega, k, power_iters)
        lev[atoms] = pi
        out.append(atoms[draw(pi, u[atoms], m)])
    sel = np.concatenate(out) if out else np.zeros(0, dtype=np.int64)
    return sel.astype(np.int64), lev
