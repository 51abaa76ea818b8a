"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics,
independent of the oracle's own loops (CPU only).

Each test names the passage of arXiv:2207.03803 it checks.  A plausible slip in
the oracle (a dropped term, a flipped sign, a wrong index or a transposed
operand) changes at least one of these numbers far beyond its tolerance;
``test_planted_mistakes_are_caught`` compiles mutated copies of the oracle and
checks exactly that.
"""
import json
import os
from fractions import Fraction

import numpy as np
import pytest
import scipy.linalg

import gapgen
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def small(seed=11, n_cfg=6, atoms=(3, 7), d=8, M=5, zeta=3, forces=True, absval=True, n_species=1,
          sparse=None, delta=1.0, jitter=1e-8, virials=False):
    r = gapgen.Recipe(n_cfg=n_cfg, atoms=atoms, d=d, n_sparse=sparse or (M,), zeta=zeta, delta=delta,
                      absval=absval, neighbours=(2, 5) if forces else None, n_species=n_species,
                      jitter=jitter, seed=seed, virials=virials)
    return gapgen.make_problem(r)


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


# ---------------------------------------------------------------- generator --

def test_generator_is_deterministic_and_normalised():
    a = small(seed=5)
    b = small(seed=5)
    for k in ("cfg_ptr", "X", "sparse_idx", "pair_ptr", "pair_src", "J", "c_star", "noise_e", "noise_f"):
        assert np.array_equal(getattr(a, k), getattr(b, k)), k
    assert np.allclose(np.linalg.norm(a.X, axis=1), 1.0, atol=1e-15)
    assert (a.X >= 0).all()
    assert len(set(a.sparse_idx.tolist())) == a.n_sparse
    c = small(seed=6)
    assert not np.array_equal(a.X[:3], c.X[:3])


def test_generator_log_and_normals():
    xs = np.geomspace(1e-300, 1.0, 2001)[:-1]
    errs = [abs(gapgen.gen_log(x) - np.log(x)) / abs(np.log(x)) for x in xs]
    assert max(errs) < 4e-16
    z = gapgen.normals(3, 1, 400000)
    assert abs(z.mean()) < 5e-3 and abs(z.std() - 1) < 5e-3
    # fourth moment of N(0,1) is 3
    assert abs(np.mean(z ** 4) - 3.0) < 0.05


def test_workload_shapes():
    # workload 2: 2000 configurations of 16-128 atoms, 8-24 neighbours per atom
    n_atoms, n_pairs = gapgen.count_shape(gapgen.RECIPES[2])
    assert 2000 * 16 <= n_atoms <= 2000 * 128
    assert abs(n_atoms / 2000 - 72) < 3 and abs(n_pairs / n_atoms - 16) < 0.2


# -------------------------------------------------------------- paper sizes --

def test_paper_printed_sizes():
    """Sec. IV.A/B: N = energies + forces + virials, M from the sub-GAP sparse
    counts, and A of (N+M) x M FP64 elements (Eq. 7) -- the printed counts."""
    g = json.load(open(os.path.join(GOLDEN, "paper_sizes.json")))
    for name in ("HEA", "SiC"):
        s = g[name]
        assert s["energies"] + s["forces"] + s["virials"] == s["N"]
        two, soap = s["sparse"]["two_body"], s["sparse"]["soap"]
        assert two[0] * two[1] + soap[0] * soap[1] == s["M"]
        assert (s["N"] + s["M"]) * s["M"] == s["n_A"]
        assert round(s["n_A"] * 8 / 1e9, 1) == s["GB"]
        assert s["forces"] % 3 == 0  # three force rows per atom


# ---------------------------------------------------------- design matrix --

def test_energy_rows_zeta1_are_a_matrix_product():
    """Eq. (6) with zeta=1: K_{A,s} = sum_{i in A} x_i . x_s, i.e. S X Xs^T."""
    p = small(zeta=1, forces=False, delta=1.7)
    S = np.zeros((p.n_cfg, p.n_atoms))
    for A in range(p.n_cfg):
        S[A, p.cfg_ptr[A]:p.cfg_ptr[A + 1]] = 1.0
    ref = (1.7 ** 2) * (S @ p.X @ p.Xs.T) / p.sigma_e[:, None]
    assert rel(oracle.design(p), ref) < 1e-14


def test_energy_rows_species_mask():
    """Different species do not interact: zeta=1 closed form with a species mask."""
    p = small(zeta=1, forces=False, n_species=2, sparse=(3, 3), n_cfg=8, atoms=(6, 9))
    mask = (p.atom_species[:, None] == p.sparse_species[None, :]).astype(float)
    G = (p.X @ p.Xs.T) * mask
    ref = np.add.reduceat(G, p.cfg_ptr[:-1], axis=0) / p.sigma_e[:, None]
    assert rel(oracle.design(p), ref) < 1e-14


def test_zeta2_prediction_closed_form():
    """Eq. (2) with zeta=2: eps(x) = delta^2 x^T (sum_s c_s x_s x_s^T) x."""
    p = small(zeta=2, forces=False, delta=0.3)
    c = np.linspace(-1, 1, p.n_sparse)
    C = (p.Xs.T * c) @ p.Xs
    eps = 0.09 * np.einsum("ik,kl,il->i", p.X, C, p.X)
    E_ref = np.add.reduceat(eps, p.cfg_ptr[:-1])
    E, _ = oracle.predict(p, c)
    assert rel(E, E_ref) < 1e-13


def test_prediction_equals_design_rows_times_c():
    """Predictions (Eqs. 1, 2 and the force chain rule) equal Sigma^{1/2} K c row
    by row: the design rows and the model agree."""
    p = small(zeta=3)
    c = gapgen.normals(9, 1, p.n_sparse)
    K = oracle.design(p) * oracle.sigma(p)[:, None]
    E, F = oracle.predict(p, c)
    assert rel(K[:p.n_cfg] @ c, E) < 1e-13
    assert rel(K[p.n_cfg:] @ c, F) < 1e-12


@pytest.mark.parametrize("zeta", [1, 2, 4])
def test_force_rows_finite_differences(zeta):
    """Force rows are -dE/dr (Sec. II): central differences of the energy with
    every x_i moved along h * d x_i/d r_{a,alpha} = h J_p[alpha]."""
    p = small(zeta=zeta, n_cfg=3, atoms=(3, 5))
    c = gapgen.normals(4, 1, p.n_sparse)
    K = oracle.design(p) * oracle.sigma(p)[:, None]
    h = 1e-5
    X0 = p.X.copy()
    for a in range(p.n_atoms):
        A = int(np.searchsorted(p.cfg_ptr, a, side="right") - 1)
        for al in range(3):
            dX = np.zeros_like(X0)
            for q in range(p.pair_ptr[a], p.pair_ptr[a + 1]):
                dX[p.pair_src[q]] += p.J[q, al]
            p.X = X0 + h * dX
            Ep, _ = oracle.predict(p, c, with_forces=False)
            p.X = X0 - h * dX
            Em, _ = oracle.predict(p, c, with_forces=False)
            p.X = X0
            fd = -(Ep[A] - Em[A]) / (2 * h)
            row = K[p.n_cfg + 3 * a + al] @ c
            assert abs(row - fd) <= 1e-7 * max(1.0, abs(fd)), (a, al, row, fd)


# ------------------------------------------------------- K_MM and Cholesky --

def test_kmm_symmetric_positive_definite_and_cholesky():
    """K_MM symmetric with jitter on the diagonal; K_MM = U^T U (Eq. 7: U = L_MM^T)."""
    p = small(M=12, d=16, atoms=(6, 9), zeta=4, jitter=1e-8)
    K = oracle.kmm(p)
    assert np.array_equal(K, K.T)
    G = p.Xs @ p.Xs.T
    assert rel(K, G ** 4 + 1e-8 * np.eye(12)) < 1e-14
    w = np.linalg.eigvalsh(K)
    assert w[0] > 0
    U = oracle.cholesky_upper(K)
    assert np.array_equal(np.triu(U), U)
    assert rel(U, np.linalg.cholesky(K).T) < 1e-13
    assert rel(U.T @ U, K) < 1e-14


def test_cholesky_reports_indefinite_pivot():
    K = np.array([[4.0, 2.0, 0.0], [2.0, 1.0, 0.0], [0.0, 0.0, 1.0]])
    with pytest.raises(oracle.OracleError, match="pivot 1"):
        oracle.cholesky_upper(K)


# ---------------------------------------------------------------- QR route --

def test_householder_matches_lapack_geqrf():
    """The reflectors, tau and R of the oracle are LAPACK dgeqrf's (the routine
    whose distributed form pdgeqrf the paper calls, Sec. III.B)."""
    rng = np.random.default_rng(0)
    A = rng.standard_normal((37, 9))
    A[:, 3] *= -1e3
    QR, tau = oracle.householder_qr(A)
    (qr_f, tau_l), _ = scipy.linalg.qr(A, mode="raw")
    assert rel(QR, qr_f) < 1e-13
    assert rel(tau, tau_l) < 1e-13


def test_qr_orthogonality_and_reconstruction():
    """Q^T Q = I (Eq. 11) and A = QR with R upper triangular."""
    rng = np.random.default_rng(1)
    A = rng.standard_normal((30, 7))
    QR, tau = oracle.householder_qr(A)
    R = np.triu(QR[:7])
    Q = np.stack([oracle.apply_q(QR, tau, np.eye(30)[:, j]) for j in range(30)], axis=1)
    assert np.abs(Q.T @ Q - np.eye(30)).max() < 1e-14
    assert rel(Q[:, :7] @ R, A) < 1e-14
    Qtb = oracle.apply_qt(QR, tau, A[:, 2])
    assert rel(Qtb[:7], R[:, 2]) < 1e-14 and np.abs(Qtb[7:]).max() < 1e-13


def test_back_substitution_matches_triangular_solve():
    rng = np.random.default_rng(2)
    R = np.triu(rng.standard_normal((9, 9))) + 4 * np.eye(9)
    z = rng.standard_normal(9)
    assert rel(oracle.back_substitution(R, z), scipy.linalg.solve_triangular(R, z)) < 1e-14
    R[4, 4] = 0.0
    with pytest.raises(oracle.OracleError):
        oracle.back_substitution(R, z)


def _normal_equation_solution(p, y):
    """Eq. (4): (K_MM + K_MN Sigma^-1 K_NM) c = K_MN Sigma^-1 y, by LAPACK gesv."""
    D = oracle.design(p)                  # Sigma^-1/2 K_NM
    s = oracle.sigma(p)
    lhs = oracle.kmm(p) + D.T @ D
    rhs = D.T @ (y / s)
    return np.linalg.solve(lhs, rhs)


@pytest.mark.parametrize("forces,virials", [(False, False), (True, False), (True, True)])
def test_qr_solution_equals_normal_equations(forces, virials):
    p = small(forces=forces, n_cfg=10, M=6, d=12, zeta=2, virials=virials)
    y = oracle.targets(p)
    c, _ = oracle.fit(p, y)
    assert rel(c, _normal_equation_solution(p, y)) < 1e-9


def test_qr_solution_against_exact_rational_least_squares():
    """The exact minimiser of ||Ac - b|| (Eqs. 9, 10) for the FP64 matrix A, by
    Gaussian elimination in rational arithmetic: pins the oracle's digits."""
    p = small(forces=True, n_cfg=3, atoms=(3, 4), M=5, d=6, zeta=2)
    y = oracle.targets(p)
    A, _ = oracle.stacked_matrix(p)
    b = np.concatenate([y / oracle.sigma(p), np.zeros(p.n_sparse)])
    Af = [[Fraction(float(v)) for v in row] for row in A]
    bf = [Fraction(float(v)) for v in b]
    n = A.shape[1]
    G = [[sum(Af[k][i] * Af[k][j] for k in range(len(Af))) for j in range(n)] for i in range(n)]
    h = [sum(Af[k][i] * bf[k] for k in range(len(Af))) for i in range(n)]
    for i in range(n):                               # exact Gaussian elimination
        for r in range(i + 1, n):
            f = G[r][i] / G[i][i]
            for j in range(i, n):
                G[r][j] -= f * G[i][j]
            h[r] -= f * h[i]
    x = [Fraction(0)] * n
    for i in reversed(range(n)):
        x[i] = (h[i] - sum(G[i][j] * x[j] for j in range(i + 1, n))) / G[i][i]
    exact = np.array([float(v) for v in x])
    c, _ = oracle.fit(p, y)
    cond = np.linalg.cond(A)
    assert rel(c, exact) < 50 * cond * 2.2e-16


def test_loss_gradient_vanishes_at_solution():
    """Eq. (3): dL/dc = 2[(K_MM) c - K_MN Sigma^-1 (y - K_NM c)] = 0 at the fit."""
    p = small(forces=True, n_cfg=12, M=8, d=10, zeta=3)
    y = oracle.targets(p)
    c, _ = oracle.fit(p, y)
    D = oracle.design(p)
    s = oracle.sigma(p)
    g = oracle.kmm(p) @ c - D.T @ (y / s - D @ c)
    assert np.linalg.norm(g) < 1e-9 * np.linalg.norm(D.T @ (y / s))


# ---------------------------------------------------------------- invariants --

def test_configuration_permutation_invariance():
    """Sec. III.B: swapping rows of A with the matching entries of b leaves the
    solution unchanged -- here whole configurations are reordered."""
    p = small(forces=True, n_cfg=7, M=6, d=10, zeta=2)
    y = oracle.targets(p)
    c, _ = oracle.fit(p, y)
    perm = np.array([3, 0, 6, 1, 5, 2, 4])
    q = _permute_configs(p, perm)
    nE = p.n_cfg
    yE, yF = y[:nE], y[nE:].reshape(-1, 3)
    atoms_new = np.concatenate([np.arange(p.cfg_ptr[A], p.cfg_ptr[A + 1]) for A in perm])
    y2 = np.concatenate([yE[perm], yF[atoms_new].reshape(-1)])
    c2, _ = oracle.fit(q, y2)
    assert rel(c2, c) < 1e-11


def _permute_configs(p, perm):
    import copy
    q = copy.copy(p)
    sizes = np.diff(p.cfg_ptr)[perm]
    q.cfg_ptr = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    atoms_new = np.concatenate([np.arange(p.cfg_ptr[A], p.cfg_ptr[A + 1]) for A in perm])
    inv = np.empty_like(atoms_new)
    inv[atoms_new] = np.arange(len(atoms_new))
    q.X = np.ascontiguousarray(p.X[atoms_new])
    q.sigma_e = np.ascontiguousarray(p.sigma_e[perm])
    q.sigma_f = np.ascontiguousarray(p.sigma_f.reshape(-1, 3)[atoms_new].reshape(-1))
    nnb = np.diff(p.pair_ptr)[atoms_new]
    q.pair_ptr = np.concatenate([[0], np.cumsum(nnb)]).astype(np.int64)
    pairs_new = np.concatenate([np.arange(p.pair_ptr[a], p.pair_ptr[a + 1]) for a in atoms_new])
    q.pair_src = np.ascontiguousarray(inv[p.pair_src[pairs_new]])
    q.J = np.ascontiguousarray(p.J[pairs_new])
    return q


def test_zero_padding_rows_do_not_change_solution():
    """Sec. III.B: zero rows appended to A and b leave the least-squares solution unchanged."""
    p = small(forces=True, n_cfg=5, M=5, d=9, zeta=2)
    y = oracle.targets(p)
    A, _ = oracle.stacked_matrix(p)
    b = np.concatenate([y / oracle.sigma(p), np.zeros(p.n_sparse)])
    QR, tau = oracle.householder_qr(A)
    c1 = oracle.back_substitution(QR[:5], oracle.apply_qt(QR, tau, b)[:5])
    Ap = np.vstack([A[:7], np.zeros((4, 5)), A[7:], np.zeros((3, 5))])
    bp = np.concatenate([b[:7], np.zeros(4), b[7:], np.zeros(3)])
    QR2, tau2 = oracle.householder_qr(Ap)
    c2 = oracle.back_substitution(QR2[:5], oracle.apply_qt(QR2, tau2, bp)[:5])
    assert rel(c2, c1) < 1e-12


def test_noise_level_fit():
    """With N >> M and targets from hidden weights, the scaled training residual
    is at the noise level (each scaled row has unit noise)."""
    p = small(forces=True, n_cfg=30, atoms=(4, 8), M=10, d=12, zeta=2)
    y = oracle.targets(p)
    c, _ = oracle.fit(p, y)
    D = oracle.design(p)
    r = D @ c - y / oracle.sigma(p)
    assert 0.5 < np.sqrt(np.mean(r ** 2)) < 1.5


# ------------------------------------------------------------- species masks --
# With species labels the covariance vanishes between different species
# (the per-species sub-GAPs of the appendix command lines), so every branch of
# the oracle that takes species labels is pinned here on a three-species problem.

def species3(zeta=3, seed=23, forces=True, delta=1.0):
    return small(seed=seed, n_cfg=6, atoms=(5, 9), d=9, zeta=zeta, forces=forces, n_species=3,
                 sparse=(2, 3, 2), delta=delta)


def _mask(p):
    return (p.atom_species[:, None] == p.sparse_species[None, :]).astype(float)


def test_species_problem_mixes_species():
    """The fixture really has several species in every role (else the pins below are void)."""
    p = species3()
    assert len(set(p.atom_species.tolist())) == 3 and len(set(p.sparse_species.tolist())) == 3
    src_sp = p.atom_species[p.pair_src]
    tgt_sp = np.repeat(p.atom_species, np.diff(p.pair_ptr))
    assert (src_sp != tgt_sp).any() and (src_sp == tgt_sp).any()
    m = _mask(p)
    assert 0 < m.sum() < m.size


def test_kmm_species_block_diagonal_closed_form():
    """K_MM = mask o delta^2 (Xs Xs^T)^zeta + jitter I: sparse points of different
    species do not covary, so K_MM is block-diagonal by species."""
    p = species3(zeta=4, delta=0.7)
    K = oracle.kmm(p)
    same = (p.sparse_species[:, None] == p.sparse_species[None, :]).astype(float)
    ref = same * (0.49 * (p.Xs @ p.Xs.T) ** 4) + p.recipe.jitter * np.eye(p.n_sparse)
    assert rel(K, ref) < 1e-14
    assert np.array_equal(K[same == 0], np.zeros(int((same == 0).sum())))
    U = oracle.cholesky_upper(K)
    assert rel(U, np.linalg.cholesky(K).T) < 1e-13


def test_force_rows_species_zeta1_closed_form():
    """Force rows at zeta=1 are linear in the Jacobians: row (a, alpha) =
    -(delta^2/sigma) sum_p mask[i(p), s] (J_p[alpha] . x_s), a masked matrix
    product summed over the pairs of each target atom."""
    p = species3(zeta=1, delta=1.3)
    m = _mask(p)
    G = np.einsum("pak,sk->pas", p.J, p.Xs) * m[p.pair_src][:, None, :]   # [pair, alpha, s]
    tgt = np.repeat(np.arange(p.n_atoms), np.diff(p.pair_ptr))
    Fr = np.zeros((p.n_atoms, 3, p.n_sparse))
    np.add.at(Fr, tgt, G)
    ref = -(1.3 ** 2) * Fr.reshape(3 * p.n_atoms, p.n_sparse) / p.sigma_f[:, None]
    assert rel(oracle.design(p)[p.n_cfg:], ref) < 1e-13


def test_species_predictions_equal_design_rows_times_c():
    """Predictions with species labels (Eqs. 1, 2 and the chain rule) equal
    Sigma^{1/2} K c row by row, energies and forces."""
    p = species3(zeta=3)
    c = gapgen.normals(19, 1, p.n_sparse)
    K = oracle.design(p) * oracle.sigma(p)[:, None]
    E, F = oracle.predict(p, c)
    assert rel(K[:p.n_cfg] @ c, E) < 1e-13
    assert rel(K[p.n_cfg:] @ c, F) < 1e-12


@pytest.mark.parametrize("zeta", [2, 4])
def test_species_force_rows_finite_differences(zeta):
    """Masked force rows are -dE/dr: central differences of the masked energy
    E_A = sum_{i in A} sum_s c_s [sp_i = sp_s] delta^2 (x_i . x_s)^zeta, with every
    x_i moved along h J_p[alpha].  The energy here is the zeta=1-pinned masked
    product raised elementwise, evaluated by numpy, not by the oracle."""
    p = species3(zeta=zeta)
    c = gapgen.normals(8, 1, p.n_sparse)
    K = oracle.design(p) * oracle.sigma(p)[:, None]
    m = _mask(p)

    def energies(X):
        eps = ((X @ p.Xs.T) ** zeta * m) @ c
        return np.add.reduceat(eps, p.cfg_ptr[:-1])

    h = 1e-5
    for a in range(p.n_atoms):
        A = int(np.searchsorted(p.cfg_ptr, a, side="right") - 1)
        for al in range(3):
            dX = np.zeros_like(p.X)
            for q in range(p.pair_ptr[a], p.pair_ptr[a + 1]):
                dX[p.pair_src[q]] += p.J[q, al]
            fd = -(energies(p.X + h * dX)[A] - energies(p.X - h * dX)[A]) / (2 * h)
            row = K[p.n_cfg + 3 * a + al] @ c
            assert abs(row - fd) <= 1e-7 * max(1.0, abs(fd)), (a, al, row, fd)


# ---------------------------------------------------------------- virials --
# Virial rows: derivatives of the energy with respect to a homogeneous lattice
# deformation (Sec. II).  Each pair p carries u_p = r_a - r_i; a strain eps moves x_i
# by sum_{p: src(p) = i} J_p eps u_p to first order.

VOIGT = [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]


def _strained(p, v, h):
    """Descriptors under the symmetric strain h (e_a e_b^T + e_b e_a^T)/2 of Voigt
    component v (first order in the strain, as the derivative needs)."""
    a, b = VOIGT[v]
    dX = np.zeros_like(p.X)
    for q in range(p.n_pairs):
        dX[p.pair_src[q]] += 0.5 * (p.J[q, a] * p.pair_u[q, b] + p.J[q, b] * p.pair_u[q, a])
    return p.X + h * dX


@pytest.mark.parametrize("zeta,n_species", [(2, 1), (4, 1), (3, 3)])
def test_virial_rows_finite_differences(zeta, n_species):
    """Virial rows are -dE/d(strain): central differences of the energy
    E_A = sum_{i in A} sum_s c_s [sp_i = sp_s] delta^2 (x_i . x_s)^zeta (evaluated
    here by numpy, not by the oracle) under each of the six symmetric strains."""
    kw = dict(n_species=3, sparse=(2, 3, 2), atoms=(5, 9)) if n_species == 3 else dict(M=5)
    p = small(zeta=zeta, n_cfg=4, d=7, virials=True, seed=31, **kw)
    c = gapgen.normals(12, 1, p.n_sparse)
    K = oracle.design(p) * oracle.sigma(p)[:, None]
    m = np.ones((p.n_atoms, p.n_sparse)) if n_species == 1 else _mask(p)
    nv = p.n_cfg + 3 * p.n_atoms

    def energies(X):
        return np.add.reduceat(((X @ p.Xs.T) ** zeta * m) @ c, p.cfg_ptr[:-1])

    h = 1e-5
    for v in range(6):
        fd = -(energies(_strained(p, v, h)) - energies(_strained(p, v, -h))) / (2 * h)
        rows = K[nv + v::6][:p.n_cfg] @ c
        assert np.allclose(rows, fd, rtol=1e-7, atol=1e-7 * np.abs(fd).max()), (v, rows, fd)


def test_virial_rows_zeta1_closed_form():
    """At zeta = 1 the virial rows are linear in the Jacobians: row (A, v) =
    -(delta^2 / sigma) sum over A's pairs of sym(J_p x_s, u_p)_v, a matrix product."""
    p = small(zeta=1, n_cfg=5, d=6, M=4, virials=True, delta=0.8, seed=33)
    G = np.einsum("pak,sk->pas", p.J, p.Xs)                       # [pair, alpha, s]
    T = np.stack([0.5 * (G[:, a] * p.pair_u[:, b, None] + G[:, b] * p.pair_u[:, a, None])
                  for a, b in VOIGT], axis=1)                     # [pair, v, s]
    cfg_of_pair = np.repeat(np.repeat(np.arange(p.n_cfg), np.diff(p.cfg_ptr)), np.diff(p.pair_ptr))
    V = np.zeros((p.n_cfg, 6, p.n_sparse))
    np.add.at(V, cfg_of_pair, T)
    ref = -(0.8 ** 2) * V.reshape(6 * p.n_cfg, p.n_sparse) / p.sigma_v[:, None]
    assert rel(oracle.design(p)[p.n_cfg + 3 * p.n_atoms:], ref) < 1e-13


def test_virial_predictions_equal_design_rows_times_c():
    """Virial predictions equal Sigma^{1/2} K c over the virial rows."""
    p = small(zeta=3, n_cfg=5, d=7, M=6, virials=True, seed=35)
    c = gapgen.normals(14, 1, p.n_sparse)
    K = oracle.design(p) * oracle.sigma(p)[:, None]
    E, F, V = oracle.predict_all(p, c)
    nf = p.n_cfg + 3 * p.n_atoms
    assert rel(K[nf:] @ c, V) < 1e-12
    assert rel(K[p.n_cfg:nf] @ c, F) < 1e-12 and rel(K[:p.n_cfg] @ c, E) < 1e-13


# ------------------------------------------------------- planted mistakes --

MUTATIONS = {
    # a dropped term: the force sum skips the last pair of each atom
    "drop_pair": ("for (int64_t p = pair_ptr[a]; p < pair_ptr[a + 1]; ++p) {\n                int64_t i = pair_src[p];",
                  "for (int64_t p = pair_ptr[a]; p < pair_ptr[a + 1] - 1; ++p) {\n                int64_t i = pair_src[p];"),
    # a flipped sign in the force rows
    "force_sign": ("out[(3 * a + al) * M + s] = -f[al]", "out[(3 * a + al) * M + s] = f[al]"),
    # a wrong power in the derivative weight
    "weight_power": ("ipow(dot(X + i * d, Xs + s * d, d), zeta - 1)", "ipow(dot(X + i * d, Xs + s * d, d), zeta)"),
    # a transposed operand in the Cholesky update
    "chol_transpose": ("t -= U[k * M + j] * U[k * M + i];", "t -= U[j * M + k] * U[k * M + i];"),
    # a wrong Householder sign convention
    "householder_sign": ("double beta = -copysign(", "double beta = copysign("),
    # jitter dropped
    "no_jitter": ("if (t == s) v += jitter;", "if (t == s) v += 0.0;"),
    # species mask of the force rows dropped (the loop's continue removed)
    "force_species": ("if (!same_species(atom_sp, i, sparse_sp, s)) continue;\n                double w",
                      "double w"),
    # species mask of K_MM dropped
    "kmm_species": ("double v = same_species(sparse_sp, s, sparse_sp, t) ? or_kernel(Xs + s * d, Xs + t * d, d, delta, zeta) : 0.0;",
                    "double v = or_kernel(Xs + s * d, Xs + t * d, d, delta, zeta);"),
    # a virial component built from the wrong index of the Jacobian product
    "virial_index": ("v[3] = 0.5 * (g[1] * u[2] + g[2] * u[1]);", "v[3] = 0.5 * (g[1] * u[2] + g[1] * u[1]);"),
    # species mask of the predictions dropped
    "predict_species": ("if (!same_species(atom_sp, i, sparse_sp, s)) continue;\n            double g",
                        "double g"),
    # the covariance's delta^2 taken as delta
    "kernel_delta": ("return delta * delta * ipow(dot(x, xs, d), zeta);", "return delta * ipow(dot(x, xs, d), zeta);"),
    # the energy rows not scaled by Sigma^-1/2
    "energy_sigma": ("out[A * M + s] = e / sigma_e[A];", "out[A * M + s] = e;"),
    # the last atom of each configuration dropped from its energy sum
    "energy_last_atom": ("for (int64_t i = cfg_ptr[A]; i < cfg_ptr[A + 1]; ++i)\n                if (same_species",
                         "for (int64_t i = cfg_ptr[A]; i < cfg_ptr[A + 1] - 1; ++i)\n                if (same_species"),
    # K_MM's lower triangle left unmirrored
    "kmm_unmirrored": ("K[s * M + t] = v;\n            K[t * M + s] = v;", "K[s * M + t] = v;"),
    # the Cholesky pivot's square root forgotten
    "chol_no_sqrt": ("double ujj = sqrt(s);", "double ujj = s;"),
    # the right-hand side not scaled by Sigma^-1/2
    "rhs_unscaled": ("for (int64_t r = 0; r < N; ++r) b[r] = y[r] / sigma[r];", "for (int64_t r = 0; r < N; ++r) b[r] = y[r];"),
    # Q^T b with the reflectors applied in reverse order (that is Q b)
    "qt_reverse": ("for (int64_t j = 0; j < kmax; ++j) {\n        double w = b[j];",
                   "for (int64_t j = kmax - 1; j >= 0; --j) {\n        double w = b[j];"),
    # a transposed operand in the back substitution
    "backsub_transpose": ("t -= R[j * ldr + k] * c[k];", "t -= R[k * ldr + j] * c[k];"),
    # a flipped sign in the predicted forces
    "predict_force_sign": ("F[3 * a + al] = -f;", "F[3 * a + al] = f;"),
    # the gradient weight of the predictions one power too high
    "predict_grad_power": ("double w = c[s] * delta * delta * (double)zeta * ipow(g, zeta - 1);",
                           "double w = c[s] * delta * delta * (double)zeta * ipow(g, zeta);"),
    # the predicted atom energies without delta^2
    "predict_energy_delta": ("e += c[s] * delta * delta * ipow(g, zeta);", "e += c[s] * ipow(g, zeta);"),
    # a flipped sign in the virial rows
    "virial_sign": ("out[(6 * A + k) * M + s] = -v[k] / sigma_v[6 * A + k];",
                    "out[(6 * A + k) * M + s] = v[k] / sigma_v[6 * A + k];"),
    # an off-diagonal Voigt component not halved (the symmetrised product's 1/2 dropped)
    "voigt_half": ("v[5] = 0.5 * (g[0] * u[1] + g[1] * u[0]);", "v[5] = (g[0] * u[1] + g[1] * u[0]);"),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistakes_are_caught(name, tmp_path):
    """Compile the oracle with one planted mistake and check that a pin above
    rejects it (the mutant is loaded in place of the real oracle)."""
    import subprocess
    import ctypes
    src = open(os.path.join(os.path.dirname(oracle.__file__), "oracle.c")).read()
    old, new = MUTATIONS[name]
    assert src.count(old) >= 1, name
    so = tmp_path / "mut.so"
    (tmp_path / "mut.c").write_text(src.replace(old, new))
    subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", "-std=c11",
                    "-o", str(so), str(tmp_path / "mut.c"), "-lm"], check=True)
    saved = oracle._lib
    try:
        oracle._lib = None
        real_so = oracle._SO
        oracle._SO = str(so)
        orig_build = oracle.build
        oracle.build = lambda force=False: str(so)
        caught = False
        checks = [lambda: test_force_rows_finite_differences(3), test_kmm_symmetric_positive_definite_and_cholesky,
                  test_householder_matches_lapack_geqrf, test_prediction_equals_design_rows_times_c,
                  test_kmm_species_block_diagonal_closed_form, lambda: test_species_force_rows_finite_differences(2),
                  test_species_predictions_equal_design_rows_times_c, lambda: test_virial_rows_finite_differences(2, 1),
                  test_energy_rows_zeta1_are_a_matrix_product, test_zeta2_prediction_closed_form,
                  test_qr_orthogonality_and_reconstruction, test_back_substitution_matches_triangular_solve,
                  lambda: test_qr_solution_equals_normal_equations(True, False)]
        for chk in checks:
            try:
                chk()
            except (AssertionError, oracle.OracleError):
                caught = True
                break
        assert caught, "mutation %s passed every pin" % name
    finally:
        oracle._lib = saved
        oracle._SO = real_so
        oracle.build = orig_build
