"""Pins of the CUR oracle (oracle/cur.py) against facts fixed by the mathematics:
closed forms of the leverage scores, invariances, the convergence of the range finder
to the exact SVD, and the sampling law of the key method.  Each pin is chosen so that a
plausible mistake (a transposed operand, a dropped normalisation, a wrong key or sort
direction, a missing re-orthonormalisation) fails at least one of them; the planted
mistakes at the end check that."""
import os
import types

import numpy as np
import pytest

import gapgen
from oracle import cur


def _low_rank(n, d, r, seed, spread=None):
    """X = A B of rank r with singular values spread (default 1 .. 2^-(r-1))."""
    A = gapgen.normals(seed, 901, n * r).reshape(n, r)
    B = gapgen.normals(seed, 902, r * d).reshape(r, d)
    Ua, _ = np.linalg.qr(A)
    Vb, _ = np.linalg.qr(B.T)
    s = spread if spread is not None else 2.0 ** -np.arange(r)
    return (Ua * s) @ Vb.T, Ua


def test_leverage_of_rank_k_matrix_is_hat_diagonal():
    """k = rank(X) <= l: pi_i = a_i^T (A^T A)^{-1} a_i / k for any A with range(A) = range(X)
    (the hat matrix diagonal), here with A = X's own factor times a random invertible map."""
    n, d, r = 300, 40, 6
    X, Ua = _low_rank(n, d, r, 11)
    A = Ua @ gapgen.normals(11, 903, r * r).reshape(r, r)
    hat = np.einsum("ij,ij->i", A, np.linalg.solve(A.T @ A, A.T).T)
    omega, _ = gapgen.cur_draws(11, n, d, 10)
    pi = cur.leverage(X, omega, r, 0)
    assert np.allclose(pi, hat / r, rtol=1e-9, atol=1e-14)


def test_leverage_rank_one_closed_form():
    """X = a b^T, k = l = 1: pi_i = a_i^2 / |a|^2."""
    a = gapgen.normals(3, 904, 50)
    b = gapgen.normals(3, 905, 7)
    omega, _ = gapgen.cur_draws(3, 50, 7, 1)
    pi = cur.leverage(np.outer(a, b), omega, 1, 0)
    assert np.allclose(pi, a * a / (a @ a), rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("k,l,q", [(4, 12, 0), (8, 24, 2), (1, 5, 1)])
def test_leverage_sums_to_one_and_is_bounded(k, l, q):
    """sum_i pi_i = |U_k|_F^2 / k = 1 and 0 <= pi_i <= 1/k (rows of orthonormal columns)."""
    X = gapgen.clustered_descriptors(7, 800, 48, 30)
    omega, _ = gapgen.cur_draws(7, 800, 48, l)
    pi = cur.leverage(X, omega, k, q)
    assert abs(pi.sum() - 1.0) < 1e-12
    assert (pi >= 0).all() and (pi <= 1.0 / k + 1e-14).all()


def test_power_iterations_converge_to_exact_svd_leverage():
    """Full-rank X with geometric spectrum: with enough power iterations the range
    finder's scores equal those of numpy's SVD of X (Halko et al., Thm. 9.2 bound)."""
    n, d = 500, 30
    X, _ = _low_rank(n, d, d, 21, spread=0.5 ** np.arange(d))
    U, _, _ = np.linalg.svd(X, full_matrices=False)
    k = 5
    exact = (U[:, :k] ** 2).sum(1) / k
    omega, _ = gapgen.cur_draws(21, n, d, 10)
    err = [np.abs(cur.leverage(X, omega, k, q) - exact).max() / exact.max() for q in (0, 2, 6)]
    assert err[2] < 1e-9 and err[0] > err[1] > err[2]


def test_leverage_invariances():
    """Rotating the descriptor space (X Q with Q^T omega), scaling X, and permuting the
    rows (the scores permute along) leave the scores unchanged."""
    n, d, l, k = 400, 24, 12, 5
    X = gapgen.clustered_descriptors(4, n, d, 25)
    omega, _ = gapgen.cur_draws(4, n, d, l)
    pi = cur.leverage(X, omega, k, 1)
    Q, _ = np.linalg.qr(gapgen.normals(4, 906, d * d).reshape(d, d))
    assert np.allclose(cur.leverage(X @ Q, Q.T @ omega, k, 1), pi, rtol=1e-9, atol=1e-14)
    assert np.allclose(cur.leverage(3.5 * X, omega, k, 1), pi, rtol=1e-10, atol=1e-15)
    perm = np.argsort(gapgen.uniforms(4, 907, n))
    assert np.allclose(cur.leverage(X[perm], omega, k, 1), pi[perm], rtol=1e-9, atol=1e-14)


def test_rare_environments_get_high_leverage():
    """Atoms alone in their direction of descriptor space have the largest scores: an
    orthogonal outlier row holds one full singular direction (pi = 1/k)."""
    n, d = 300, 20
    X = np.abs(gapgen.normals(8, 908, n * d).reshape(n, d)) * 0.05
    X[:, 0] += 1.0
    X[17] = 0.0
    X[:, 19] = 0.0
    X[17, 19] = 5.0  # alone along axis 19, strongest after the common direction
    omega, _ = gapgen.cur_draws(8, n, d, 8)
    pi = cur.leverage(X, omega, 2, 3)
    assert np.argmax(pi) == 17 and abs(pi[17] - 0.5) < 1e-9


def test_draw_takes_largest_keys_ties_to_lower_index():
    pi = np.array([0.1, 0.2, 0.0, 0.3, 0.2, 0.2])
    u = np.array([0.5, 0.9, 0.99, 0.1, 0.9, 0.9])
    key = np.log(u) / np.where(pi > 0, pi, 1)
    # keys: -6.93, -0.527, -inf, -7.68, -0.527, -0.527
    assert list(cur.draw(pi, u, 2)) == [1, 4]
    assert list(cur.draw(pi, u, 4)) == [0, 1, 4, 5]
    assert list(cur.draw(pi, u, 6)) == [0, 1, 2, 3, 4, 5]  # pi = 0 last
    assert list(cur.draw(pi, u, 5)) == [0, 1, 3, 4, 5]
    assert key[1] == key[4]
    # a heavy item with a middling u beats a light one with a larger u: log(0.5)/0.5 > log(0.6)/0.1
    assert list(cur.draw(np.array([0.5, 0.1]), np.array([0.5, 0.6]), 1)) == [0]


def test_draw_follows_successive_sampling_law():
    """The key method draws like successive sampling without replacement: the first
    item is i with probability p_i, and the pair {i, j} (m = 2) with probability
    p_i p_j / (1 - p_i) + p_j p_i / (1 - p_j).  Checked over 40000 seeded draws, to 5
    standard deviations."""
    p = np.array([0.4, 0.25, 0.2, 0.1, 0.05])
    T = 40000
    U = (1.0 - gapgen.uniforms(5, 909, T * len(p))).reshape(T, len(p))
    first = np.zeros(len(p))
    pairs = {}
    for t in range(T):
        with np.errstate(divide="ignore"):
            key = np.log(U[t]) / p
        first[np.argmax(key)] += 1
        sel = tuple(cur.draw(p, U[t], 2))
        pairs[sel] = pairs.get(sel, 0) + 1
    sd = np.sqrt(p * (1 - p) / T)
    assert np.all(np.abs(first / T - p) < 5 * sd)
    for i in range(len(p)):
        for j in range(i + 1, len(p)):
            q = p[i] * p[j] / (1 - p[i]) + p[j] * p[i] / (1 - p[j])
            f = pairs.get((i, j), 0) / T
            assert abs(f - q) < 5 * np.sqrt(q * (1 - q) / T) + 1e-4, (i, j, f, q)


def test_select_cur_species_blocks():
    """Each species draws from its own atoms, with scores of its own rows only."""
    n, d, l, k = 600, 32, 16, 6
    X = gapgen.clustered_descriptors(9, n, d, 30)
    species = gapgen.uniform_ints(9, 910, n, 0, 2).astype(np.int32)
    omega, u = gapgen.cur_draws(9, n, d, l)
    sel, lev = cur.select_cur(X, species, [20, 0, 35], k, l, 1, omega, u)
    assert len(sel) == 55 and (species[sel[:20]] == 0).all() and (species[sel[20:]] == 2).all()
    assert (np.diff(sel[:20]) > 0).all() and (np.diff(sel[20:]) > 0).all()
    assert np.isnan(lev[species == 1]).all()
    a0 = np.nonzero(species == 0)[0]
    assert np.allclose(lev[a0], cur.leverage(X[a0], omega, k, 1), rtol=0, atol=0)
    assert abs(lev[species == 2].sum() - 1.0) < 1e-12


# planted mistakes: each rewrites one line of oracle/cur.py; some pin above must fail
MUTATIONS = {
    "transposed_operand": ("B = Q.T @ X", "B = X.T @ Q"),
    "no_normalisation": ("return (Uk * Uk).sum(axis=1) / k", "return (Uk * Uk).sum(axis=1)"),
    "smallest_eigenvalues": ("order = np.argsort(-lam, kind=\"stable\")[:k]",
                             "order = np.argsort(lam, kind=\"stable\")[:k]"),
    "no_reorthonormalisation": ("Q, _ = np.linalg.qr(X @ (X.T @ Q))", "Q = X @ (X.T @ Q)"),
    "key_sign": ("order = np.lexsort((np.arange(len(pi)), -key))", "order = np.lexsort((np.arange(len(pi)), key))"),
    "key_multiplies": ("np.log(u) / np.where(pi > 0, pi, 1.0)", "np.log(u) * np.where(pi > 0, pi, 1.0)"),
    "power_iterations_skipped": ("    for _ in range(power_iters):", "    for _ in range(0):"),
    "species_ignored": ("atoms = np.nonzero(species == t)[0]", "atoms = np.arange(n)"),
    "smallest_keys_drawn": ("return np.sort(order[:m])", "return np.sort(order[len(order) - m:])"),
}

PINS = [test_leverage_of_rank_k_matrix_is_hat_diagonal, test_leverage_rank_one_closed_form,
        lambda: test_leverage_sums_to_one_and_is_bounded(8, 24, 2), test_power_iterations_converge_to_exact_svd_leverage,
        test_leverage_invariances, test_rare_environments_get_high_leverage,
        test_draw_takes_largest_keys_ties_to_lower_index, test_select_cur_species_blocks,
        test_draw_follows_successive_sampling_law]


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistakes_are_caught(name, monkeypatch):
    src = open(cur.__file__).read()
    old, new = MUTATIONS[name]
    assert src.count(old) == 1, name
    mod = types.ModuleType("cur_mutant")
    exec(compile(src.replace(old, new), os.path.join(os.path.dirname(cur.__file__), "cur_mutant.py"), "exec"),
         mod.__dict__)
    for fn in ("range_basis", "leverage", "draw", "select_cur"):
        monkeypatch.setattr(cur, fn, getattr(mod, fn))
    caught = False
    for chk in PINS:
        try:
            chk()
        except Exception:  # a failed pin, or a mutant that no longer runs
            caught = True
            break
    assert caught, "mutation %s passed every pin" % name
