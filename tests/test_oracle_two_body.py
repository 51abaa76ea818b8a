"""Pins of the two-body sub-GAP oracle (oracle/two_body.py): central finite differences of
its energy with respect to atom positions and to a homogeneous strain (with the bonds
rebuilt from the moved positions, so that bonds crossing the cutoff are included), the
closed form of a dimer, the K_MM block's diagonal, predictions equal to the design rows
times the weights, and the whole fit against numpy's least squares.  Planted mistakes in
the oracle's source must each fail a pin."""
import copy
import os
import types

import numpy as np
import pytest

import gapgen
import oracle
from oracle import two_body


def _problem(seed=7, virials=True, n_cfg=5):
    r = gapgen.Recipe(n_cfg=n_cfg, atoms=(2, 30), d=9, n_sparse=(8,), zeta=2, neighbours=(1, 4), two_body=True,
                      virials=virials, seed=seed)
    return gapgen.make_problem(r)


def _moved(p, pos):
    """p with its two-body inputs rebuilt from atom positions pos."""
    q = copy.copy(p)
    tb = p.two_body
    ptr, rr, uu = gapgen.bonds_from_positions(pos, p.cfg_ptr, tb.cutoff)
    q.two_body = gapgen.TwoBody(pos, ptr, rr, uu, tb.sparse_r, tb.delta, tb.theta, tb.cutoff, tb.width)
    return q


def _energy(p, c2):
    return two_body.predict_2b(p, c2)[0]


def test_forces_are_minus_energy_gradient():
    p = _problem()
    c2 = gapgen.normals(3, 950, len(p.two_body.sparse_r))
    _, F, _ = two_body.predict_2b(p, c2)
    F = F.reshape(-1, 3)
    h = 1e-6
    cfg_of = np.repeat(np.arange(p.n_cfg), np.diff(p.cfg_ptr))
    for a in range(0, p.n_atoms, 7):
        for al in range(3):
            pos = p.two_body.positions.copy()
            pos[a, al] += h
            ep = _energy(_moved(p, pos), c2)[cfg_of[a]]
            pos[a, al] -= 2 * h
            em = _energy(_moved(p, pos), c2)[cfg_of[a]]
            assert abs(-(ep - em) / (2 * h) - F[a, al]) < 1e-6 * (1 + abs(F[a, al]))


@pytest.mark.parametrize("v", range(6))
def test_virials_are_minus_strain_derivative(v):
    p = _problem()
    c2 = gapgen.normals(4, 951, len(p.two_body.sparse_r))
    _, _, V = two_body.predict_2b(p, c2)
    V = V.reshape(-1, 6)
    al, be = two_body.VOIGT[v]
    h = 1e-6

    def e_at(eps):
        S = np.eye(3)
        S[al, be] += eps
        return _energy(_moved(p, p.two_body.positions @ S.T), c2)

    fd = -(e_at(h) - e_at(-h)) / (2 * h)
    assert np.allclose(fd, V[:, v], rtol=1e-6, atol=1e-8)


def test_dimer_closed_form():
    """Two atoms at distance r: one energy row k(r, r_t) (the bond listed twice, halved),
    and on atom 0 the force row -dk/dr (r_0 - r_1) / r."""
    p = _problem(n_cfg=1)
    pos = np.array([[0.0, 0.0, 0.0], [1.1, -0.7, 2.0]])
    q = copy.copy(p)
    q.cfg_ptr = np.array([0, 2], np.int64)
    q.X = p.X[:2]
    q.sigma_e = np.ones(1)
    q.noise_e = np.zeros(1)
    q.pair_ptr = np.array([0, 1, 2], np.int64)
    q.pair_src = np.array([0, 1], np.int64)
    q.J = p.J[:2]
    q.sigma_f = np.ones(6)
    q.pair_u, q.sigma_v = None, None
    q = _moved(q, pos)
    tb = q.two_body
    r = np.linalg.norm(pos[0] - pos[1])
    D = two_body.design_2b(q)
    f = lambda x: 0.5 * (1 + np.cos(np.pi * np.clip((x - tb.cutoff + tb.width) / tb.width, 0, 1))) * (x < tb.cutoff)  # noqa: E731
    g = tb.delta ** 2 * np.exp(-(r - tb.sparse_r) ** 2 / (2 * tb.theta ** 2))
    k = g * f(r) * f(tb.sparse_r)
    assert np.allclose(D[0], k, rtol=1e-13, atol=1e-300)
    # d/dr of k by central differences of the closed form, then the chain rule along the bond
    hh = 1e-6
    kp = tb.delta ** 2 * np.exp(-(r + hh - tb.sparse_r) ** 2 / (2 * tb.theta ** 2)) * f(r + hh) * f(tb.sparse_r)
    km = tb.delta ** 2 * np.exp(-(r - hh - tb.sparse_r) ** 2 / (2 * tb.theta ** 2)) * f(r - hh) * f(tb.sparse_r)
    dk = (kp - km) / (2 * hh)
    u = (pos[0] - pos[1]) / r
    for al in range(3):
        assert np.allclose(D[1 + al], -dk * u[al], rtol=1e-6, atol=1e-10)


def test_kmm_block_diagonal_and_positive():
    p = _problem()
    tb = p.two_body
    K = oracle.kmm(p)
    M, Ms = p.n_weights, p.n_sparse
    assert np.array_equal(K[:Ms, Ms:], np.zeros((Ms, M - Ms)))
    f, _ = two_body.cutoff(tb.sparse_r, tb.cutoff, tb.width)
    assert np.allclose(np.diag(K)[Ms:], tb.delta ** 2 * f * f + p.recipe.jitter, rtol=1e-14, atol=0.0)
    assert np.allclose(K, K.T)
    np.linalg.cholesky(K)


def test_predictions_equal_design_rows_times_c():
    p = _problem()
    c = gapgen.normals(5, 952, p.n_weights)
    E, F, V = oracle.predict_all(p, c)
    D = oracle.design(p)
    y = D @ c * oracle.sigma(p)
    assert np.allclose(np.concatenate([E, F, V]), y, rtol=1e-12, atol=1e-12 * np.abs(y).max())


def test_fit_solves_the_normal_equations():
    p = _problem()
    y = oracle.targets(p)
    c, _ = oracle.fit(p, y)
    A, _ = oracle.stacked_matrix(p)
    b = np.concatenate([y / oracle.sigma(p), np.zeros(p.n_weights)])
    # the loss gradient A^T (b - A c) vanishes at the solution, relative to |A^T b|
    g = A.T @ (b - A @ c)
    assert np.linalg.norm(g) < 1e-8 * np.linalg.norm(A.T @ b)


MUTATIONS = {
    "energy_not_halved": ("np.add.at(E, cfg, 0.5 * k)", "np.add.at(E, cfg, k)"),
    "force_sign": ("np.add.at(F[:, al, :], atom, -dk * tb.bond_u[:, al:al + 1])",
                   "np.add.at(F[:, al, :], atom, dk * tb.bond_u[:, al:al + 1])"),
    "cutoff_derivative_dropped": ("dk = g * (-(r - rt) / tb.theta ** 2 * f + df) * ft",
                                  "dk = g * (-(r - rt) / tb.theta ** 2 * f) * ft"),
    "theta_not_squared": ("g = tb.delta ** 2 * np.exp(-(r - rt) ** 2 / (2.0 * tb.theta ** 2))",
                          "g = tb.delta ** 2 * np.exp(-(r - rt) ** 2 / (2.0 * tb.theta))"),
    "virial_index": ("g = -0.5 * dk * (tb.bond_r * tb.bond_u[:, al] * tb.bond_u[:, be])[:, None]",
                     "g = -0.5 * dk * (tb.bond_r * tb.bond_u[:, al] * tb.bond_u[:, al])[:, None]"),
    "predict_force_sign": ("np.add.at(F, atom, -deps[:, None] * tb.bond_u)",
                           "np.add.at(F, atom, deps[:, None] * tb.bond_u)"),
    "energy_rows_unscaled": ("rows.append(E / p.sigma_e[:, None])", "rows.append(E)"),
    "sparse_cutoff_dropped": ("k = g * f * ft", "k = g * f"),
    "kmm_jitter_dropped": ("return K + p.recipe.jitter * np.eye(len(tb.sparse_r))", "return K"),
    "cutoff_slope_sign": ("df = np.where(inside, -0.5 * np.pi / w * np.sin(np.pi * x), 0.0)",
                          "df = np.where(inside, 0.5 * np.pi / w * np.sin(np.pi * x), 0.0)"),
}

PINS = [test_forces_are_minus_energy_gradient, lambda: [test_virials_are_minus_strain_derivative(v) for v in range(6)],
        test_dimer_closed_form, test_kmm_block_diagonal_and_positive, test_predictions_equal_design_rows_times_c]


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistakes_are_caught(name, monkeypatch):
    src = open(two_body.__file__).read()
    old, new = MUTATIONS[name]
    assert src.count(old) == 1, name
    mod = types.ModuleType("two_body_mutant")
    exec(compile(src.replace(old, new), os.path.join(os.path.dirname(two_body.__file__), "two_body_mutant.py"),
                 "exec"), mod.__dict__)
    for fn in ("cutoff", "kernel", "design_2b", "kmm_2b", "predict_2b"):
        monkeypatch.setattr(two_body, fn, getattr(mod, fn))
    caught = False
    for chk in PINS:
        try:
            chk()
        except Exception:
            caught = True
            break
    assert caught, "mutation %s passed every pin" % name
