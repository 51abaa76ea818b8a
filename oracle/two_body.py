"""ORACLE -- test infrastructure only.

Plain FP64 numpy statement of the two-body sub-GAP of the paper's appendix
(``distance_2b`` descriptors with ``covariance_type=ard_se``): a second model summed into
the same design matrix, its sparse points a second column block.  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may use it; the GPU
library never does, and the two share no code.

Readings (the paper gives only the command line):
* the descriptor of an atom pair is its distance r; every pair within the cutoff r_c is
  one descriptor instance, so E_2b = sum over pairs i < j of eps(r_ij).  The inputs list
  every pair from both ends (directed bonds, grouped by atom a, with the unit vector
  u = (r_a - r_j) / r), so E_2b = (1/2) sum over directed bonds of eps(r);
* ard_se covariance with one length scale theta (theta_uniform) for the one dimension,
  weighted by a smooth cutoff of both instances:
      k(r, r') = delta^2 exp(-(r - r')^2 / (2 theta^2)) f(r) f(r'),
      f(r) = 1 below r_c - w, (1 + cos(pi (r - r_c + w) / w)) / 2 up to r_c, 0 beyond;
* eps(r) = sum_t c_t k(r, r_t) over the two-body sparse points r_t (given);
* rows follow the SOAP block's conventions: energy rows sum over the configuration's
  atoms, force rows are -dE/dr_a, virial rows -dE/d(strain) in Voigt order, each row
  scaled by 1/sigma.  A bond's length moves by u . dr_a under a displacement of its atom a
  (the bond listed from a), and by r u_alpha u_beta eps_alpha_beta under a homogeneous
  strain, so
      K_(A,t)       = (1/2) sum_{a in A} sum_{b of a} k(r_b, r_t),
      K_((a,al),t)  = -sum_{b of a} dk/dr(r_b, r_t) u_b[al],
      K_((A,v),t)   = -(1/2) sum_{a in A} sum_{b of a} dk/dr(r_b, r_t) r_b u_b[al] u_b[be].
"""
from __future__ import annotations

import numpy as np

VOIGT = ((0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1))


def cutoff(r, rc, w):
    """The cutoff weight f(r) and its derivative."""
    r = np.asarray(r, dtype=np.float64)
    x = np.clip((r - (rc - w)) / w, 0.0, 1.0)
    f = np.where(r >= rc, 0.0, 0.5 * (1.0 + np.cos(np.pi * x)))
    inside = (r > rc - w) & (r < rc)
    df = np.where(inside, -0.5 * np.pi / w * np.sin(np.pi * x), 0.0)
    return f, df


def kernel(r, rt, tb):
    """k(r, r_t) [len(r) x len(rt)] and dk/dr, for tb = the problem's TwoBody block."""
    r = np.asarray(r, dtype=np.float64)[:, None]
    rt = np.asarray(rt, dtype=np.float64)[None, :]
    f, df = cutoff(r, tb.cutoff, tb.width)
    ft, _ = cutoff(rt, tb.cutoff, tb.width)
    g = tb.delta ** 2 * np.exp(-(r - rt) ** 2 / (2.0 * tb.theta ** 2))
    k = g * f * ft
    dk = g * (-(r - rt) / tb.theta ** 2 * f + df) * ft
    return k, dk


def _bond_atom(tb, n_atoms):
    return np.repeat(np.arange(n_atoms), np.diff(tb.bond_ptr))


def design_2b(p):
    """The two-body column block of the data rows Sigma^{-1/2} K_NM: [N x M_2b], energies,
    forces, then virials, in the row order of the SOAP block."""
    tb = p.two_body
    k, dk = kernel(tb.bond_r, tb.sparse_r, tb)
    atom = _bond_atom(tb, p.n_atoms)
    cfg_of_atom = np.repeat(np.arange(p.n_cfg), np.diff(p.cfg_ptr))
    cfg = cfg_of_atom[atom]
    M2 = len(tb.sparse_r)
    rows = []
    E = np.zeros((p.n_cfg, M2))
    np.add.at(E, cfg, 0.5 * k)
    rows.append(E / p.sigma_e[:, None])
    if p.has_forces:
        F = np.zeros((p.n_atoms, 3, M2))
        for al in range(3):
            np.add.at(F[:, al, :], atom, -dk * tb.bond_u[:, al:al + 1])
        rows.append(F.reshape(3 * p.n_atoms, M2) / p.sigma_f[:, None])
    if p.has_virials:
        V = np.zeros((p.n_cfg, 6, M2))
        for v, (al, be) in enumerate(VOIGT):
            g = -0.5 * dk * (tb.bond_r * tb.bond_u[:, al] * tb.bond_u[:, be])[:, None]
            np.add.at(V[:, v, :], cfg, g)
        rows.append(V.reshape(6 * p.n_cfg, M2) / p.sigma_v[:, None])
    return np.vstack(rows)


def kmm_2b(p):
    """The two-body block of K_MM, with the absolute jitter on its diagonal."""
    tb = p.two_body
    K, _ = kernel(tb.sparse_r, tb.sparse_r, tb)
    return K + p.recipe.jitter * np.eye(len(tb.sparse_r))


def predict_2b(p, c2):
    """The two-body model's energies [n_cfg], forces [3 n_atoms] (or None) and virials
    [6 n_cfg] (or None) for its weights c2."""
    tb = p.two_body
    k, dk = kernel(tb.bond_r, tb.sparse_r, tb)
    eps, deps = k @ c2, dk @ c2
    atom = _bond_atom(tb, p.n_atoms)
    cfg = np.repeat(np.arange(p.n_cfg), np.diff(p.cfg_ptr))[atom]
    E = np.zeros(p.n_cfg)
    np.add.at(E, cfg, 0.5 * eps)
    F = V = None
    if p.has_forces:
        F = np.zeros((p.n_atoms, 3))
        np.add.at(F, atom, -deps[:, None] * tb.bond_u)
        F = F.reshape(-1)
    if p.has_virials:
        V = np.zeros((p.n_cfg, 6))
        for v, (al, be) in enumerate(VOIGT):
            np.add.at(V[:, v], cfg, -0.5 * deps * tb.bond_r * tb.bond_u[:, al] * tb.bond_u[:, be])
        V = V.reshape(-1)
    return E, F, V
