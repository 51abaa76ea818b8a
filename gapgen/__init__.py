"""Seeded synthetic inputs for sparse-GP (GAP) fits.

This module draws the raw inputs of a fit and nothing else: configuration
sizes, species, neighbour lists, unit-length descriptors, descriptor Jacobians,
sparse-point indices, a hidden weight vector c* and target noise.  It holds no
arithmetic of the fitting method (no kernel evaluation, no sums over
configurations, no linear algebra), so both the FP64 oracle and the GPU
library can consume it without sharing any of the method's code.

Targets y are NOT produced here: the hidden-weight targets y = K c* + noise
need the method's forward model, so the tests compute them with the oracle
(small problems) and a committed script under ``tests/golden`` stores them for
the large workload.

Workload recipes (the synthetic stand-ins for the paper's HEA and SiC training
sets, Sec. IV; energies plus three force rows per atom, nonnegative SOAP-like
descriptors, thousands of sparse points, uneven configuration sizes) are in
``RECIPES``.  Seeds are ``2207038030 + workload number``.
"""
from __future__ import annotations

import ctypes
import hashlib
import math
import os
import subprocess
from dataclasses import dataclass, field, replace as dataclasses_replace
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_gapgen.so")
_lib = None

SEED_BASE = 2207038030

# array ids of the counter-based generator (one independent stream per array)
_AID_CFG, _AID_SPECIES, _AID_NNB, _AID_SRC, _AID_X, _AID_J = 1, 2, 3, 4, 5, 6
_AID_CSTAR, _AID_NOISE_E, _AID_NOISE_F, _AID_SPARSE = 7, 8, 9, 10
_AID_U, _AID_NOISE_V = 11, 12
_AID_CUR_OMEGA, _AID_CUR_U, _AID_CUR_X, _AID_CUR_Z = 13, 14, 15, 16
_AID_POS, _AID_CSTAR_2B = 17, 18
_AID_FIT = 100  # batched sweeps: per-fit hyperparameter draws


def build(force: bool = False) -> str:
    """Compile the generator library in place (gcc, OpenMP, no FMA contraction)."""
    src = os.path.join(_HERE, "gen.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", "-std=c11",
               "-o", _SO + ".tmp", src, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(_SO + ".tmp", _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        u64, i64, i32, dbl, p = ctypes.c_uint64, ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_void_p
        lib.gg_normals.argtypes = [u64, u64, i64, i64, dbl, p]
        lib.gg_ints.argtypes = [u64, u64, i64, i64, i64, p]
        lib.gg_uniforms.argtypes = [u64, u64, i64, p]
        lib.gg_descriptors.argtypes = [u64, u64, i64, i64, i64, i32, p]
        lib.gg_pair_src.argtypes = [u64, u64, i64, p, p, p, p]
        lib.gg_descriptor_rows.argtypes = [u64, u64, p, i64, i64, i32, p]
        lib.gg_subset.argtypes = [u64, u64, i64, p, i64]
        lib.gg_subset.restype = i32
        lib.gg_log_public.argtypes = [dbl]
        lib.gg_log_public.restype = dbl
        _lib = lib
    return _lib


def _ptr(a: np.ndarray) -> int:
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


def gen_log(x: float) -> float:
    """The generator's own platform-independent natural logarithm."""
    return _load().gg_log_public(float(x))


def normals(seed: int, aid: int, n: int, scale: float = 1.0, offset: int = 0, out=None) -> np.ndarray:
    out = np.empty(n, np.float64) if out is None else out
    _load().gg_normals(seed, aid, offset, n, scale, _ptr(out))
    return out


def uniform_ints(seed: int, aid: int, n: int, lo: int, hi: int) -> np.ndarray:
    out = np.empty(n, np.int64)
    _load().gg_ints(seed, aid, n, lo, hi, _ptr(out))
    return out


def uniforms(seed: int, aid: int, n: int) -> np.ndarray:
    out = np.empty(n, np.float64)
    _load().gg_uniforms(seed, aid, n, _ptr(out))
    return out


def descriptors(seed: int, n: int, d: int, absval: bool, row0: int = 0, out=None, aid: int = _AID_X) -> np.ndarray:
    out = np.empty((n, d), np.float64) if out is None else out
    _load().gg_descriptors(seed, aid, row0, n, d, int(absval), _ptr(out))
    return out


@dataclass
class Recipe:
    """Shape of one synthetic fit (all ranges inclusive)."""
    n_cfg: int
    atoms: tuple          # (lo, hi) atoms per configuration, uniform
    d: int                # descriptor length
    n_sparse: tuple       # sparse points per species
    zeta: int
    delta: float = 1.0
    absval: bool = True   # |N(0,1)| (SOAP-like, nonnegative) before normalising
    neighbours: Optional[tuple] = None  # (lo, hi) pairs per atom; None = energies only
    j_std: float = 0.1
    sigma_e_atom: float = 1e-3   # energy sigma per atom; sigma_A = sigma_e_atom * sqrt(n_A)
    sigma_f: float = 1e-2
    noise_e_abs: Optional[float] = None  # fixed energy-noise std (else sigma_A)
    virials: bool = False        # six virial rows per configuration (needs neighbours)
    u_std: float = 1.5           # pair displacement r_a - r_i per component, N(0, u_std^2)
    sigma_v_atom: float = 1e-2   # virial sigma per atom; sigma_V = sigma_v_atom * sqrt(n_A)
    n_species: int = 1
    jitter: float = 1e-8
    seed: int = SEED_BASE
    # two-body sub-GAP (distance_2b, ard_se): atoms uniform in a cube per configuration at
    # this number density, every pair closer than cutoff_2b a bond; n_sparse_2b sparse
    # distances at the midpoints of n_sparse_2b equal bins of [0, cutoff_2b]
    two_body: bool = False
    n_sparse_2b: int = 20
    delta_2b: float = 1.0
    theta_2b: float = 0.75
    cutoff_2b: float = 4.5
    width_2b: float = 0.5
    density_2b: float = 0.05


RECIPES = {
    # workload 1: 64 configurations of 8-32 atoms, d=32 signed N(0,1) descriptors,
    # M=64, zeta=2, energies only, noise N(0, 1e-3^2)
    1: Recipe(n_cfg=64, atoms=(8, 32), d=32, n_sparse=(64,), zeta=2, absval=False,
              neighbours=None, noise_e_abs=1e-3, seed=SEED_BASE + 1),
    # workload 2: 2000 configurations of 16-128 atoms, d=512 nonnegative, M=4000,
    # zeta=4, 8-24 neighbours with N(0, 0.1^2) Jacobians, sigma_E=1e-3/atom, sigma_F=1e-2
    2: Recipe(n_cfg=2000, atoms=(16, 128), d=512, n_sparse=(4000,), zeta=4,
              neighbours=(8, 24), seed=SEED_BASE + 2),
    # workload 5: 3 species, 5334+5333+5333 sparse points, d=1024, zeta=4,
    # 6000 configurations of 16-96 atoms, energies and forces
    5: Recipe(n_cfg=6000, atoms=(16, 96), d=1024, n_sparse=(5334, 5333, 5333), zeta=4,
              neighbours=(8, 24), n_species=3, seed=SEED_BASE + 5),
}


@dataclass
class TwoBody:
    """Inputs of the two-body sub-GAP: atom positions (drawn) and the bonds derived from
    them, every pair within the cutoff listed from both ends, grouped by atom."""
    positions: np.ndarray      # [n_atoms, 3]
    bond_ptr: np.ndarray       # [n_atoms+1] int64: bonds of atom a
    bond_r: np.ndarray         # [n_bonds] |r_a - r_j|
    bond_u: np.ndarray         # [n_bonds, 3] (r_a - r_j) / |r_a - r_j|
    sparse_r: np.ndarray       # [M_2b] sparse distances
    delta: float
    theta: float
    cutoff: float
    width: float

    @property
    def n_bonds(self): return len(self.bond_r)


def bonds_from_positions(pos: np.ndarray, cfg_ptr: np.ndarray, rc: float):
    """(bond_ptr, bond_r, bond_u): for every atom a, the atoms j != a of its configuration
    with |r_a - r_j| < rc, in ascending j."""
    ptr, rr, uu = [0], [], []
    for A in range(len(cfg_ptr) - 1):
        P = pos[cfg_ptr[A]:cfg_ptr[A + 1]]
        D = P[:, None, :] - P[None, :, :]
        R = np.sqrt((D * D).sum(-1))
        for i in range(len(P)):
            js = np.nonzero((R[i] < rc) & (np.arange(len(P)) != i))[0]
            rr.append(R[i, js])
            uu.append(D[i, js] / R[i, js, None])
            ptr.append(ptr[-1] + len(js))
    bond_r = np.concatenate(rr) if rr else np.zeros(0)
    bond_u = np.concatenate(uu) if uu else np.zeros((0, 3))
    return np.array(ptr, np.int64), np.ascontiguousarray(bond_r), np.ascontiguousarray(bond_u.reshape(-1, 3))


def make_two_body(r: Recipe, cfg_ptr: np.ndarray) -> TwoBody:
    """Positions uniform in a cube of volume n_A / density per configuration (the first
    atoms' positions do not depend on how many configurations are kept), and their bonds."""
    n_atoms = int(cfg_ptr[-1])
    pos = uniforms(r.seed, _AID_POS, 3 * n_atoms).reshape(n_atoms, 3)
    n_cfg_atoms = np.diff(cfg_ptr).astype(np.float64)
    side = np.repeat((n_cfg_atoms / r.density_2b) ** (1.0 / 3.0), np.diff(cfg_ptr))
    pos = pos * side[:, None]
    bond_ptr, bond_r, bond_u = bonds_from_positions(pos, cfg_ptr, r.cutoff_2b)
    sparse_r = (np.arange(r.n_sparse_2b) + 0.5) * (r.cutoff_2b / r.n_sparse_2b)
    return TwoBody(pos, bond_ptr, bond_r, bond_u, sparse_r, r.delta_2b, r.theta_2b, r.cutoff_2b, r.width_2b)


@dataclass
class Problem:
    """Raw inputs of one fit (host numpy arrays, row-major, FP64 canonical)."""
    recipe: Recipe
    cfg_ptr: np.ndarray        # [n_cfg+1] int64
    X: np.ndarray              # [n_atoms, d] unit rows
    sparse_idx: np.ndarray     # [M] int64, atom index of each sparse point
    Xs: np.ndarray             # [M, d]
    c_star: np.ndarray         # [M] hidden weights N(0,1)
    noise_e: np.ndarray        # [n_cfg] energy noise (already scaled)
    sigma_e: np.ndarray        # [n_cfg] per-configuration sigma
    atom_species: Optional[np.ndarray] = None    # [n_atoms] int32 (None: one species)
    sparse_species: Optional[np.ndarray] = None  # [M] int32
    pair_ptr: Optional[np.ndarray] = None   # [n_atoms+1] int64 (None: energies only)
    pair_src: Optional[np.ndarray] = None   # [n_pairs] int64
    J: Optional[np.ndarray] = None          # [n_pairs, 3, d]
    noise_f: Optional[np.ndarray] = None    # [3 n_atoms]
    sigma_f: Optional[np.ndarray] = None    # [3 n_atoms]
    pair_u: Optional[np.ndarray] = None     # [n_pairs, 3] displacement r_a - r_i of each pair (virials)
    noise_v: Optional[np.ndarray] = None    # [6 n_cfg]
    sigma_v: Optional[np.ndarray] = None    # [6 n_cfg]
    two_body: Optional[TwoBody] = None      # the two-body sub-GAP's inputs, or None
    extra: dict = field(default_factory=dict)

    @property
    def n_cfg(self): return len(self.cfg_ptr) - 1

    @property
    def n_atoms(self): return int(self.cfg_ptr[-1])

    @property
    def n_sparse(self): return len(self.sparse_idx)

    @property
    def n_weights(self):
        """Weights of the fit: the SOAP sparse points, then the two-body ones."""
        return self.n_sparse + (0 if self.two_body is None else len(self.two_body.sparse_r))

    @property
    def d(self): return self.X.shape[1]

    @property
    def n_pairs(self): return 0 if self.pair_src is None else len(self.pair_src)

    @property
    def has_forces(self): return self.pair_ptr is not None

    @property
    def has_virials(self): return self.pair_u is not None

    @property
    def n_rows(self):
        """Design rows: one energy row per configuration, 3 per atom with forces, then 6
        per configuration with virials (Voigt order xx, yy, zz, yz, xz, xy)."""
        return self.n_cfg + (3 * self.n_atoms if self.has_forces else 0) + (6 * self.n_cfg if self.has_virials else 0)


def _sparse_set(r: Recipe, species_full: Optional[np.ndarray], n_atoms_full: int) -> np.ndarray:
    """Sparse points: per species, a seeded random subset of that species' atoms (atom
    indices of the full problem)."""
    idx = []
    for t, m in enumerate(r.n_sparse):
        cand = np.arange(n_atoms_full, dtype=np.int64) if species_full is None else \
            np.nonzero(species_full == t)[0].astype(np.int64)
        cand = np.ascontiguousarray(cand)
        if _load().gg_subset(r.seed, _AID_SPARSE + 1000 * t, len(cand), _ptr(cand), m) != 0:
            raise ValueError("not enough atoms for %d sparse points of species %d" % (m, t))
        idx.append(cand[:m].copy())
    return np.concatenate(idx)


def make_problem(r: Recipe, J_out: Optional[np.ndarray] = None, max_cfg: Optional[int] = None) -> Problem:
    """Draw every input of recipe ``r``.  ``J_out`` may be a preallocated
    [n_pairs, 3, d] float64 buffer (e.g. pinned host memory) to fill in place.

    ``max_cfg`` keeps only the first ``max_cfg`` configurations (their atoms,
    pairs, Jacobians, noise) of the full problem while the sparse set is still
    drawn from all of its atoms: every kept value equals the full problem's."""
    s = r.seed
    n_atoms_cfg_full = uniform_ints(s, _AID_CFG, r.n_cfg, r.atoms[0], r.atoms[1])
    n_atoms_full = int(n_atoms_cfg_full.sum())
    k_cfg = r.n_cfg if max_cfg is None else min(max_cfg, r.n_cfg)
    n_atoms_cfg = n_atoms_cfg_full[:k_cfg]
    cfg_ptr = np.zeros(k_cfg + 1, np.int64)
    np.cumsum(n_atoms_cfg, out=cfg_ptr[1:])
    n_atoms = int(cfg_ptr[-1])
    X = descriptors(s, n_atoms, r.d, r.absval)
    atom_species = species_full = None
    if r.n_species > 1:
        species_full = uniform_ints(s, _AID_SPECIES, n_atoms_full, 0, r.n_species - 1).astype(np.int32)
        atom_species = np.ascontiguousarray(species_full[:n_atoms])
    sparse_idx = _sparse_set(r, species_full, n_atoms_full)
    if n_atoms == n_atoms_full:
        Xs = np.ascontiguousarray(X[sparse_idx])
    else:
        Xs = np.empty((len(sparse_idx), r.d))
        _load().gg_descriptor_rows(s, _AID_X, _ptr(sparse_idx), len(sparse_idx), r.d, int(r.absval), _ptr(Xs))
    sparse_species = None
    if species_full is not None:
        sparse_species = np.ascontiguousarray(species_full[sparse_idx])
    M = len(sparse_idx)
    c_star = normals(s, _AID_CSTAR, M)
    sigma_e = r.sigma_e_atom * np.sqrt(n_atoms_cfg.astype(np.float64))
    if r.noise_e_abs is not None:
        noise_e = normals(s, _AID_NOISE_E, k_cfg, r.noise_e_abs)
    else:
        noise_e = normals(s, _AID_NOISE_E, k_cfg) * sigma_e
    if r.two_body:
        c_star = np.concatenate([c_star, normals(s, _AID_CSTAR_2B, r.n_sparse_2b)])
    p = Problem(r, cfg_ptr, X, sparse_idx, Xs, c_star, noise_e, sigma_e,
                atom_species=atom_species, sparse_species=sparse_species)
    if r.two_body:
        p.two_body = make_two_body(r, cfg_ptr)
    if r.neighbours is not None:
        nnb = uniform_ints(s, _AID_NNB, n_atoms, r.neighbours[0], r.neighbours[1])
        pair_ptr = np.zeros(n_atoms + 1, np.int64)
        np.cumsum(nnb, out=pair_ptr[1:])
        n_pairs = int(pair_ptr[-1])
        cfg_of = np.repeat(np.arange(k_cfg, dtype=np.int64), n_atoms_cfg)
        pair_src = np.empty(n_pairs, np.int64)
        _load().gg_pair_src(s, _AID_SRC, n_atoms, _ptr(cfg_ptr), _ptr(cfg_of), _ptr(pair_ptr), _ptr(pair_src))
        if J_out is None:
            J = np.empty((n_pairs, 3, r.d), np.float64)
        else:
            J = J_out
            assert J.shape == (n_pairs, 3, r.d) and J.dtype == np.float64
        normals(s, _AID_J, n_pairs * 3 * r.d, r.j_std, out=J.reshape(-1))
        p.pair_ptr, p.pair_src, p.J = pair_ptr, pair_src, J
        p.sigma_f = np.full(3 * n_atoms, r.sigma_f)
        p.noise_f = normals(s, _AID_NOISE_F, 3 * n_atoms, r.sigma_f)
        if r.virials:
            p.pair_u = normals(s, _AID_U, 3 * n_pairs, r.u_std).reshape(n_pairs, 3)
            p.sigma_v = np.repeat(r.sigma_v_atom * np.sqrt(n_atoms_cfg.astype(np.float64)), 6)
            p.noise_v = normals(s, _AID_NOISE_V, 6 * k_cfg) * p.sigma_v
    p.extra["n_cfg_full"] = r.n_cfg
    return p


def make_part(r: Recipe, c0: int, c1: int, J_out: Optional[np.ndarray] = None) -> Problem:
    """Configurations [c0, c1) of recipe ``r``'s full problem, drawn on their own: every
    value equals ``select_configurations(make_problem(r), range(c0, c1))``'s (the
    generator is counter-based, so each array's entries are drawn at their positions in
    the full problem), with the full problem's sparse set.  Problems whose Jacobians do
    not fit in memory at once are handled part by part this way.  Not for recipes with a
    two-body block or virials."""
    if r.two_body or r.virials:
        raise ValueError("make_part does not draw two-body or virial inputs")
    s = r.seed
    n_atoms_cfg_full = uniform_ints(s, _AID_CFG, r.n_cfg, r.atoms[0], r.atoms[1])
    if not 0 <= c0 <= c1 <= r.n_cfg:
        raise ValueError("configurations [%d, %d) outside [0, %d)" % (c0, c1, r.n_cfg))
    ptr_full = np.zeros(r.n_cfg + 1, np.int64)
    np.cumsum(n_atoms_cfg_full, out=ptr_full[1:])
    a0, a1 = int(ptr_full[c0]), int(ptr_full[c1])
    n_atoms_full = int(ptr_full[-1])
    cfg_ptr = ptr_full[c0:c1 + 1] - a0
    X = descriptors(s, a1 - a0, r.d, r.absval, row0=a0)
    atom_species = species_full = None
    if r.n_species > 1:
        species_full = uniform_ints(s, _AID_SPECIES, n_atoms_full, 0, r.n_species - 1).astype(np.int32)
        atom_species = np.ascontiguousarray(species_full[a0:a1])
    sparse_idx = _sparse_set(r, species_full, n_atoms_full)
    Xs = np.empty((len(sparse_idx), r.d))
    _load().gg_descriptor_rows(s, _AID_X, _ptr(sparse_idx), len(sparse_idx), r.d, int(r.absval), _ptr(Xs))
    sparse_species = None if species_full is None else np.ascontiguousarray(species_full[sparse_idx])
    c_star = normals(s, _AID_CSTAR, len(sparse_idx))
    n_atoms_cfg = n_atoms_cfg_full[c0:c1]
    sigma_e = r.sigma_e_atom * np.sqrt(n_atoms_cfg.astype(np.float64))
    if r.noise_e_abs is not None:
        noise_e = normals(s, _AID_NOISE_E, c1 - c0, r.noise_e_abs, offset=c0)
    else:
        noise_e = normals(s, _AID_NOISE_E, c1 - c0, offset=c0) * sigma_e
    p = Problem(r, cfg_ptr, X, sparse_idx, Xs, c_star, noise_e, sigma_e,
                atom_species=atom_species, sparse_species=sparse_species)
    if r.neighbours is not None:
        # neighbour counts and pair sources of the atoms before a1 (cheap integer arrays),
        # then the part's pairs; sources renumbered from the part's first atom
        nnb = uniform_ints(s, _AID_NNB, a1, r.neighbours[0], r.neighbours[1])
        pp = np.zeros(a1 + 1, np.int64)
        np.cumsum(nnb, out=pp[1:])
        cfg_of = np.repeat(np.arange(c1, dtype=np.int64), n_atoms_cfg_full[:c1])
        src = np.empty(int(pp[-1]), np.int64)
        _load().gg_pair_src(s, _AID_SRC, a1, _ptr(ptr_full), _ptr(cfg_of), _ptr(pp), _ptr(src))
        q0, q1 = int(pp[a0]), int(pp[a1])
        if J_out is None:
            J = np.empty((q1 - q0, 3, r.d), np.float64)
        else:
            J = J_out
            assert J.shape == (q1 - q0, 3, r.d) and J.dtype == np.float64
        normals(s, _AID_J, (q1 - q0) * 3 * r.d, r.j_std, offset=q0 * 3 * r.d, out=J.reshape(-1))
        p.pair_ptr = np.ascontiguousarray(pp[a0:a1 + 1] - q0)
        p.pair_src = np.ascontiguousarray(src[q0:q1] - a0)
        p.J = J
        p.sigma_f = np.full(3 * (a1 - a0), r.sigma_f)
        p.noise_f = normals(s, _AID_NOISE_F, 3 * (a1 - a0), r.sigma_f, offset=3 * a0)
    p.extra["n_cfg_full"] = r.n_cfg
    p.extra["part"] = (c0, c1)
    return p


def fingerprint_of_recipe(r: Recipe) -> str:
    """``fingerprint(make_problem(r))`` without drawing the whole problem: the integer
    structure, and only the strided samples of X and J that the fingerprint hashes."""
    if r.two_body or r.virials:
        raise ValueError("fingerprint_of_recipe does not draw two-body or virial inputs")
    s = r.seed
    head = make_part(dataclasses_replace(r, neighbours=None), 0, 0)  # sparse set, c*
    n_atoms_cfg = uniform_ints(s, _AID_CFG, r.n_cfg, r.atoms[0], r.atoms[1])
    cfg_ptr = np.zeros(r.n_cfg + 1, np.int64)
    np.cumsum(n_atoms_cfg, out=cfg_ptr[1:])
    n_atoms = int(cfg_ptr[-1])
    h = hashlib.sha256()
    h.update(cfg_ptr.tobytes())
    h.update(head.sparse_idx.tobytes())
    pair_ptr = pair_src = None
    if r.neighbours is not None:
        nnb = uniform_ints(s, _AID_NNB, n_atoms, r.neighbours[0], r.neighbours[1])
        pair_ptr = np.zeros(n_atoms + 1, np.int64)
        np.cumsum(nnb, out=pair_ptr[1:])
        cfg_of = np.repeat(np.arange(r.n_cfg, dtype=np.int64), n_atoms_cfg)
        pair_src = np.empty(int(pair_ptr[-1]), np.int64)
        _load().gg_pair_src(s, _AID_SRC, n_atoms, _ptr(cfg_ptr), _ptr(cfg_of), _ptr(pair_ptr), _ptr(pair_src))
        h.update(pair_ptr.tobytes())
        h.update(pair_src.tobytes())
    rows = np.arange(0, n_atoms, 97, dtype=np.int64)
    Xr = np.empty((len(rows), r.d))
    _load().gg_descriptor_rows(s, _AID_X, _ptr(rows), len(rows), r.d, int(r.absval), _ptr(Xr))
    h.update(Xr.tobytes())
    if pair_src is not None:
        n_pairs = len(pair_src)
        Js = np.empty((len(range(0, n_pairs, 1009)), 3, r.d))
        for i, q in enumerate(range(0, n_pairs, 1009)):
            normals(s, _AID_J, 3 * r.d, r.j_std, offset=q * 3 * r.d, out=Js[i].reshape(-1))
        h.update(Js.tobytes())
    h.update(head.c_star.tobytes())
    n_e = r.n_cfg
    if r.noise_e_abs is not None:
        noise_e = normals(s, _AID_NOISE_E, n_e, r.noise_e_abs)
    else:
        noise_e = normals(s, _AID_NOISE_E, n_e) * (r.sigma_e_atom * np.sqrt(n_atoms_cfg.astype(np.float64)))
    h.update(noise_e.tobytes())
    if pair_src is not None:
        h.update(normals(s, _AID_NOISE_F, 3 * n_atoms, r.sigma_f).tobytes())
    return h.hexdigest()


def select_configurations(p: Problem, cfgs) -> Problem:
    """The problem made of configurations ``cfgs`` (in that order) of ``p``: their atoms,
    pairs (sources renumbered), Jacobians, displacements, noise and sigmas, with p's
    sparse set.  Data selection only (how a multi-GPU fit places configurations on ranks);
    ``rows_of`` gives the matching rows of p's targets."""
    import copy
    cfgs = np.asarray(cfgs, dtype=np.int64)
    atoms = np.concatenate([np.arange(p.cfg_ptr[A], p.cfg_ptr[A + 1]) for A in cfgs]).astype(np.int64)
    new_of = np.full(p.n_atoms, -1, np.int64)
    new_of[atoms] = np.arange(len(atoms))
    q = copy.copy(p)
    q.cfg_ptr = np.concatenate([[0], np.cumsum(np.diff(p.cfg_ptr)[cfgs])]).astype(np.int64)
    q.X = np.ascontiguousarray(p.X[atoms])
    q.noise_e = np.ascontiguousarray(p.noise_e[cfgs])
    q.sigma_e = np.ascontiguousarray(p.sigma_e[cfgs])
    if p.atom_species is not None:
        q.atom_species = np.ascontiguousarray(p.atom_species[atoms])
    if p.has_forces:
        pairs = np.concatenate([np.arange(p.pair_ptr[a], p.pair_ptr[a + 1]) for a in atoms]).astype(np.int64)
        q.pair_ptr = np.concatenate([[0], np.cumsum(np.diff(p.pair_ptr)[atoms])]).astype(np.int64)
        q.pair_src = np.ascontiguousarray(new_of[p.pair_src[pairs]])
        q.J = np.ascontiguousarray(p.J[pairs])
        rows3 = (3 * atoms[:, None] + np.arange(3)).reshape(-1)
        q.noise_f = np.ascontiguousarray(p.noise_f[rows3])
        q.sigma_f = np.ascontiguousarray(p.sigma_f[rows3])
        if p.has_virials:
            q.pair_u = np.ascontiguousarray(p.pair_u[pairs])
            rows6 = (6 * cfgs[:, None] + np.arange(6)).reshape(-1)
            q.noise_v = np.ascontiguousarray(p.noise_v[rows6])
            q.sigma_v = np.ascontiguousarray(p.sigma_v[rows6])
    if p.two_body is not None:
        tb = p.two_body
        bonds = np.concatenate([np.arange(tb.bond_ptr[a], tb.bond_ptr[a + 1]) for a in atoms]).astype(np.int64)
        q.two_body = TwoBody(np.ascontiguousarray(tb.positions[atoms]),
                             np.concatenate([[0], np.cumsum(np.diff(tb.bond_ptr)[atoms])]).astype(np.int64),
                             np.ascontiguousarray(tb.bond_r[bonds]), np.ascontiguousarray(tb.bond_u[bonds]),
                             tb.sparse_r, tb.delta, tb.theta, tb.cutoff, tb.width)
    q.extra = dict(p.extra, selected=cfgs)
    return q


def rows_of(p: Problem, cfgs) -> np.ndarray:
    """Rows of p's targets (energies, forces, virials) that belong to configurations cfgs,
    in the order select_configurations(p, cfgs) lays them out."""
    cfgs = np.asarray(cfgs, dtype=np.int64)
    rows = [cfgs]
    if p.has_forces:
        atoms = np.concatenate([np.arange(p.cfg_ptr[A], p.cfg_ptr[A + 1]) for A in cfgs]).astype(np.int64)
        rows.append(p.n_cfg + (3 * atoms[:, None] + np.arange(3)).reshape(-1))
        if p.has_virials:
            rows.append(p.n_cfg + 3 * p.n_atoms + (6 * cfgs[:, None] + np.arange(6)).reshape(-1))
    return np.concatenate(rows).astype(np.int64)


def structure(r: Recipe):
    """(cfg_ptr, pair_ptr or None) of a recipe's full problem, drawn without the float arrays."""
    n_atoms_cfg = uniform_ints(r.seed, _AID_CFG, r.n_cfg, r.atoms[0], r.atoms[1])
    cfg_ptr = np.zeros(r.n_cfg + 1, np.int64)
    np.cumsum(n_atoms_cfg, out=cfg_ptr[1:])
    if r.neighbours is None:
        return cfg_ptr, None
    nnb = uniform_ints(r.seed, _AID_NNB, int(cfg_ptr[-1]), r.neighbours[0], r.neighbours[1])
    pair_ptr = np.zeros(len(nnb) + 1, np.int64)
    np.cumsum(nnb, out=pair_ptr[1:])
    return cfg_ptr, pair_ptr


def count_shape(r: Recipe):
    """(n_atoms, n_pairs) of a recipe without drawing the float arrays."""
    s = r.seed
    n_atoms_cfg = uniform_ints(s, _AID_CFG, r.n_cfg, r.atoms[0], r.atoms[1])
    n_atoms = int(n_atoms_cfg.sum())
    n_pairs = 0
    if r.neighbours is not None:
        n_pairs = int(uniform_ints(s, _AID_NNB, n_atoms, r.neighbours[0], r.neighbours[1]).sum())
    return n_atoms, n_pairs


def sweep_recipes(n_fits: int = 64, seed: int = SEED_BASE + 4, d: int = 256):
    """Workload 4: independent fits with rows ~ logU[2000, 40000] (configurations
    of 16-128 atoms, 1 + 3 n_A rows each, added until the row target is met),
    M ~ logU[200, 2000], zeta in {2,3,4}, sigma_E in {1e-4,1e-3,1e-2}, d=256."""
    u = uniforms(seed, _AID_FIT, 4 * n_fits).reshape(n_fits, 4)
    out = []
    for f in range(n_fits):
        rows_target = math.exp(math.log(2000) + u[f, 0] * (math.log(40000) - math.log(2000)))
        M = int(round(math.exp(math.log(200) + u[f, 1] * (math.log(2000) - math.log(200)))))
        zeta = (2, 3, 4)[min(int(u[f, 2] * 3), 2)]
        sig = (1e-4, 1e-3, 1e-2)[min(int(u[f, 3] * 3), 2)]
        fseed = seed * 1000 + f
        # grow the configuration count until the design rows reach the target
        sizes = uniform_ints(fseed, _AID_CFG, 4096, 16, 128)
        rows = np.cumsum(1 + 3 * sizes)
        n_cfg = int(np.searchsorted(rows, rows_target) + 1)
        # sparse points are distinct atoms, so M cannot exceed the atom count
        M = min(M, int(sizes[:n_cfg].sum()))
        out.append(Recipe(n_cfg=n_cfg, atoms=(16, 128), d=d, n_sparse=(M,), zeta=zeta,
                          neighbours=(8, 24), sigma_e_atom=sig, seed=fseed))
    return out


def recipe_descriptors(r: Recipe):
    """The descriptor rows and atom species of recipe ``r`` (equal to make_problem's),
    without drawing its pairs and Jacobians."""
    n_atoms, _ = count_shape(r)
    X = descriptors(r.seed, n_atoms, r.d, r.absval)
    species = None
    if r.n_species > 1:
        species = uniform_ints(r.seed, _AID_SPECIES, n_atoms, 0, r.n_species - 1).astype(np.int32)
    return X, species


def cur_draws(seed: int, n_atoms: int, d: int, l: int):
    """The random inputs of a CUR choice of the sparse set: the range finder's test
    matrix omega [d x l] (standard normal) and one uniform u in (0, 1] per atom."""
    omega = normals(seed, _AID_CUR_OMEGA, d * l).reshape(d, l)
    u = 1.0 - uniforms(seed, _AID_CUR_U, n_atoms)
    return omega, u


def clustered_descriptors(seed: int, n: int, d: int, n_clusters: int, spread: float = 0.3) -> np.ndarray:
    """Unit-length nonnegative descriptor rows [n x d] of atoms in a few common and many
    rare environments: atom i belongs to cluster z with probability proportional to
    1 / (z + 1) (Zipf), and its row is |c_z + spread N(0, I)| normalised, c_z a
    normalised |N(0, I)| centre."""
    w = 1.0 / np.arange(1, n_clusters + 1)
    cdf = np.cumsum(w) / w.sum()
    z = np.minimum(np.searchsorted(cdf, uniforms(seed, _AID_CUR_Z, n), side="right"), n_clusters - 1)
    C = np.abs(normals(seed, _AID_CUR_X, n_clusters * d).reshape(n_clusters, d))
    C /= np.linalg.norm(C, axis=1, keepdims=True)
    X = np.abs(C[z] + normals(seed, _AID_CUR_X + 1000, n * d, spread).reshape(n, d))
    X /= np.linalg.norm(X, axis=1, keepdims=True)
    return np.ascontiguousarray(X)


def fingerprint(p: Problem) -> str:
    """sha256 over the integer structure and strided samples of the float inputs
    of a drawn problem (identifies the inputs stored targets belong to)."""
    h = hashlib.sha256()
    for a in (p.cfg_ptr, p.sparse_idx, p.pair_ptr, p.pair_src):
        if a is not None:
            h.update(np.ascontiguousarray(a).tobytes())
    h.update(np.ascontiguousarray(p.X[::97]).tobytes())
    if p.J is not None:
        h.update(np.ascontiguousarray(p.J[::1009]).tobytes())
    h.update(p.c_star.tobytes())
    h.update(p.noise_e.tobytes())
    if p.noise_f is not None:
        h.update(p.noise_f.tobytes())
    if p.pair_u is not None:
        h.update(p.pair_u.tobytes())
    if p.two_body is not None:
        h.update(p.two_body.bond_ptr.tobytes())
        h.update(p.two_body.bond_r.tobytes())
        h.update(p.two_body.sparse_r.tobytes())
    return h.hexdigest()


def targets_path(workload: int) -> str:
    """Stored hidden-weight targets of a workload (written by tests/golden/make_workload_targets.py)."""
    return os.path.join(os.path.dirname(_HERE), "tests", "golden", "workload%d_targets.npz" % workload)


def load_targets(p: Problem, workload: int) -> np.ndarray:
    """Stored targets y of workload ``workload``, checked against the drawn inputs."""
    z = np.load(targets_path(workload))
    if str(z["fingerprint"]) != fingerprint(p):
        raise ValueError("stored targets of workload %d belong to other inputs" % workload)
    return np.ascontiguousarray(z["y"])


def load_sweep_targets(p: Problem, f: int) -> np.ndarray:
    """Stored targets of fit f of the workload-4 sweep (``sweep_recipes()[f]``), checked
    against the drawn inputs."""
    z = np.load(targets_path(4))
    if str(z["fingerprints"][f]) != fingerprint(p):
        raise ValueError("stored targets of sweep fit %d belong to other inputs" % f)
    o = z["offsets"]
    return np.ascontiguousarray(z["y"][o[f]:o[f + 1]])


def load_targets_slice(p: Problem, workload: int) -> np.ndarray:
    """Stored targets of a ``make_problem(..., max_cfg=k)`` slice: its rows are
    the full problem's first k energy rows and first 3 n_atoms force rows (every
    kept input equals the full problem's), so they are cut out of the stored
    vector.  Only the stored row count is checked here: the fingerprint covers
    the full problem, which a slice does not draw."""
    z = np.load(targets_path(workload))
    r = p.recipe
    n_full = int(p.extra["n_cfg_full"])
    n_atoms_full, _ = count_shape(r)
    if int(z["n_rows"]) != n_full + 3 * n_atoms_full:
        raise ValueError("stored targets of workload %d have another shape" % workload)
    y = z["y"]
    return np.ascontiguousarray(np.concatenate([y[:p.n_cfg], y[n_full:n_full + 3 * p.n_atoms]]))
