"""ORACLE -- test infrastructure only.

Python entry points of the plain FP64 CPU oracle in ``oracle.c`` (the sparse-GP
fit of arXiv:2207.03803, Sec. II).  Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import this package; the GPU
library never does, and the two share no code.  Inputs come from ``gapgen``.
"""
from __future__ import annotations

import ctypes
import time as _time
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c (gcc -O2, OpenMP, no FMA contraction)."""
    src = os.path.join(_HERE, "oracle.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", "-std=c11",
                        "-o", _SO + ".tmp", src, "-lm"], check=True)
        os.replace(_SO + ".tmp", _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        p, i64, i32, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
        lib.or_kernel.argtypes = [p, p, i64, dbl, i32]
        lib.or_kernel.restype = dbl
        lib.or_design_energy.argtypes = [i64, p, i64, p, p, i64, p, p, dbl, i32, p, p]
        lib.or_design_force.argtypes = [i64, p, p, p, i64, p, p, i64, p, p, dbl, i32, p, p]
        lib.or_design_virial.argtypes = [i64, p, p, p, p, p, i64, p, p, i64, p, p, dbl, i32, p, p]
        lib.or_kmm.argtypes = [i64, i64, p, p, dbl, i32, dbl, p]
        lib.or_cholesky_upper.argtypes = [i64, p, p]
        lib.or_cholesky_upper.restype = i32
        lib.or_householder_qr.argtypes = [i64, i64, p, p]
        lib.or_apply_qt.argtypes = [i64, i64, p, p, p]
        lib.or_apply_q.argtypes = [i64, i64, p, p, p]
        lib.or_back_substitution.argtypes = [i64, p, i64, p, p]
        lib.or_back_substitution.restype = i32
        lib.or_predict.argtypes = [i64, p, i64, p, p, i64, p, p, dbl, i32, p, p, p, p, p, p, p, p]
        lib.or_fit.argtypes = [i64, p, i64, p, p, i64, p, p, dbl, i32, dbl, p, p, p, p, p, p, p, p, p]
        lib.or_fit.restype = i32
        _lib = lib
    return _lib


def _p(a):
    if a is None:
        return None
    assert isinstance(a, np.ndarray) and a.flags["C_CONTIGUOUS"], "oracle inputs must be C-contiguous"
    return a.ctypes.data


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class OracleError(RuntimeError):
    pass


def kernel(x, xs, delta, zeta):
    x, xs = _f64(x), _f64(xs)
    return _load().or_kernel(_p(x), _p(xs), x.shape[-1], delta, zeta)


def sigma(p):
    """Per-row sigma: [sigma_A for each configuration ; sigma_F per force component ;
    sigma_V per virial component]."""
    parts = [p.sigma_e]
    if p.has_forces:
        parts.append(p.sigma_f)
    if p.has_virials:
        parts.append(p.sigma_v)
    return np.concatenate(parts)


def design(p):
    """Data rows Sigma^{-1/2} K_NM of Eq. (7): [N x M], energies, forces, then virials;
    with a two-body sub-GAP its column block follows the SOAP block's."""
    out = _design_soap(p)
    if p.two_body is not None:
        from . import two_body
        out = np.hstack([out, two_body.design_2b(p)])
    return out


def _design_soap(p):
    r = p.recipe
    lib = _load()
    out = np.empty((p.n_rows, p.n_sparse))
    se = _f64(p.sigma_e)
    lib.or_design_energy(p.n_cfg, _p(p.cfg_ptr), p.d, _p(p.X), _p(p.atom_species), p.n_sparse, _p(p.Xs),
                         _p(p.sparse_species), r.delta, r.zeta, _p(se), _p(out))
    if p.has_forces:
        sub = out[p.n_cfg:p.n_cfg + 3 * p.n_atoms]
        tmp = np.empty_like(sub)
        sf = _f64(p.sigma_f)
        lib.or_design_force(p.n_atoms, _p(p.pair_ptr), _p(p.pair_src), _p(p.J), p.d, _p(p.X),
                            _p(p.atom_species), p.n_sparse, _p(p.Xs), _p(p.sparse_species), r.delta, r.zeta,
                            _p(sf), _p(tmp))
        sub[:] = tmp
    if p.has_virials:
        nf = p.n_cfg + 3 * p.n_atoms
        vo = np.empty((6 * p.n_cfg, p.n_sparse))
        lib.or_design_virial(p.n_cfg, _p(p.cfg_ptr), _p(p.pair_ptr), _p(p.pair_src), _p(p.J), _p(_f64(p.pair_u)),
                             p.d, _p(p.X), _p(p.atom_species), p.n_sparse, _p(p.Xs), _p(p.sparse_species), r.delta,
                             r.zeta, _p(_f64(p.sigma_v)), _p(vo))
        out[nf:] = vo
    return out


def kmm(p):
    """K_MM with the absolute sparse_jitter on the diagonal; block diagonal over the
    SOAP and two-body sparse points (the sub-GAPs are independent)."""
    r = p.recipe
    K = np.empty((p.n_sparse, p.n_sparse))
    _load().or_kmm(p.n_sparse, p.d, _p(p.Xs), _p(p.sparse_species), r.delta, r.zeta, r.jitter, _p(K))
    if p.two_body is not None:
        from . import two_body
        K2 = two_body.kmm_2b(p)
        Kb = np.zeros((p.n_weights, p.n_weights))
        Kb[:p.n_sparse, :p.n_sparse] = K
        Kb[p.n_sparse:, p.n_sparse:] = K2
        K = Kb
    return K


def cholesky_upper(K):
    K = _f64(K)
    U = np.empty_like(K)
    st = _load().or_cholesky_upper(K.shape[0], _p(K), _p(U))
    if st != 0:
        raise OracleError("K_MM not positive definite at pivot %d" % (st - 1))
    return U


def householder_qr(A):
    """Returns (factored A, tau) in the LAPACK geqrf layout (row-major)."""
    A = _f64(A).copy()
    m, n = A.shape
    tau = np.zeros(min(m, n))
    _load().or_householder_qr(m, n, _p(A), _p(tau))
    return A, tau


def apply_qt(QR, tau, b):
    b = _f64(b).copy()
    QR, tau = _f64(QR), _f64(tau)
    _load().or_apply_qt(QR.shape[0], QR.shape[1], _p(QR), _p(tau), _p(b))
    return b


def apply_q(QR, tau, x):
    x = _f64(x).copy()
    QR, tau = _f64(QR), _f64(tau)
    _load().or_apply_q(QR.shape[0], QR.shape[1], _p(QR), _p(tau), _p(x))
    return x


def back_substitution(R, z):
    R = _f64(R)
    n = R.shape[1]
    c = np.empty(n)
    z = _f64(z)
    st = _load().or_back_substitution(n, _p(R), R.shape[1], _p(z), _p(c))
    if st != 0:
        raise OracleError("zero diagonal in R at %d" % (st - 1))
    return c


def predict_all(p, c, with_forces=True, with_virials=True):
    """(E [n_cfg], F [3 n_atoms] or None, V [6 n_cfg] or None) of the model with weights c
    (Eqs. 1, 2 and the lattice-deformation derivatives)."""
    r = p.recipe
    E = np.empty(p.n_cfg)
    F = np.empty(3 * p.n_atoms) if (with_forces and p.has_forces) else None
    V = np.empty(6 * p.n_cfg) if (with_virials and p.has_virials) else None
    pairs = F is not None or V is not None
    c = _f64(c)
    c2 = c[p.n_sparse:]
    c = np.ascontiguousarray(c[:p.n_sparse])
    _load().or_predict(p.n_cfg, _p(p.cfg_ptr), p.d, _p(p.X), _p(p.atom_species), p.n_sparse, _p(p.Xs),
                       _p(p.sparse_species), r.delta, r.zeta, _p(c),
                       _p(p.pair_ptr) if pairs else None, _p(p.pair_src) if pairs else None,
                       _p(p.J) if pairs else None, _p(_f64(p.pair_u)) if V is not None else None,
                       _p(E), _p(F), _p(V))
    if p.two_body is not None:
        from . import two_body
        E2, F2, V2 = two_body.predict_2b(p, c2)
        E += E2
        if F is not None:
            F += F2
        if V is not None:
            V += V2
    return E, F, V


def predict(p, c, with_forces=True):
    """(E [n_cfg], F [3 n_atoms] or None) of the model with weights c (Eqs. 1, 2)."""
    E, F, _ = predict_all(p, c, with_forces=with_forces, with_virials=False)
    return E, F


def targets(p):
    """Hidden-weight targets y = K c* + noise (energies, then forces, then virials)."""
    E, F, V = predict_all(p, p.c_star)
    parts = [E + p.noise_e]
    if F is not None:
        parts.append(F + p.noise_f)
    if V is not None:
        parts.append(V + p.noise_v)
    return np.concatenate(parts) if len(parts) > 1 else parts[0]


def fit(p, y, return_factor=False):
    """Weights c of the fit of Sec. II (Eqs. 7, 8, 12).  Returns (c, times[4]) or
    (c, times, factored A) with ``return_factor``."""
    if p.two_body is not None:
        return _fit_stacked(p, y, return_factor)
    r = p.recipe
    M = p.n_sparse
    c = np.empty(M)
    times = np.zeros(4)
    Aout = np.empty((p.n_rows + M, M)) if return_factor else None
    y, sg = _f64(y), sigma(p)
    st = _load().or_fit(p.n_cfg, _p(p.cfg_ptr), p.d, _p(p.X), _p(p.atom_species), M, _p(p.Xs),
                        _p(p.sparse_species), r.delta, r.zeta, r.jitter,
                        _p(p.pair_ptr), _p(p.pair_src), _p(p.J),
                        _p(_f64(p.pair_u)) if p.has_virials else None, _p(y), _p(sg),
                        _p(c), _p(times), _p(Aout))
    if st < 0:
        raise OracleError("K_MM not positive definite at pivot %d" % (-st - 1))
    if st > 0:
        raise OracleError("zero diagonal in R at %d" % (st - 1))
    return (c, times, Aout) if return_factor else (c, times)


def _fit_stacked(p, y, return_factor=False):
    """The fit of Eqs. (7), (8), (12) from the oracle's pieces: [Sigma^{-1/2} K_NM | b]
    with U below, Householder QR, back substitution (problems with a two-body sub-GAP)."""
    t = [0.0] * 4
    t0 = _time.time()
    D = design(p)
    t[0] = _time.time() - t0
    t0 = _time.time()
    U = cholesky_upper(kmm(p))
    t[1] = _time.time() - t0
    M = p.n_weights
    b = np.concatenate([_f64(y) / sigma(p), np.zeros(M)])
    t0 = _time.time()
    QR, _ = householder_qr(np.hstack([np.vstack([D, U]), b[:, None]]))
    t[2] = _time.time() - t0
    t0 = _time.time()
    c = back_substitution(np.triu(QR[:M, :M]), QR[:M, M])
    t[3] = _time.time() - t0
    if return_factor:
        return c, np.array(t), QR[:, :M]
    return c, np.array(t)


def stacked_matrix(p):
    """A = [Sigma^{-1/2} K_NM ; U] of Eq. (7) and U, unfactored."""
    U = cholesky_upper(kmm(p))
    return np.vstack([design(p), U]), U
