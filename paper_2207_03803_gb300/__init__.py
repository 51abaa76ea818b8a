"""Python binding of libgap, the GB300 (sm_103a) sparse-GP (GAP) fitting library.

This module only marshals arguments into the C-ABI declared in ``include/gap.h``;
every step of the fit (assembly of the design matrix, K_MM and its Cholesky
factor, the Householder QR, the solves, the refinement and the predictions)
runs in the library's CUDA kernels.  PyTorch provides device memory and
streams.  There is no CPU fallback: ``load()`` raises if ``libgap.so`` has not
been built, and the library reports a CUDA error on any GPU it was not built for.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgap.so")
_lib = None

GAP_OK, GAP_ERR_INVALID, GAP_ERR_NOMEM, GAP_ERR_CUDA, GAP_ERR_NOT_SPD = 0, 1, 2, 3, 4
GAP_ERR_RANK, GAP_ERR_NOT_CONVERGED, GAP_ERR_TIMEOUT, GAP_ERR_STATE = 5, 6, 7, 8
PRECISIONS = {"fp64": 0, "mixed_bf16": 1, "mixed_tf32": 2, "mixed_fp16": 3}
GAP_MEM_DEVICE, GAP_MEM_HOST = 0, 1

# every symbol include/gap.h declares
EXPORTS = ("gap_create", "gap_destroy", "gap_last_error", "gap_set_option", "gap_workspace_size",
           "gap_design_rows", "gap_assemble", "gap_factor", "gap_solve", "gap_predict", "gap_read_design",
           "gap_read_r", "gap_fit_batched", "gap_get_profile", "gap_predict_static", "gap_tsqr_blocks", "gap_tsqr_plan",
           "gap_predict_virial", "gap_tsqr_local", "gap_tsqr_merge", "gap_select_cur", "gap_workspace_size_ring")
PROF_CLASSES = ("copy_in", "pack", "gemm_energy", "gemm_force", "kmm_chol", "qr_panel", "qr_update", "solve",
                "refine", "predict")


class GapError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("libgap status %d: %s" % (status, msg))
        self.status = status


class gap_problem(ctypes.Structure):
    _fields_ = [("n_cfg", ctypes.c_int64), ("n_atoms", ctypes.c_int64), ("d", ctypes.c_int64),
                ("n_pairs", ctypes.c_int64), ("n_sparse", ctypes.c_int64),
                ("cfg_ptr", ctypes.c_void_p), ("X", ctypes.c_void_p), ("Xs", ctypes.c_void_p),
                ("atom_species", ctypes.c_void_p), ("sparse_species", ctypes.c_void_p),
                ("pair_ptr", ctypes.c_void_p), ("pair_src", ctypes.c_void_p), ("J", ctypes.c_void_p),
                ("y", ctypes.c_void_p), ("sigma", ctypes.c_void_p),
                ("delta", ctypes.c_double), ("zeta", ctypes.c_int32), ("memory", ctypes.c_int32),
                ("jitter", ctypes.c_double), ("pair_u", ctypes.c_void_p),
                ("n_bonds", ctypes.c_int64), ("n_sparse_2b", ctypes.c_int64), ("bond_ptr", ctypes.c_void_p),
                ("bond_r", ctypes.c_void_p), ("bond_u", ctypes.c_void_p), ("sparse_r", ctypes.c_void_p),
                ("delta_2b", ctypes.c_double), ("theta_2b", ctypes.c_double), ("cutoff_2b", ctypes.c_double),
                ("width_2b", ctypes.c_double)]


class gap_profile(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * 10), ("groups", ctypes.c_int32 * 10)]


class gap_solve_info(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("converged", ctypes.c_int32), ("rel_update", ctypes.c_double),
                ("residual_norm", ctypes.c_double), ("time_ms", ctypes.c_double * 4)]

    def as_dict(self):
        return {"iterations": self.iterations, "converged": bool(self.converged), "rel_update": self.rel_update,
                "residual_norm": self.residual_norm, "time_ms": list(self.time_ms)}


def build(force=False, verbose=False):
    from . import buildlib as _b
    return _b.build(force=force, verbose=verbose)


def load():
    """The loaded libgap (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libgap.so is not built (run paper_2207_03803_gb300.build())")
        lib = ctypes.CDLL(LIB_PATH)
        P, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
        pp = ctypes.POINTER(gap_problem)
        lib.gap_create.argtypes = [ctypes.POINTER(P), i32, P]
        lib.gap_create.restype = i32
        lib.gap_destroy.argtypes = [P]
        lib.gap_destroy.restype = None
        lib.gap_last_error.argtypes = [P]
        lib.gap_last_error.restype = ctypes.c_char_p
        lib.gap_set_option.argtypes = [P, ctypes.c_char_p, dbl]
        lib.gap_set_option.restype = i32
        lib.gap_workspace_size.argtypes = [pp, i32, ctypes.POINTER(ctypes.c_size_t)]
        lib.gap_workspace_size.restype = i32
        lib.gap_workspace_size_ring.argtypes = [pp, i32, i64, ctypes.POINTER(ctypes.c_size_t)]
        lib.gap_workspace_size_ring.restype = i32
        lib.gap_design_rows.argtypes = [pp]
        lib.gap_design_rows.restype = i64
        lib.gap_assemble.argtypes = [P, pp]
        lib.gap_assemble.restype = i32
        lib.gap_factor.argtypes = [P]
        lib.gap_factor.restype = i32
        lib.gap_solve.argtypes = [P, P, ctypes.POINTER(gap_solve_info)]
        lib.gap_solve.restype = i32
        lib.gap_predict.argtypes = [P, pp, P, P, P]
        lib.gap_predict.restype = i32
        lib.gap_predict_virial.argtypes = [P, pp, P, P, P, P]
        lib.gap_predict_virial.restype = i32
        lib.gap_tsqr_local.argtypes = [P, P, ctypes.POINTER(ctypes.c_double)]
        lib.gap_tsqr_local.restype = i32
        lib.gap_tsqr_merge.argtypes = [P, ctypes.c_int, P, ctypes.c_double]
        lib.gap_tsqr_merge.restype = i32
        lib.gap_read_design.argtypes = [P, i32, i64, i64, P]
        lib.gap_read_design.restype = i32
        lib.gap_read_r.argtypes = [P, P]
        lib.gap_read_r.restype = i32
        lib.gap_tsqr_blocks.argtypes = [P]
        lib.gap_tsqr_blocks.restype = ctypes.c_int
        lib.gap_tsqr_plan.argtypes = [i64, i64, ctypes.c_int, P, P]
        lib.gap_tsqr_plan.restype = ctypes.c_int
        lib.gap_fit_batched.argtypes = [P, i32, ctypes.POINTER(pp), ctypes.POINTER(P),
                                        ctypes.POINTER(gap_solve_info)]
        lib.gap_fit_batched.restype = i32
        lib.gap_get_profile.argtypes = [P, ctypes.POINTER(gap_profile)]
        lib.gap_get_profile.restype = i32
        lib.gap_predict_static.argtypes = [pp, P, P, P, P, ctypes.c_char_p, ctypes.c_size_t]
        lib.gap_predict_static.restype = i32
        lib.gap_select_cur.argtypes = [P, i64, i64, P, i32, P, i32, i32, i32, P, P, P, P, P, ctypes.c_char_p,
                                       ctypes.c_size_t]
        lib.gap_select_cur.restype = i32
        _lib = lib
    return _lib


def _addr(a):
    """Data pointer of a torch tensor or numpy array (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"]
        return a.ctypes.data
    assert a.is_contiguous(), "tensors passed to libgap must be contiguous"
    return a.data_ptr()


class Problem:
    """A gap_problem over arrays that stay referenced for the problem's lifetime.

    Device problems take CUDA torch tensors; host problems take numpy arrays or
    CPU tensors (pinned memory makes the in-call copies asynchronous)."""

    def __init__(self, *, cfg_ptr, X, Xs, delta, zeta, jitter=1e-8, y=None, sigma=None, pair_ptr=None,
                 pair_src=None, J=None, atom_species=None, sparse_species=None, memory=None, pair_u=None,
                 bond_ptr=None, bond_r=None, bond_u=None, sparse_r=None, delta_2b=1.0, theta_2b=1.0,
                 cutoff_2b=1.0, width_2b=1.0):
        self._keep = [cfg_ptr, X, Xs, y, sigma, pair_ptr, pair_src, J, atom_species, sparse_species, pair_u,
                      bond_ptr, bond_r, bond_u, sparse_r]
        if memory is None:
            memory = GAP_MEM_HOST if isinstance(X, np.ndarray) or not X.is_cuda else GAP_MEM_DEVICE
        n_cfg = len(cfg_ptr) - 1
        n_atoms = int(X.shape[0])
        s = gap_problem()
        s.n_cfg, s.n_atoms, s.d = n_cfg, n_atoms, int(X.shape[1])
        s.n_pairs = 0 if pair_src is None else int(pair_src.shape[0])
        s.n_sparse = int(Xs.shape[0])
        s.cfg_ptr, s.X, s.Xs = _addr(cfg_ptr), _addr(X), _addr(Xs)
        s.atom_species, s.sparse_species = _addr(atom_species), _addr(sparse_species)
        s.pair_ptr, s.pair_src, s.J = _addr(pair_ptr), _addr(pair_src), _addr(J)
        s.y, s.sigma = _addr(y), _addr(sigma)
        s.pair_u = _addr(pair_u)
        s.delta, s.zeta, s.memory, s.jitter = float(delta), int(zeta), int(memory), float(jitter)
        if sparse_r is not None:  # two-body sub-GAP
            s.n_sparse_2b = int(sparse_r.shape[0])
            s.n_bonds = int(bond_r.shape[0])
            s.bond_ptr, s.bond_r, s.bond_u, s.sparse_r = _addr(bond_ptr), _addr(bond_r), _addr(bond_u), _addr(sparse_r)
            s.delta_2b, s.theta_2b = float(delta_2b), float(theta_2b)
            s.cutoff_2b, s.width_2b = float(cutoff_2b), float(width_2b)
        self.struct = s

    @property
    def n_rows(self):
        return load().gap_design_rows(ctypes.byref(self.struct))

    @property
    def X(self):
        """The descriptor rows the problem was built over."""
        return self._keep[1]


def workspace_size(problem: Problem, precision="fp64", j_ring_rows: int = 0) -> int:
    """Device bytes of a fit of this problem (gap_workspace_size, or with the option
    "j_ring_rows" gap_workspace_size_ring)."""
    out = ctypes.c_size_t()
    if j_ring_rows:
        st = load().gap_workspace_size_ring(ctypes.byref(problem.struct), PRECISIONS[precision], int(j_ring_rows),
                                            ctypes.byref(out))
    else:
        st = load().gap_workspace_size(ctypes.byref(problem.struct), PRECISIONS[precision], ctypes.byref(out))
    if st != GAP_OK:
        raise GapError(st, "workspace_size")
    return out.value


def tsqr_plan(n_data_rows: int, n_sparse: int, want: int) -> list:
    """Row blocks (first row, rows) of the TSQR factorisation for this many data rows,
    sparse points and "tsqr_shards" (empty: one QR of the whole matrix)."""
    r0 = (ctypes.c_int64 * 64)()
    n = (ctypes.c_int64 * 64)()
    G = load().gap_tsqr_plan(n_data_rows, n_sparse, want, r0, n)
    if G < 0:
        raise GapError(GAP_ERR_INVALID, "negative sizes")
    return [(int(r0[g]), int(n[g])) for g in range(G)]


def design_rows(problem: Problem) -> int:
    return load().gap_design_rows(ctypes.byref(problem.struct))


class Context:
    """A gap_ctx bound to a CUDA stream (default: torch's current stream)."""

    def __init__(self, precision="fp64", stream=None):
        import torch
        self.lib = load()
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        self.precision = precision
        h = ctypes.c_void_p()
        st = self.lib.gap_create(ctypes.byref(h), PRECISIONS[precision], ctypes.c_void_p(stream.cuda_stream))
        if st != GAP_OK:
            raise GapError(st, "gap_create failed")
        self.h = h

    def _check(self, st):
        if st != GAP_OK:
            raise GapError(st, self.lib.gap_last_error(self.h).decode())

    def set_option(self, key: str, value: float):
        self._check(self.lib.gap_set_option(self.h, key.encode(), float(value)))

    def assemble(self, problem: Problem):
        self._problem = problem
        self._check(self.lib.gap_assemble(self.h, ctypes.byref(problem.struct)))

    def factor(self):
        self._check(self.lib.gap_factor(self.h))

    def solve(self, c_out, check=True) -> dict:
        info = gap_solve_info()
        st = self.lib.gap_solve(self.h, _addr(c_out), ctypes.byref(info))
        d = info.as_dict()
        d["status"] = st
        if check:
            self._check(st)
        return d

    def predict(self, targets: Optional[Problem], c, E_out, F_out=None):
        """gap_predict; targets None predicts for the last assembled problem."""
        tp = ctypes.byref(targets.struct) if targets is not None else None
        self._check(self.lib.gap_predict(self.h, tp, _addr(c), _addr(E_out), _addr(F_out)))

    def predict_virial(self, targets: Optional[Problem], c, E_out, F_out=None, V_out=None):
        """gap_predict_virial: energies, forces (F_out may be None) and the six virial
        components per configuration (V_out [6 n_cfg])."""
        tp = ctypes.byref(targets.struct) if targets is not None else None
        self._check(self.lib.gap_predict_virial(self.h, tp, _addr(c), _addr(E_out), _addr(F_out), _addr(V_out)))

    def tsqr_local(self, Rz_out) -> float:
        """gap_tsqr_local: [R_g | z_g] of this ctx's assembled row block into Rz_out (device,
        [M, M + 1] FP64); returns the squared norm of the block's residual tail."""
        t2 = ctypes.c_double()
        self._check(self.lib.gap_tsqr_local(self.h, _addr(Rz_out), ctypes.byref(t2)))
        return t2.value

    def tsqr_merge(self, Rz_blocks, tail2: float):
        """gap_tsqr_merge: the QR of the G stacked blocks (device, [G, M, M + 1] FP64) on U."""
        self._check(self.lib.gap_tsqr_merge(self.h, int(Rz_blocks.shape[0]), _addr(Rz_blocks), float(tail2)))

    def read_design(self, which: int, row0: int, nrows: int, out):
        self._check(self.lib.gap_read_design(self.h, which, row0, nrows, _addr(out)))

    def profile(self) -> dict:
        """Device ms and launch-group counts per kernel class since the last assemble."""
        pr = gap_profile()
        self._check(self.lib.gap_get_profile(self.h, ctypes.byref(pr)))
        return {k: {"ms": pr.ms[i], "groups": pr.groups[i]} for i, k in enumerate(PROF_CLASSES)}

    def read_r(self, out):
        self._check(self.lib.gap_read_r(self.h, _addr(out)))

    def tsqr_blocks(self) -> int:
        """Row blocks of the last factor's TSQR (0: one QR of the whole matrix)."""
        return int(self.lib.gap_tsqr_blocks(self.h))

    def fit_batched(self, problems: Sequence[Problem], c_outs: Sequence) -> list:
        n = len(problems)
        arr = (ctypes.POINTER(gap_problem) * n)(*[ctypes.pointer(p.struct) for p in problems])
        cs = (ctypes.c_void_p * n)(*[_addr(c) for c in c_outs])
        infos = (gap_solve_info * n)()
        self._check(self.lib.gap_fit_batched(self.h, n, arr, cs, infos))
        return [i.as_dict() for i in infos]

    def close(self):
        if getattr(self, "h", None):
            self.lib.gap_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def predict_static(targets: Problem, c, E_out, F_out=None, stream=None):
    """gap_predict_static: predictions with no device allocation (scratch in the
    library's fixed-size device array); device tensors only."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    err = ctypes.create_string_buffer(256)
    st = load().gap_predict_static(ctypes.byref(targets.struct), _addr(c), _addr(E_out), _addr(F_out),
                                   ctypes.c_void_p(stream.cuda_stream), err, len(err))
    if st != GAP_OK:
        raise GapError(st, err.value.decode())


def select_cur(X, n_select, k, l, omega, u, power_iters=2, atom_species=None, leverage=False, stream=None):
    """gap_select_cur: CUR (leverage-score) choice of the sparse set, per species.

    X [n_atoms, d], omega [d, l] and u [n_atoms] are FP64 CUDA tensors, atom_species
    an int32 CUDA tensor (or None for one species), n_select a sequence of counts per
    species.  Returns the chosen atom indices (int64 CUDA tensor, species after
    species, ascending within each) and, with leverage=True, the leverage scores
    [n_atoms] (NaN for the atoms of species with no sparse points)."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    for name, t in (("X", X), ("omega", omega), ("u", u)):
        if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
            raise ValueError("%s must be a contiguous float64 CUDA tensor" % name)
    if atom_species is not None and not (atom_species.is_cuda and atom_species.dtype == torch.int32
                                         and atom_species.is_contiguous()):
        raise ValueError("atom_species must be a contiguous int32 CUDA tensor")
    n_atoms, d = X.shape
    counts = np.ascontiguousarray(np.asarray(n_select, dtype=np.int64))
    sel = torch.empty(int(counts.sum()), dtype=torch.int64, device=X.device)
    lev = torch.full((n_atoms,), float("nan"), dtype=torch.float64, device=X.device) if leverage else None
    err = ctypes.create_string_buffer(256)
    st = load().gap_select_cur(_addr(X), n_atoms, d, _addr(atom_species), len(counts), counts.ctypes.data, k, l,
                               power_iters, _addr(omega), _addr(u), _addr(sel), _addr(lev),
                               ctypes.c_void_p(stream.cuda_stream), err, len(err))
    if st != GAP_OK:
        raise GapError(st, err.value.decode())
    return (sel, lev) if leverage else sel


def problem_from_arrays(p, y, device="cuda", pinned=False) -> Problem:
    """A Problem over the arrays of a ``gapgen.Problem`` plus targets ``y``.

    device='cuda' copies every array into device tensors (a device problem);
    device='cpu' keeps host arrays (pinned=True copies them into pinned tensors)."""
    import torch
    sigma = [p.sigma_e] + ([p.sigma_f] if p.has_forces else []) + ([p.sigma_v] if p.has_virials else [])
    arrs = dict(cfg_ptr=p.cfg_ptr, X=p.X, Xs=p.Xs, y=np.ascontiguousarray(y, dtype=np.float64),
                sigma=np.ascontiguousarray(np.concatenate(sigma), dtype=np.float64))
    if p.has_forces:
        arrs.update(pair_ptr=p.pair_ptr, pair_src=p.pair_src, J=p.J)
    if p.has_virials:
        arrs.update(pair_u=p.pair_u)
    if p.atom_species is not None:
        arrs.update(atom_species=p.atom_species, sparse_species=p.sparse_species)
    scal = {}
    if getattr(p, "two_body", None) is not None:
        tb = p.two_body
        arrs.update(bond_ptr=tb.bond_ptr, bond_r=tb.bond_r, bond_u=tb.bond_u, sparse_r=tb.sparse_r)
        scal = dict(delta_2b=tb.delta, theta_2b=tb.theta, cutoff_2b=tb.cutoff, width_2b=tb.width)
    if device == "cuda":
        t = {k: torch.from_numpy(np.ascontiguousarray(v)).to("cuda") for k, v in arrs.items()}
        return Problem(delta=p.recipe.delta, zeta=p.recipe.zeta, jitter=p.recipe.jitter, memory=GAP_MEM_DEVICE, **t,
                       **scal)
    if pinned:
        t = {k: torch.from_numpy(np.ascontiguousarray(v)).pin_memory() for k, v in arrs.items()}
        return Problem(delta=p.recipe.delta, zeta=p.recipe.zeta, jitter=p.recipe.jitter, memory=GAP_MEM_HOST, **t,
                       **scal)
    return Problem(delta=p.recipe.delta, zeta=p.recipe.zeta, jitter=p.recipe.jitter, memory=GAP_MEM_HOST,
                   **{k: np.ascontiguousarray(v) for k, v in arrs.items()}, **scal)
