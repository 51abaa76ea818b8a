"""GPU parity: libgap (through its C-ABI) against the FP64 oracle on the same
seeded inputs.  Sizes span several tiles with ragged tails (M, d and the atom,
pair and configuration counts are not multiples of any tile size).

Gates (relative L2 error of predicted energies and forces against the
oracle's fit): 1e-8 in FP64 mode, 1e-6 in the mixed precisions after FP64
refinement.  The error of c is reported, not gated (the weights of an
ill-conditioned fit agree to fewer digits than its predictions, Sec. IV).
"""
import dataclasses

import numpy as np
import pytest

import gapgen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2207_03803_gb300 as gapgpu  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def built():
    gapgpu.build()
    gapgpu.load()


def rel(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def recipe(seed=21, n_cfg=37, atoms=(3, 128), d=47, M=150, zeta=4, nb=(0, 20), n_species=1, sparse=None,
           absval=True, delta=1.0, sigma_e=None, virials=False):
    kw = {} if sigma_e is None else {"sigma_e_atom": sigma_e}
    if virials:
        kw["virials"] = True
    return gapgen.Recipe(n_cfg=n_cfg, atoms=atoms, d=d, n_sparse=sparse or (M,), zeta=zeta, delta=delta,
                         neighbours=nb, n_species=n_species, absval=absval, seed=seed, **kw)


_cache = {}


def problem(key, **kw):
    if key not in _cache:
        p = gapgen.make_problem(recipe(**kw))
        y = oracle.targets(p)
        c, _ = oracle.fit(p, y)
        E, F = oracle.predict(p, c)
        _cache[key] = (p, y, c, E, F)
    return _cache[key]


def gpu_fit(p, y, precision, device="cuda", **opts):
    prob = gapgpu.problem_from_arrays(p, y, device=device)
    ctx = gapgpu.Context(precision)
    for k, v in opts.items():
        ctx.set_option(k, v)
    ctx.assemble(prob)
    ctx.factor()
    c = torch.empty(p.n_sparse, dtype=torch.float64, device="cuda")
    info = ctx.solve(c)
    return ctx, prob, c, info


def gpu_predict(ctx, p, c):
    tgt = gapgpu.problem_from_arrays(p, np.zeros(p.n_rows), device="cuda")
    E = torch.empty(p.n_cfg, dtype=torch.float64, device="cuda")
    F = torch.empty(3 * p.n_atoms, dtype=torch.float64, device="cuda") if p.has_forces else None
    ctx.predict(tgt, c, E, F)
    return E.cpu().numpy(), (F.cpu().numpy() if F is not None else None)


# ------------------------------------------------------------- assembly --

@pytest.mark.parametrize("precision", ["fp64", "mixed_tf32", "mixed_bf16", "mixed_fp16"])
def test_design_rows_match_oracle(precision):
    p, y, *_ = problem("base")
    prob = gapgpu.problem_from_arrays(p, y)
    ctx = gapgpu.Context(precision)
    ctx.assemble(prob)
    ref = oracle.design(p)
    out = torch.empty((p.n_rows, p.n_sparse), dtype=torch.float64, device="cuda")
    ctx.read_design(1, 0, p.n_rows, out)
    got = out.cpu().numpy()
    tol = 1e-12 if precision == "fp64" else 2e-6
    print(precision, "energy rows %.2e force rows %.2e" % (rel(got[:p.n_cfg], ref[:p.n_cfg]),
                                                          rel(got[p.n_cfg:], ref[p.n_cfg:])))
    # the mixed precisions' energy rows come from a double-float epilogue, in FP64
    assert rel(got[:p.n_cfg], ref[:p.n_cfg]) < (tol if precision == "fp64" else 2e-7)
    assert rel(got[p.n_cfg:], ref[p.n_cfg:]) < tol
    # elementwise on a sample of entries (relative to the row scale)
    scale = np.abs(ref).max(axis=1, keepdims=True) + 1e-300
    assert np.max(np.abs(got - ref) / scale) < (1e-12 if precision == "fp64" else 1e-5)
    if precision != "fp64":
        ctx.read_design(0, 0, p.n_rows, out)
        lo = out.cpu().numpy()
        # single-pass BF16/TF32 products: accurate to their input rounding only
        assert rel(lo, ref) < (5e-3 if precision == "mixed_tf32" else 3e-2)
        if precision == "mixed_fp16":  # FP16 force rows: 11 significant bits per operand
            assert rel(lo[p.n_cfg:], ref[p.n_cfg:]) < 2e-3


@pytest.mark.parametrize("precision", ["mixed_tf32", "mixed_bf16"])
def test_regulariser_rows_match_oracle(precision):
    """The U rows (Cholesky factor of K_MM + jitter, with K_MM's dot products in
    double-float on the FP32 units in the mixed precisions) stacked under the data
    rows, against the oracle's FP64 U, to the FP32 rounding of the stored matrix."""
    p, y, *_ = problem("base")
    ctx, *_ = gpu_fit(p, y, precision)
    out = torch.empty((p.n_sparse, p.n_sparse), dtype=torch.float64, device="cuda")
    ctx.read_design(1, p.n_rows, p.n_sparse, out)
    A, _ = oracle.stacked_matrix(p)
    assert rel(out.cpu().numpy(), A[p.n_rows:]) < 1e-6


def test_species_design_rows():
    p, y, *_ = problem("species", n_species=3, sparse=(40, 37, 45), atoms=(5, 60), n_cfg=30)
    prob = gapgpu.problem_from_arrays(p, y)
    ctx = gapgpu.Context("fp64")
    ctx.assemble(prob)
    out = torch.empty((p.n_rows, p.n_sparse), dtype=torch.float64, device="cuda")
    ctx.read_design(0, 0, p.n_rows, out)
    assert rel(out.cpu().numpy(), oracle.design(p)) < 1e-12


@pytest.mark.parametrize("precision,gate", [("fp64", 1e-8), ("mixed_bf16", 1e-6)])
def test_species_fit_in_either_sparse_order(precision, gate):
    """Three species with the sparse points grouped by species (K_MM block diagonal, its
    Cholesky factored block by block) and interleaved (one block): both fits against the
    oracle's fit of each ordering (the same model, its weights permuted)."""
    p, y, c_or, E_or, F_or = problem("species_fit", n_species=3, sparse=(40, 37, 45), atoms=(5, 60), n_cfg=30)
    assert np.all(np.diff(p.sparse_species) >= 0)  # grouped by species
    import copy
    q = copy.copy(p)
    perm = np.argsort(np.arange(p.n_sparse) % 7, kind="stable")  # interleaves the species
    q.sparse_idx, q.Xs = p.sparse_idx[perm], np.ascontiguousarray(p.Xs[perm])
    q.sparse_species, q.c_star = np.ascontiguousarray(p.sparse_species[perm]), p.c_star[perm]
    assert np.any(np.diff(q.sparse_species) < 0)
    for pp in (p, q):
        ctx, prob, c, info = gpu_fit(pp, y, precision)
        E1, F1 = oracle.predict(pp, c.cpu().numpy())
        print(precision, "grouped" if pp is p else "interleaved", "E %.2e F %.2e" % (rel(E1, E_or), rel(F1, F_or)))
        assert rel(E1, E_or) < gate and rel(F1, F_or) < gate
        ctx.close()


# ------------------------------------------------------------- full fit --

@pytest.mark.parametrize("precision,gate", [("fp64", 1e-8), ("mixed_tf32", 1e-6), ("mixed_bf16", 1e-6),
                                            ("mixed_fp16", 1e-6)])
def test_fit_predictions_match_oracle(precision, gate):
    p, y, c_or, E_or, F_or = problem("base")
    ctx, prob, c, info = gpu_fit(p, y, precision)
    c_gpu = c.cpu().numpy()
    # the fitted model evaluated by the oracle (isolates the fit)
    E1, F1 = oracle.predict(p, c_gpu)
    print(precision, "c rel err %.2e" % rel(c_gpu, c_or), "E %.2e F %.2e" % (rel(E1, E_or), rel(F1, F_or)), info)
    assert rel(E1, E_or) < gate and rel(F1, F_or) < gate
    # the same through the library's own prediction kernels
    E2, F2 = gpu_predict(ctx, p, c)
    assert rel(E2, E_or) < gate and rel(F2, F_or) < gate
    if precision != "fp64":
        assert info["converged"] and info["iterations"] >= 1


def test_r_factor_matches_oracle_up_to_row_signs():
    p, y, *_ = problem("base")
    ctx, *_ = gpu_fit(p, y, "fp64")
    R = torch.empty((p.n_sparse, p.n_sparse), dtype=torch.float64, device="cuda")
    ctx.read_r(R)
    A, _ = oracle.stacked_matrix(p)
    QR, _ = oracle.householder_qr(A)
    R_or = np.triu(QR[:p.n_sparse])
    assert rel(np.abs(R.cpu().numpy()), np.abs(R_or)) < 1e-10


def _tsqr_blocks(N, M, want):
    """libgap's TSQR plan: up to `want` row blocks of whole 128-row tiles, each at least
    M + 128 rows long; none when N < M + 128 or the column (N + M rounded up to 128
    rows) leaves less than 128 rows after the data."""
    ld = -(-(N + M) // 128) * 128
    if want < 1 or N < M + 128 or ld < N + 128:
        return 0
    G = min(want, 64)
    while G > 1 and (N // G) // 128 * 128 < M + 128:
        G -= 1
    return G


@pytest.mark.parametrize("shards", [1, 4, 7])
@pytest.mark.parametrize("precision,gate,r_tol", [("fp64", 1e-8, 1e-10), ("mixed_tf32", 1e-6, 5e-3),
                                                  ("mixed_bf16", 1e-6, 5e-3)])
def test_tsqr_factor_matches_oracle(precision, gate, r_tol, shards):
    """The row-block (TSQR) factorisation: blocks of 1024 rows with a ragged last one,
    merged with U; same R up to row signs, same predictions, and in FP64 the same
    residual norm as the one-matrix QR."""
    p, y, c_or, E_or, F_or = problem("base")
    ctx, prob, c, info = gpu_fit(p, y, precision, tsqr_shards=shards)
    G = ctx.tsqr_blocks()
    assert G == _tsqr_blocks(p.n_rows, p.n_sparse, shards) and G >= 1
    E1, F1 = oracle.predict(p, c.cpu().numpy())
    print(precision, shards, G, "E %.2e F %.2e" % (rel(E1, E_or), rel(F1, F_or)), info["iterations"])
    assert rel(E1, E_or) < gate and rel(F1, F_or) < gate
    E2, F2 = gpu_predict(ctx, p, c)
    assert rel(E2, E_or) < gate and rel(F2, F_or) < gate
    R = torch.empty((p.n_sparse, p.n_sparse), dtype=torch.float64, device="cuda")
    ctx.read_r(R)
    A, _ = oracle.stacked_matrix(p)
    QR, _ = oracle.householder_qr(A)
    assert rel(np.abs(R.cpu().numpy()), np.abs(np.triu(QR[:p.n_sparse]))) < r_tol
    if precision == "fp64":
        *_, info1 = gpu_fit(p, y, "fp64")
        assert abs(info["residual_norm"] - info1["residual_norm"]) < 1e-10 * info1["residual_norm"]
    else:
        assert info["converged"]


def test_tsqr_two_level_outer_panels_and_short_problems():
    """TSQR blocks under the two-level FP32 QR (M = 300: outer panels of 128 with a
    ragged last one), and a problem too short for any block (one QR instead)."""
    p, y, c_ref, E_ref, F_ref = problem("qr2", n_cfg=60, atoms=(3, 60), M=300, d=40, zeta=3)
    ctx, _, c, info = gpu_fit(p, y, "mixed_tf32", tsqr_shards=3)
    assert ctx.tsqr_blocks() == _tsqr_blocks(p.n_rows, p.n_sparse, 3) >= 2
    assert info["converged"]
    E, F = gpu_predict(ctx, p, c)
    assert rel(E, E_ref) < 1e-6 and rel(F, F_ref) < 1e-6
    q = gapgen.make_problem(gapgen.RECIPES[1])
    yq = oracle.targets(q)
    ctx, _, c, info = gpu_fit(q, yq, "fp64", tsqr_shards=4)
    assert ctx.tsqr_blocks() == 0
    c_or, _ = oracle.fit(q, yq)
    E_or, _ = oracle.predict(q, c_or)
    E, _ = gpu_predict(ctx, q, c)
    assert rel(E, E_or) < 1e-8


_w5 = {}


@pytest.mark.parametrize("precision,gate", [("fp64", 1e-8), ("mixed_tf32", 1e-6), ("mixed_bf16", 1e-6),
                                            ("mixed_fp16", 1e-6)])
def test_workload5_reduced(precision, gate):
    """The workload-5 recipe with 60 configurations and 54 + 53 + 53 sparse points:
    three species (kernel zero across species), d = 1024 (the longest contraction of
    any workload: 32 k-blocks of the BF16 GEMMs), zeta = 4, energies and forces."""
    if not _w5:
        r = dataclasses.replace(gapgen.RECIPES[5], n_cfg=60, n_sparse=(54, 53, 53))
        p = gapgen.make_problem(r)
        y = oracle.targets(p)
        c, _ = oracle.fit(p, y)
        _w5.update(p=p, y=y, E=oracle.predict(p, c))
    p, y, (E_or, F_or) = _w5["p"], _w5["y"], _w5["E"]
    ctx, prob, c, info = gpu_fit(p, y, precision)
    E1, F1 = oracle.predict(p, c.cpu().numpy())
    E2, F2 = gpu_predict(ctx, p, c)
    print("workload 5 reduced", precision, "E %.2e F %.2e" % (rel(E1, E_or), rel(F1, F_or)), info["iterations"])
    assert rel(E1, E_or) < gate and rel(F1, F_or) < gate
    assert rel(E2, E_or) < gate and rel(F2, F_or) < gate


def test_energy_only_workload_1():
    """Workload 1 (64 configurations, d=32, M=64, zeta=2, energies only), both precisions."""
    p = gapgen.make_problem(gapgen.RECIPES[1])
    y = oracle.targets(p)
    c_or, _ = oracle.fit(p, y)
    E_or, _ = oracle.predict(p, c_or)
    for precision, gate in (("fp64", 1e-8), ("mixed_tf32", 1e-6), ("mixed_bf16", 1e-6)):
        ctx, prob, c, info = gpu_fit(p, y, precision)
        E, _ = gpu_predict(ctx, p, c)
        assert rel(E, E_or) < gate, precision


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed_tf32", 2e-6), ("mixed_bf16", 1e-6)])
def test_predict_kernel_matches_oracle_for_given_weights(precision, tol):
    """FP64 SIMT predictions to rounding; the mixed precisions' tensor-core
    predictions (split products accurate to FP32, FP64 sums) to FP32 level."""
    p, y, *_ = problem("base")
    ctx, prob, c, info = gpu_fit(p, y, precision)
    w = gapgen.normals(5, 1, p.n_sparse)
    E_or, F_or = oracle.predict(p, w)
    E, F = gpu_predict(ctx, p, torch.from_numpy(w).cuda())
    assert rel(E, E_or) < tol and rel(F, F_or) < tol


# ------------------------------------------------------------ edge cases --

@pytest.mark.parametrize("precision", ["fp64", "mixed_bf16"])
def test_host_memory_problem_equals_device_problem(precision):
    """A host problem gives the same fit as its device copy.  In the mixed precisions
    the host J is staged in chunks on a copy stream, and the force pass runs on each
    chunk as it lands."""
    p, y, *_ = problem("base")
    _, _, c_dev, _ = gpu_fit(p, y, precision)
    _, _, c_host, _ = gpu_fit(p, y, precision, device="cpu")
    assert torch.equal(c_dev, c_host)


def test_predict_without_targets_uses_the_assembled_problem():
    """gap_predict(NULL): the problem of the last gap_assemble from its device copies,
    for host and device problems; host targets replace those copies (GAP_ERR_STATE)."""
    p, y, c_or, E_or, F_or = problem("base")
    for device in ("cuda", "cpu"):
        ctx, prob, c, info = gpu_fit(p, y, "mixed_bf16", device=device)
        E0, F0 = gpu_predict(ctx, p, c)
        E1 = torch.empty(p.n_cfg, dtype=torch.float64, device="cuda")
        F1 = torch.empty(3 * p.n_atoms, dtype=torch.float64, device="cuda")
        ctx.predict(None, c, E1, F1)
        assert rel(E1.cpu().numpy(), E0) < 1e-12 and rel(F1.cpu().numpy(), F0) < 1e-12
        assert rel(E1.cpu().numpy(), E_or) < 1e-6 and rel(F1.cpu().numpy(), F_or) < 1e-6
    host = gapgpu.problem_from_arrays(p, np.zeros(p.n_rows), device="cpu")
    ctx.predict(host, c, E1, F1)
    with pytest.raises(gapgpu.GapError) as e:
        ctx.predict(None, c, E1, F1)
    assert e.value.status == gapgpu.GAP_ERR_STATE


def test_bitwise_reproducible():
    p, y, *_ = problem("base")
    c1 = gpu_fit(p, y, "fp64")[2]
    c2 = gpu_fit(p, y, "fp64")[2]
    assert torch.equal(c1, c2)


@pytest.mark.parametrize("kw", [dict(atoms=(1, 3), n_cfg=60, M=20, d=9),          # one-atom configurations
                                dict(M=1, n_cfg=12, d=5),                          # a single sparse point
                                dict(nb=None, n_cfg=50, M=33, d=17),               # energies only
                                dict(atoms=(126, 128), n_cfg=9, M=65, d=16, zeta=1),  # full tiles, zeta=1
                                dict(zeta=3, absval=False, delta=0.7, M=129)])     # signed descriptors
def test_edge_shapes(kw):
    p, y, c_or, E_or, F_or = problem(str(sorted(kw.items())), **kw)
    ctx, prob, c, info = gpu_fit(p, y, "fp64")
    E, F = gpu_predict(ctx, p, c)
    assert rel(E, E_or) < 1e-8
    if F_or is not None:
        assert rel(F, F_or) < 1e-8


@pytest.mark.parametrize("kw", [dict(M=1, n_cfg=12, d=5),                          # a single sparse point
                                dict(nb=None, n_cfg=50, M=33, d=17),               # energies only
                                dict(zeta=3, absval=False, delta=0.7, M=129)])     # signed descriptors
def test_edge_shapes_mixed(kw):
    """Edge shapes through the mixed precision: K_MM factored with a double-float
    trailing matrix (one panel, a one-column last panel, a ragged 64-row tile), the
    QR in FP32, refinement to the mixed gate."""
    p, y, c_or, E_or, F_or = problem(str(sorted(kw.items())), **kw)
    ctx, prob, c, info = gpu_fit(p, y, "mixed_bf16")
    E, F = gpu_predict(ctx, p, c)
    assert info["converged"]
    assert rel(E, E_or) < 1e-6
    if F_or is not None:
        assert rel(F, F_or) < 1e-6



# Segment shapes of the tensor-core epilogues.  The energy pass sums the atoms of a
# configuration along a 128-atom tile; configurations of 129-400 atoms span three or
# more tiles, each adding its partial sum.  The force pass sums the pairs of a target
# along 64-row half-tiles of Jacobian rows (three per pair); targets with 43-80 pairs
# own 129-240 rows, so their sums cross one or two 128-row tiles and their run is too
# long for the staged stores.  One-atom configurations and zeta = 1 (power 0 in the
# force weights) complete the set.
SEGMENT_SHAPES = {
    "configurations of 129-400 atoms": dict(atoms=(129, 400), n_cfg=7, M=150, d=47, nb=(2, 6)),
    "targets of 43-80 pairs": dict(atoms=(3, 20), n_cfg=14, M=100, d=40, nb=(43, 80)),
    "both, three species": dict(atoms=(100, 300), n_cfg=6, d=33, nb=(30, 70), n_species=3,
                                sparse=(50, 45, 40)),
    "one-atom configurations": dict(atoms=(1, 3), n_cfg=60, M=20, d=9),
    "zeta = 1": dict(atoms=(126, 128), n_cfg=9, M=40, d=47, zeta=1),
}


@pytest.mark.parametrize("shape", sorted(SEGMENT_SHAPES))
@pytest.mark.parametrize("precision", ["mixed_bf16", "mixed_tf32", "mixed_fp16"])
def test_segment_shapes_mixed(precision, shape):
    """Design rows of both mixed matrices against the oracle for every segment shape,
    then the refined fit's predictions at the mixed gate."""
    kw = SEGMENT_SHAPES[shape]
    p, y, c_or, E_or, F_or = problem("seg " + shape, **kw)
    prob = gapgpu.problem_from_arrays(p, y)
    ctx = gapgpu.Context(precision)
    ctx.assemble(prob)
    ref = oracle.design(p)
    out = torch.empty((p.n_rows, p.n_sparse), dtype=torch.float64, device="cuda")
    ctx.read_design(1, 0, p.n_rows, out)
    got = out.cpu().numpy()
    e_err, f_err = rel(got[:p.n_cfg], ref[:p.n_cfg]), rel(got[p.n_cfg:], ref[p.n_cfg:])
    print(shape, precision, "energy rows %.2e force rows %.2e" % (e_err, f_err))
    assert e_err < 2e-7 and f_err < 2e-6
    scale = np.abs(ref).max(axis=1, keepdims=True) + 1e-300
    assert np.max(np.abs(got - ref) / scale) < 1e-5
    ctx.read_design(0, 0, p.n_rows, out)
    assert rel(out.cpu().numpy(), ref) < (5e-3 if precision == "mixed_tf32" else 3e-2)
    ctx.factor()
    c = torch.empty(p.n_sparse, dtype=torch.float64, device="cuda")
    info = ctx.solve(c)
    assert info["converged"]
    E1, F1 = oracle.predict(p, c.cpu().numpy())
    E2, F2 = gpu_predict(ctx, p, c)
    print(shape, precision, "E %.2e F %.2e" % (rel(E1, E_or), rel(F1, F_or)), info["iterations"])
    assert rel(E1, E_or) < 1e-6 and rel(F1, F_or) < 1e-6
    assert rel(E2, E_or) < 1e-6 and rel(F2, F_or) < 1e-6


@pytest.mark.parametrize("shape", ["configurations of 129-400 atoms", "targets of 43-80 pairs",
                                   "both, three species"])
def test_segment_shapes_fp64(shape):
    """The FP64 path on the long segments: a segment cut into three or more tiles is
    summed by atomic adds in arrival order, so the rows match the oracle to rounding
    (not bit for bit between runs)."""
    p, y, c_or, E_or, F_or = problem("seg " + shape, **SEGMENT_SHAPES[shape])
    ctx = gapgpu.Context("fp64")
    ctx.assemble(gapgpu.problem_from_arrays(p, y))
    out = torch.empty((p.n_rows, p.n_sparse), dtype=torch.float64, device="cuda")
    ctx.read_design(0, 0, p.n_rows, out)  # the QR matrix, readable until gap_factor
    assert rel(out.cpu().numpy(), oracle.design(p)) < 1e-12
    ctx.factor()
    c = torch.empty(p.n_sparse, dtype=torch.float64, device="cuda")
    ctx.solve(c)
    E, F = gpu_predict(ctx, p, c)
    assert rel(E, E_or) < 1e-8 and rel(F, F_or) < 1e-8


# Virial rows (Sec. II, lattice-deformation derivatives): six per configuration after the
# force rows, the force rows of two pseudo-targets per configuration whose pseudo-pairs are
# its atoms, with the strain Jacobians G_i = sum over i's pairs of sym(J_p u_p^T).
VIRIAL = dict(n_cfg=23, atoms=(3, 90), d=41, M=110, nb=(1, 14), zeta=3, virials=True, seed=57)


def _virial_gpu_predict(ctx, p, c):
    tgt = gapgpu.problem_from_arrays(p, np.zeros(p.n_rows), device="cuda")
    E = torch.empty(p.n_cfg, dtype=torch.float64, device="cuda")
    F = torch.empty(3 * p.n_atoms, dtype=torch.float64, device="cuda")
    V = torch.empty(6 * p.n_cfg, dtype=torch.float64, device="cuda")
    ctx.predict_virial(tgt, c, E, F, V)
    return E.cpu().numpy(), F.cpu().numpy(), V.cpu().numpy()


@pytest.mark.parametrize("precision", ["fp64", "mixed_bf16", "mixed_tf32", "mixed_fp16"])
def test_virial_rows_match_oracle(precision):
    p, y, *_ = problem("virial", **VIRIAL)
    assert p.has_virials and p.n_rows == p.n_cfg + 3 * p.n_atoms + 6 * p.n_cfg
    ctx = gapgpu.Context(precision)
    ctx.assemble(gapgpu.problem_from_arrays(p, y))
    ref = oracle.design(p)
    nv = p.n_cfg + 3 * p.n_atoms
    out = torch.empty((p.n_rows, p.n_sparse), dtype=torch.float64, device="cuda")
    ctx.read_design(1 if precision != "fp64" else 0, 0, p.n_rows, out)
    got = out.cpu().numpy()
    err = rel(got[nv:], ref[nv:])
    print(precision, "virial rows %.2e" % err)
    assert err < (1e-12 if precision == "fp64" else 2e-6)
    assert rel(got[:nv], ref[:nv]) < (1e-12 if precision == "fp64" else 2e-6)


@pytest.mark.parametrize("precision,gate", [("fp64", 1e-8), ("mixed_bf16", 1e-6), ("mixed_tf32", 1e-6),
                                            ("mixed_fp16", 1e-6)])
def test_virial_fit_predictions_match_oracle(precision, gate):
    """A fit with energy, force and virial targets: its predictions of all three against
    the oracle's fit; the library's virial predictions for given weights against the
    oracle's."""
    p, y, c_or, *_ = problem("virial", **VIRIAL)
    E_or, F_or, V_or = oracle.predict_all(p, c_or)
    ctx, prob, c, info = gpu_fit(p, y, precision)
    E1, F1, V1 = oracle.predict_all(p, c.cpu().numpy())
    print(precision, "virial fit: E %.2e F %.2e V %.2e" % (rel(E1, E_or), rel(F1, F_or), rel(V1, V_or)), info["iterations"])
    assert rel(E1, E_or) < gate and rel(F1, F_or) < gate and rel(V1, V_or) < gate
    E2, F2, V2 = _virial_gpu_predict(ctx, p, c)
    assert rel(E2, E_or) < gate and rel(F2, F_or) < gate and rel(V2, V_or) < gate
    w = gapgen.normals(61, 1, p.n_sparse)
    E3, F3, V3 = oracle.predict_all(p, w)
    Eg, Fg, Vg = _virial_gpu_predict(ctx, p, torch.from_numpy(w).cuda())
    tol = 1e-12 if precision == "fp64" else 2e-6
    assert rel(Eg, E3) < tol and rel(Fg, F3) < tol and rel(Vg, V3) < tol


@pytest.mark.parametrize("precision", ["fp64", "mixed_fp16"])
def test_virial_host_problem_equals_device_problem(precision):
    """A host problem with virials (its pair displacements staged with J, which the mixed
    assembly copies in chunks) fits exactly as its device copy.  Configurations of at most
    40 atoms keep every pseudo-target's rows within two tiles (two-part sums, which do not
    depend on their order)."""
    p, y, *_ = problem("virial small", **dict(VIRIAL, atoms=(3, 40), n_cfg=30))
    _, _, c_dev, _ = gpu_fit(p, y, precision)
    _, _, c_host, _ = gpu_fit(p, y, precision, device="cpu")
    assert torch.equal(c_dev, c_host)


@pytest.mark.parametrize("key,kw", [("base", {}), ("virial", VIRIAL)])
def test_row_blocks_merged_over_contexts_match_oracle(key, kw):
    """The fit over several GPUs (Sec. III-B as a TSQR over contexts): the configurations
    placed by greedy LPT in three row blocks, each assembled and factored by its own FP64
    context (gap_tsqr_local), the blocks stacked as the exchange leaves them, merged and
    solved (gap_tsqr_merge, gap_solve): the oracle's fit of the whole problem to the FP64
    gate, with the whole fit's residual norm."""
    from paper_2207_03803_gb300.distributed import place_configurations
    p, y, c_or, E_or, F_or = problem(key, **kw)
    M = p.n_sparse
    sizes = 1 + 3 * np.diff(p.cfg_ptr)
    blocks, tails, ctxs = [], 0.0, []
    for cfgs in place_configurations(sizes, 3):
        q = gapgen.select_configurations(p, cfgs)
        ctx = gapgpu.Context("fp64")
        ctx.assemble(gapgpu.problem_from_arrays(q, y[gapgen.rows_of(p, cfgs)]))
        Rz = torch.empty((M, M + 1), dtype=torch.float64, device="cuda")
        tails += ctx.tsqr_local(Rz)
        blocks.append(Rz)
        ctxs.append(ctx)
    ctx = ctxs[0]
    ctx.tsqr_merge(torch.stack(blocks).contiguous(), tails)
    assert ctx.tsqr_blocks() == 3
    c = torch.empty(M, dtype=torch.float64, device="cuda")
    info = ctx.solve(c)
    E1, F1 = oracle.predict(p, c.cpu().numpy())
    print(key, "row blocks over contexts: E %.2e F %.2e c %.2e" % (rel(E1, E_or), rel(F1, F_or),
                                                                   rel(c.cpu().numpy(), c_or)))
    assert rel(E1, E_or) < 1e-8 and rel(F1, F_or) < 1e-8
    A, _ = oracle.stacked_matrix(p)
    bb = np.concatenate([y / oracle.sigma(p), np.zeros(M)])
    res = np.linalg.norm(bb - A @ c_or)
    assert abs(info["residual_norm"] - res) < 1e-8 * res
    for cx in ctxs:
        cx.close()

def test_invalid_inputs_and_state_errors():
    p, y, *_ = problem("base")
    ctx = gapgpu.Context("fp64")
    with pytest.raises(gapgpu.GapError) as e:
        ctx.factor()
    assert e.value.status == gapgpu.GAP_ERR_STATE
    # a pair source outside its target's configuration (device-side validation)
    bad = p.pair_src.copy()
    bad[5] = p.n_atoms - 1
    q = gapgpu.Problem(cfg_ptr=torch.from_numpy(p.cfg_ptr).cuda(), X=torch.from_numpy(p.X).cuda(),
                       Xs=torch.from_numpy(p.Xs).cuda(), y=torch.from_numpy(y).cuda(),
                       sigma=torch.from_numpy(oracle.sigma(p)).cuda(), pair_ptr=torch.from_numpy(p.pair_ptr).cuda(),
                       pair_src=torch.from_numpy(bad).cuda(), J=torch.from_numpy(p.J).cuda(), delta=1.0, zeta=4)
    with pytest.raises(gapgpu.GapError) as e:
        ctx.assemble(q)
    assert e.value.status == gapgpu.GAP_ERR_INVALID
    # sigma <= 0 (host-side validation)
    s = oracle.sigma(p)
    s[3] = 0.0
    q = gapgpu.Problem(cfg_ptr=p.cfg_ptr, X=p.X, Xs=p.Xs, y=y, sigma=s, pair_ptr=p.pair_ptr, pair_src=p.pair_src,
                       J=p.J, delta=1.0, zeta=4)
    with pytest.raises(gapgpu.GapError) as e:
        ctx.assemble(q)
    assert e.value.status == gapgpu.GAP_ERR_INVALID


def test_not_positive_definite_is_reported():
    """delta = 0 and no jitter: K_MM = 0, the first Cholesky pivot is 0."""
    p, y, *_ = problem("base")
    q = gapgpu.Problem(cfg_ptr=p.cfg_ptr, X=p.X, Xs=p.Xs, y=y, sigma=oracle.sigma(p), pair_ptr=p.pair_ptr,
                       pair_src=p.pair_src, J=p.J, delta=0.0, zeta=4, jitter=0.0)
    ctx = gapgpu.Context("fp64")
    ctx.assemble(q)
    with pytest.raises(gapgpu.GapError) as e:
        ctx.factor()
    assert e.value.status == gapgpu.GAP_ERR_NOT_SPD


def test_batched_fits_equal_single_fits():
    probs, ys, cs_single = [], [], []
    for k in range(3):
        p, y, *_ = problem("batch%d" % k, seed=100 + k, n_cfg=10 + 7 * k, M=30 + 20 * k, d=24 + k, zeta=2 + k)
        probs.append((p, y))
        cs_single.append(gpu_fit(p, y, "fp64")[2])
    ctx = gapgpu.Context("fp64")
    gprobs = [gapgpu.problem_from_arrays(p, y) for p, y in probs]
    outs = [torch.empty(p.n_sparse, dtype=torch.float64, device="cuda") for p, _ in probs]
    infos = ctx.fit_batched(gprobs, outs)
    assert len(infos) == 3
    for c1, c2 in zip(outs, cs_single):
        assert torch.equal(c1, c2)


@pytest.mark.parametrize("precision", ["fp64", "mixed_bf16"])
def test_batched_fits_in_concurrent_lanes_equal_single_fits(precision):
    """gap_fit_batched with several fits in flight (worker contexts on their own
    streams and host threads): every fit equals the same fit run alone, bit for
    bit, for one lane and for three."""
    probs, singles = [], []
    for k in range(5):
        p, y, *_ = problem("lanes%d" % k, seed=300 + k, n_cfg=6 + 9 * k, M=20 + 31 * k, d=20 + 3 * k, zeta=2 + k % 3)
        probs.append((p, y))
        singles.append(gpu_fit(p, y, precision)[2])
    for lanes in (1, 3):
        ctx = gapgpu.Context(precision)
        ctx.set_option("batch_lanes", lanes)
        gprobs = [gapgpu.problem_from_arrays(p, y) for p, y in probs]
        outs = [torch.empty(p.n_sparse, dtype=torch.float64, device="cuda") for p, _ in probs]
        infos = ctx.fit_batched(gprobs, outs)
        for k in range(5):
            assert torch.equal(outs[k], singles[k]), (lanes, k)
            assert infos[k]["converged"]
        ctx.close()


def test_workload4_sweep_fits_in_one_batched_call():
    """Workload 4 (a hyperparameter sweep of independent fits of uneven shape): the
    smallest fits of the seeded 64-fit sweep (d = 256; zeta, sigma_E and M varying
    per fit) through one gap_fit_batched call in the mixed precision; each fit's
    predictions against the oracle's at the mixed gate."""
    recs = gapgen.sweep_recipes()
    small = sorted(range(len(recs)), key=lambda f: recs[f].n_cfg * recs[f].n_sparse[0])[:4]
    probs, refs = [], []
    for f in small:
        p, y, c_or, E_or, F_or = problem("sweep%d" % f, seed=recs[f].seed, n_cfg=recs[f].n_cfg, atoms=recs[f].atoms,
                                         d=recs[f].d, M=recs[f].n_sparse[0], zeta=recs[f].zeta,
                                         nb=recs[f].neighbours, sigma_e=recs[f].sigma_e_atom)
        probs.append((p, y))
        refs.append((E_or, F_or))
    ctx = gapgpu.Context("mixed_bf16")
    gprobs = [gapgpu.problem_from_arrays(p, y) for p, y in probs]
    outs = [torch.empty(p.n_sparse, dtype=torch.float64, device="cuda") for p, _ in probs]
    infos = ctx.fit_batched(gprobs, outs)
    for k, (p, y) in enumerate(probs):
        assert infos[k]["converged"], k
        E1, F1 = oracle.predict(p, outs[k].cpu().numpy())
        print("sweep fit", small[k], p.n_rows, p.n_sparse, "E %.2e F %.2e" % (rel(E1, refs[k][0]), rel(F1, refs[k][1])))
        assert rel(E1, refs[k][0]) < 1e-6 and rel(F1, refs[k][1]) < 1e-6, k
    ctx.close()


_fit16 = {}


@pytest.mark.parametrize("precision", ["mixed_bf16", "mixed_tf32", "mixed_fp16"])
def test_sweep_fit_16_small_energy_sigma(precision):
    """Sweep fit 16 (zeta = 2, sigma_E = 1e-4 per atom, M = 529, 23,322 data rows,
    condition number about 6e4) with its stored targets: the energy rows weigh so much
    that their FP32 rounding alone moves the fitted forces by about 8e-7; they reach
    the residual matrix in FP64 (double-float epilogue), which keeps this fit under
    the mixed gate."""
    f = 16
    r = gapgen.sweep_recipes()[f]
    if not _fit16:
        p = gapgen.make_problem(r)
        y = gapgen.load_sweep_targets(p, f)
        c, _ = oracle.fit(p, y)
        _fit16.update(p=p, y=y, EF=oracle.predict(p, c))
    p, y, (E_or, F_or) = _fit16["p"], _fit16["y"], _fit16["EF"]
    ctx, prob, c, info = gpu_fit(p, y, precision)
    E1, F1 = oracle.predict(p, c.cpu().numpy())
    print("sweep fit 16", precision, "E %.2e F %.2e" % (rel(E1, E_or), rel(F1, F_or)), info["iterations"])
    assert info["converged"]
    assert rel(E1, E_or) < 1e-6 and rel(F1, F_or) < 1e-6


def test_autotuner_picks_a_converging_schedule_and_caches_it(tmp_path):
    """The schedule autotuner times its candidates on the problem itself, keeps a
    converging one, and a second context of the same shape class reads the choice
    from the JSON cache; the batched tuner does the same for the fits in flight."""
    from paper_2207_03803_gb300 import autotune
    p, y, c_or, E_or, F_or = problem("base")
    prob = gapgpu.problem_from_arrays(p, y, device="cuda")
    path = str(tmp_path / "tune.json")
    c = torch.empty(p.n_sparse, dtype=torch.float64, device="cuda")
    ctx = gapgpu.Context("mixed_bf16")
    best = autotune.tune_fit(ctx, prob, c, autotune.TuneCache(path))
    assert best in [dict(x) for x in autotune.FIT_CANDIDATES]
    ctx.assemble(prob)
    ctx.factor()
    assert ctx.solve(c)["converged"]
    E, F = gpu_predict(ctx, p, c)
    assert rel(E, E_or) < 1e-6 and rel(F, F_or) < 1e-6
    cache = autotune.TuneCache(path)
    assert len(cache.entries) == 1
    ctx2 = gapgpu.Context("mixed_bf16")
    assert autotune.tune_fit(ctx2, prob, c, cache) == best
    recs = gapgen.sweep_recipes()
    small = sorted(range(len(recs)), key=lambda f: recs[f].n_cfg * recs[f].n_sparse[0])[:3]
    gprobs, outs = [], []
    for f in small:
        q = gapgen.make_problem(recs[f])
        gprobs.append(gapgpu.problem_from_arrays(q, oracle.targets(q)))
        outs.append(torch.empty(q.n_sparse, dtype=torch.float64, device="cuda"))
    lanes = autotune.tune_batched(ctx2, gprobs, outs, cache)
    assert lanes in [dict(x) for x in autotune.BATCH_CANDIDATES]
    assert all(i["converged"] for i in ctx2.fit_batched(gprobs, outs))
    assert len(autotune.TuneCache(path).entries) == 2
    ctx.close()
    ctx2.close()


def test_batched_fit_reports_the_failing_fit():
    probs = []
    for k in range(4):
        p, y, *_ = problem("bfail%d" % k, seed=400 + k, n_cfg=8 + 3 * k, M=25, d=16)
        probs.append((p, y))
    import copy
    bad = copy.copy(probs[2][0])
    bad.sigma_e = bad.sigma_e.copy()
    bad.sigma_e[0] = -1.0  # an invalid noise level in fit 2 only
    probs[2] = (bad, probs[2][1])
    gprobs = [gapgpu.problem_from_arrays(p, y) for p, y in probs]
    ctx = gapgpu.Context("mixed_bf16")
    ctx.set_option("batch_lanes", 2)
    outs = [torch.empty(p.n_sparse, dtype=torch.float64, device="cuda") for p, _ in probs]
    with pytest.raises(gapgpu.GapError) as ei:
        ctx.fit_batched(gprobs, outs)
    assert "fit 2" in str(ei.value)


def test_two_level_qr_matches_flat_qr():
    """FP32 QR with outer panels of 128 applied on the tensor cores against the
    flat FP32 blocked QR: with split-TF32 operands (3 passes) and two CholeskyQR
    passes per panel the same R up to row signs and FP32 rounding; with plain TF32
    (1 pass) and one or two CholeskyQR passes the same R to TF32 accuracy, and the
    refined fit still meets the 1e-6 gate.  M = 300 spans three outer panels with
    a ragged last one."""
    p, y, c_ref, E_ref, F_ref = problem("qr2", n_cfg=60, atoms=(3, 60), M=300, d=40, zeta=3)
    Rs = {}
    for two, passes, cqr in ((0, 3, 2), (1, 3, 2), (1, 1, 2), (1, 1, 1)):
        ctx, _, c, info = gpu_fit(p, y, "mixed_tf32", qr_two_level=two, qr_passes=passes, cqr_passes=cqr)
        R = torch.empty((p.n_sparse, p.n_sparse), dtype=torch.float64, device="cuda")
        ctx.read_r(R)
        Rs[(two, passes, cqr)] = np.abs(R.cpu().numpy())
        assert info["converged"]
        E, F = gpu_predict(ctx, p, c)
        assert rel(E, E_ref) < 1e-6 and rel(F, F_ref) < 1e-6, (two, passes, cqr)
    assert rel(Rs[(1, 3, 2)], Rs[(0, 3, 2)]) < 1e-5
    assert rel(Rs[(1, 1, 2)], Rs[(0, 3, 2)]) < 5e-3
    assert rel(Rs[(1, 1, 1)], Rs[(0, 3, 2)]) < 5e-3


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-15), ("mixed_bf16", 5e-7)])
def test_cholesky_square_roots(precision, tol):
    """The square roots of the Cholesky pivots (the FP64 factor's Newton-refined reciprocal
    square root, the double-float factor's pair version) against numpy's sqrt.  Orthonormal
    sparse points make K_MM = (delta^2 + jitter) I, so U = sqrt(delta^2 + jitter) I.  FP64:
    atom descriptors orthogonal to the sparse points make K_NM zero, so R of the QR of [0; U]
    has |R_ii| = U_ii, to a couple of rounding errors.  Mixed precisions: U's rows as stacked
    into the FP32-accurate matrix, to their FP32 rounding (their R comes from an FP32 QR with
    one-pass TF32 updates, and their centred energy products leave K_NM at about 1e-7 of
    delta^2 instead of zero, so R does not isolate the factor)."""
    M, n = 40, 50
    d = M + n
    for delta in (1e-3, 0.37, 1.0, 5.9, 1234.5):
        for jitter in (1e-8, 1e-3, 2.5):
            X = np.zeros((n, d))
            X[np.arange(n), M + np.arange(n)] = 1.0
            Xs = np.zeros((M, d))
            Xs[np.arange(M), np.arange(M)] = 1.0
            prob = gapgpu.Problem(cfg_ptr=np.arange(n + 1, dtype=np.int64), X=X, Xs=Xs, delta=delta, zeta=1,
                                  jitter=jitter, y=np.zeros(n), sigma=np.ones(n), memory=gapgpu.GAP_MEM_HOST)
            ctx = gapgpu.Context(precision)
            ctx.assemble(prob)
            ctx.factor()
            R = torch.empty((M, M), dtype=torch.float64, device="cuda")
            if precision == "fp64":
                ctx.read_r(R)
            else:
                ctx.read_design(1, n, M, R)  # the rows of U below the data rows
            diag = np.abs(np.diag(R.cpu().numpy()))
            ref = np.sqrt(delta * delta + jitter)
            err = np.max(np.abs(diag - ref)) / ref
            assert err < tol, (precision, delta, jitter, err)
            ctx.close()

