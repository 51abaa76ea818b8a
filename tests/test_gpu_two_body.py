"""The two-body sub-GAP (appendix: distance_2b with ard_se) on the GPU against the oracle
(oracle/two_body.py, composed with the SOAP block in oracle/__init__.py): the design rows
of both column blocks, the fits' predictions, predictions for given weights (energies,
forces, virials), host-memory problems, and a species problem, in every precision.

With the appendix's 20 sparse distances over the 4.5 A cutoff and theta = 0.75 A, the
two-body columns are so nearly dependent that the stacked matrix of these problems has a
condition number of about 2.6e9: beyond what the mixed precisions' FP32 matrices carry.  The
FP64 fits use that setting; the mixed fits use 8 sparse distances (condition about 2.4e3),
and the mixed precisions are checked to report the ill-conditioned fit as not converged."""
import numpy as np
import pytest

import gapgen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2207_03803_gb300 as gapgpu  # noqa: E402

PRECISIONS = ["fp64", "mixed_bf16", "mixed_tf32", "mixed_fp16"]


@pytest.fixture(scope="module", autouse=True)
def built():
    gapgpu.build()
    gapgpu.load()


def rel(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


_cache = {}


def problem(key, n2=20):
    if (key, n2) not in _cache:
        kw = dict(n_cfg=23, atoms=(2, 60), d=37, n_sparse=(90,), zeta=4, neighbours=(0, 14), two_body=True,
                  seed=71, n_sparse_2b=n2)
        if key == "virial":
            kw.update(virials=True, seed=72)
        if key == "species":
            kw.update(n_species=3, n_sparse=(30, 31, 29), seed=73)
        p = gapgen.make_problem(gapgen.Recipe(**kw))
        y = oracle.targets(p)
        c, _ = oracle.fit(p, y)
        _cache[(key, n2)] = (p, y, c)
    return _cache[(key, n2)]


def predict_gpu(ctx, p, c, device="cuda"):
    tgt = gapgpu.problem_from_arrays(p, np.zeros(p.n_rows), device=device)
    E = torch.empty(p.n_cfg, dtype=torch.float64, device="cuda")
    F = torch.empty(3 * p.n_atoms, dtype=torch.float64, device="cuda")
    if p.has_virials:
        V = torch.empty(6 * p.n_cfg, dtype=torch.float64, device="cuda")
        ctx.predict_virial(tgt, c, E, F, V)
        return E.cpu().numpy(), F.cpu().numpy(), V.cpu().numpy()
    ctx.predict(tgt, c, E, F)
    return E.cpu().numpy(), F.cpu().numpy(), None


@pytest.mark.parametrize("key", ["base", "virial", "species"])
@pytest.mark.parametrize("precision", PRECISIONS)
def test_design_rows_of_both_blocks_match_oracle(precision, key):
    p, y, _ = problem(key)
    ctx = gapgpu.Context(precision)
    ctx.assemble(gapgpu.problem_from_arrays(p, y))
    ref = oracle.design(p)
    assert ref.shape == (p.n_rows, p.n_weights)
    out = torch.empty((p.n_rows, p.n_weights), dtype=torch.float64, device="cuda")
    ctx.read_design(1 if precision != "fp64" else 0, 0, p.n_rows, out)
    got = out.cpu().numpy()
    Ms = p.n_sparse
    e2 = rel(got[:, Ms:], ref[:, Ms:])
    e1 = rel(got[:, :Ms], ref[:, :Ms])
    print(precision, key, "SOAP block %.2e two-body block %.2e" % (e1, e2))
    tol = 1e-12 if precision == "fp64" else 2e-6
    assert e1 < tol
    assert e2 < (1e-12 if precision == "fp64" else 1e-7)  # FP64 rows stored in FP32 (mixed)
    ctx.close()


@pytest.mark.parametrize("key", ["base", "virial", "species"])
@pytest.mark.parametrize("precision,gate", [("fp64", 1e-8), ("mixed_bf16", 1e-6), ("mixed_tf32", 1e-6),
                                            ("mixed_fp16", 1e-6)])
def test_fit_predictions_match_oracle(precision, gate, key):
    p, y, c_or = problem(key, 20 if precision == "fp64" else 8)
    E_or, F_or, V_or = oracle.predict_all(p, c_or)
    ctx = gapgpu.Context(precision)
    ctx.assemble(gapgpu.problem_from_arrays(p, y))
    ctx.factor()
    c = torch.empty(p.n_weights, dtype=torch.float64, device="cuda")
    info = ctx.solve(c)
    E1, F1, V1 = oracle.predict_all(p, c.cpu().numpy())
    errs = [rel(E1, E_or), rel(F1, F_or)] + ([rel(V1, V_or)] if V_or is not None else [])
    print(precision, key, "fit", ["%.2e" % e for e in errs], info["iterations"])
    assert max(errs) < gate
    # the library's own predictions of its fit, with the two-body model added
    E2, F2, V2 = predict_gpu(ctx, p, c)
    assert rel(E2, E_or) < gate and rel(F2, F_or) < gate
    if V_or is not None:
        assert rel(V2, V_or) < gate
    ctx.close()


@pytest.mark.parametrize("precision", PRECISIONS)
def test_predictions_for_given_weights(precision):
    """Both blocks' predictions for weights the oracle also uses; the two-body part alone
    (SOAP weights zero), to FP64 rounding in every precision (its kernels are FP64)."""
    p, y, _ = problem("virial")
    ctx = gapgpu.Context(precision)
    ctx.assemble(gapgpu.problem_from_arrays(p, y))
    w = gapgen.normals(81, 1, p.n_weights)
    E, F, V = oracle.predict_all(p, w)
    Eg, Fg, Vg = predict_gpu(ctx, p, torch.from_numpy(w).cuda())
    tol = 1e-12 if precision == "fp64" else 2e-6
    assert rel(Eg, E) < tol and rel(Fg, F) < tol and rel(Vg, V) < tol
    w2 = w.copy()
    w2[:p.n_sparse] = 0.0
    E, F, V = oracle.predict_all(p, w2)
    Eg, Fg, Vg = predict_gpu(ctx, p, torch.from_numpy(w2).cuda())
    assert rel(Eg, E) < 1e-12 and rel(Fg, F) < 1e-12 and rel(Vg, V) < 1e-12
    ctx.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed_bf16"])
def test_host_problem_equals_device_problem(precision):
    p, y, _ = problem("base", 8)
    out = []
    for device in ("cuda", "cpu"):
        ctx = gapgpu.Context(precision)
        ctx.assemble(gapgpu.problem_from_arrays(p, y, device=device))
        ctx.factor()
        c = torch.empty(p.n_weights, dtype=torch.float64, device="cuda")
        ctx.solve(c)
        out.append((c.cpu().numpy(), predict_gpu(ctx, p, c, device=device)))
        ctx.close()
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1][0], out[1][1][0]) and np.array_equal(out[0][1][1], out[1][1][1])


@pytest.mark.parametrize("precision", ["mixed_bf16", "mixed_fp16"])
def test_ill_conditioned_mixed_fit_reports_not_converged(precision):
    p, y, _ = problem("base", 20)
    ctx = gapgpu.Context(precision)
    ctx.assemble(gapgpu.problem_from_arrays(p, y))
    ctx.factor()
    c = torch.empty(p.n_weights, dtype=torch.float64, device="cuda")
    with pytest.raises(gapgpu.GapError) as e:
        ctx.solve(c)
    assert e.value.status == gapgpu.GAP_ERR_NOT_CONVERGED
    ctx.close()


def test_invalid_two_body_inputs_are_rejected():
    p, y, _ = problem("base")
    tb = p.two_body
    bad = tb.bond_ptr.copy()
    bad[5], bad[6] = bad[6], bad[5] - 1  # not monotone
    prob = gapgpu.problem_from_arrays(p, y, device="cpu")
    prob._keep[11][:] = bad
    ctx = gapgpu.Context("fp64")
    with pytest.raises(gapgpu.GapError) as e:
        ctx.assemble(prob)
    assert e.value.status == gapgpu.GAP_ERR_INVALID
    prob = gapgpu.problem_from_arrays(p, y, device="cuda")
    prob._keep[12][3] = -1.0  # a bond length <= 0, checked on the device
    with pytest.raises(gapgpu.GapError) as e:
        ctx.assemble(prob)
    assert e.value.status == gapgpu.GAP_ERR_INVALID
    ctx.close()
