"""Workload 2 at full size (2000 configurations, 441,968 design rows, M = 4000, d = 512),
through the calls the benchmark times, checked on what the oracle can compute at this
size:
- sampled rows: the first 8 configurations' energy rows, and their atoms' force rows, of
  the assembled matrices against the oracle's rows for those configurations (a row depends
  only on its configuration and the sparse set, and ``make_problem(max_cfg=8)`` draws
  exactly the full problem's values);
- sampled predictions: the library's energies and forces of those configurations against
  the oracle's predictions with the same weights, to 1e-6.  The forces' gradient product
  contracts over all M = 4000 sparse points; it runs in K-chunks of at most 32 MMA steps,
  without which the truncating FP32 accumulation left a bias of 4.75e-6;
- a property of the fit that holds at any size: the targets carry noise of the stated
  sigmas, so the squared weighted residual of the fit is close to N - M (N data rows);
- the mixed fit against the plain FP64 GPU fit, which is held to the oracle at 1e-8 at
  the sizes the oracle fits: the oracle's predictions of the sampled configurations with
  either fit's weights agree to the mixed gate, 1e-6.
"""
import numpy as np
import pytest

import gapgen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2207_03803_gb300 as gapgpu  # noqa: E402

K = 8  # sampled configurations
_mixed = {}


def rel(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def full():
    gapgpu.build()
    gapgpu.load()
    r = gapgen.RECIPES[2]
    p = gapgen.make_problem(r)
    y = gapgen.load_targets(p, 2)
    sub = gapgen.make_problem(r, max_cfg=K)
    prob = gapgpu.problem_from_arrays(p, y, device="cuda")
    return p, y, sub, oracle.design(sub), prob


def _sampled_rows(ctx, p, sub, which):
    """Rows of the sampled configurations: energy rows [0, K) and their force rows."""
    M = p.n_sparse
    nf = 3 * sub.n_atoms
    e = torch.empty((K, M), dtype=torch.float64, device="cuda")
    f = torch.empty((nf, M), dtype=torch.float64, device="cuda")
    ctx.read_design(which, 0, K, e)
    ctx.read_design(which, p.n_cfg, nf, f)
    return e.cpu().numpy(), f.cpu().numpy()


def _predict(ctx, p, c):
    E = torch.empty(p.n_cfg, dtype=torch.float64, device="cuda")
    F = torch.empty(3 * p.n_atoms, dtype=torch.float64, device="cuda")
    ctx.predict(None, c, E, F)
    return E.cpu().numpy(), F.cpu().numpy()


def test_workload2_mixed_bf16_full_size(full):
    p, y, sub, D_sub, prob = full
    ctx = gapgpu.Context("mixed_bf16")
    ctx.assemble(prob)
    nf = 3 * sub.n_atoms
    # the QR matrix (single-pass BF16 products) and the residual matrix (split products,
    # energy rows in FP64)
    e0, f0 = _sampled_rows(ctx, p, sub, 0)
    assert rel(e0, D_sub[:K]) < 3e-2 and rel(f0, D_sub[K:K + nf]) < 3e-2
    e1, f1 = _sampled_rows(ctx, p, sub, 1)
    print("workload 2 sampled rows: energy %.2e force %.2e" % (rel(e1, D_sub[:K]), rel(f1, D_sub[K:K + nf])))
    assert rel(e1, D_sub[:K]) < 3e-7 and rel(f1, D_sub[K:K + nf]) < 2e-6
    ctx.factor()
    c = torch.empty(p.n_sparse, dtype=torch.float64, device="cuda")
    info = ctx.solve(c)
    assert info["converged"]
    chi2 = info["residual_norm"] ** 2 / (p.n_rows - p.n_sparse)
    E, F = _predict(ctx, p, c)
    c_np = c.cpu().numpy()
    E_or, F_or = oracle.predict(sub, c_np)
    print("workload 2: %d iterations, residual^2 / (N - M) = %.4f, sampled predictions E %.2e F %.2e"
          % (info["iterations"], chi2, rel(E[:K], E_or), rel(F[:nf], F_or)))
    assert 0.9 < chi2 < 1.1
    assert rel(E[:K], E_or) < 1e-6 and rel(F[:nf], F_or) < 1e-6
    _mixed.update(c=c_np, E=E, F=F, res=info["residual_norm"])
    ctx.close()


def test_workload2_fp64_full_size_agrees(full):
    p, y, sub, D_sub, prob = full
    ctx = gapgpu.Context("fp64")
    ctx.assemble(prob)
    nf = 3 * sub.n_atoms
    e, f = _sampled_rows(ctx, p, sub, 1)
    assert rel(e, D_sub[:K]) < 1e-12 and rel(f, D_sub[K:K + nf]) < 1e-12
    ctx.factor()
    c = torch.empty(p.n_sparse, dtype=torch.float64, device="cuda")
    info = ctx.solve(c)
    E, F = _predict(ctx, p, c)
    E_or, F_or = oracle.predict(sub, c.cpu().numpy())
    assert rel(E[:K], E_or) < 1e-10 and rel(F[:nf], F_or) < 1e-10
    assert 0.9 < info["residual_norm"] ** 2 / (p.n_rows - p.n_sparse) < 1.1
    if _mixed:
        # the two fits compared through the oracle's predictions with their weights
        Em, Fm = oracle.predict(sub, _mixed["c"])
        print("workload 2, mixed_bf16 fit against the fp64 fit (sampled, oracle predictions): E %.2e F %.2e, "
              "residual %.2e" % (rel(Em, E_or), rel(Fm, F_or),
                                 abs(_mixed["res"] - info["residual_norm"]) / info["residual_norm"]))
        assert rel(Em, E_or) < 1e-6 and rel(Fm, F_or) < 1e-6
    ctx.close()
