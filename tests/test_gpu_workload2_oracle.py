"""Workload 2 at full size (2000 configurations, 441,968 design rows, M = 4000, d = 512)
against the FP64 oracle's own fit of the whole problem.

``tests/golden/make_workload2_fit.py`` fits the full problem once with the oracle (plain
FP64 loops: assembly of Eq. 7, Cholesky, Householder QR, back substitution of Eq. 12)
and stores its weights and its predictions for every configuration and atom.  Here the
library fits the same inputs in every precision, through the calls the benchmark times,
and all 2000 energies and 439,968 force components of its fitted model (its own
prediction kernels, for the problem it assembled) are compared with the oracle's: the
gates are 1e-8 (FP64) and 1e-6 (mixed precisions after FP64 refinement), relative L2.
The error of c is reported, not gated (an ill-conditioned fit's weights agree to fewer
digits than its predictions, Sec. IV).
"""
import json
import os

import numpy as np
import pytest

import gapgen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2207_03803_gb300 as gapgpu  # noqa: E402

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "workload2_oracle_fit.npz")


def rel(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def full():
    if not os.path.exists(GOLDEN):
        pytest.skip("the oracle's full workload-2 fit has not been recorded")
    gapgpu.build()
    gapgpu.load()
    z = np.load(GOLDEN)
    p = gapgen.make_problem(gapgen.RECIPES[2])
    assert str(z["fingerprint"]) == gapgen.fingerprint(p), "the stored oracle fit belongs to other inputs"
    y = gapgen.load_targets(p, 2)
    prob = gapgpu.problem_from_arrays(p, y, device="cuda")
    return p, prob, z


@pytest.mark.parametrize("precision,gate", [("mixed_bf16", 1e-6), ("mixed_fp16", 1e-6), ("mixed_tf32", 1e-6),
                                            ("fp64", 1e-8)])
def test_workload2_full_fit_matches_oracle_fit(full, precision, gate):
    p, prob, z = full
    ctx = gapgpu.Context(precision)
    ctx.assemble(prob)
    ctx.factor()
    c = torch.empty(p.n_sparse, dtype=torch.float64, device="cuda")
    info = ctx.solve(c)
    E = torch.empty(p.n_cfg, dtype=torch.float64, device="cuda")
    F = torch.empty(3 * p.n_atoms, dtype=torch.float64, device="cuda")
    ctx.predict(None, c, E, F)
    eE, eF = rel(E.cpu().numpy(), z["E"]), rel(F.cpu().numpy(), z["F"])
    ec = rel(c.cpu().numpy(), z["c"])
    print("workload 2 full, %s against the oracle's fit: E %.2e F %.2e (c %.2e), %d refinement iterations"
          % (precision, eE, eF, ec, info["iterations"]))
    assert eE < gate and eF < gate
    if precision != "fp64":
        assert info["converged"]
    ctx.close()


def test_workload2_oracle_record_is_complete(full):
    """The record holds the whole fit: weights, every prediction, the phase times and the
    machine it ran on."""
    p, _, z = full
    assert z["c"].shape == (p.n_sparse,) and z["E"].shape == (p.n_cfg,) and z["F"].shape == (3 * p.n_atoms,)
    assert np.isfinite(z["c"]).all() and np.isfinite(z["F"]).all()
    host = json.loads(str(z["host"]))
    assert host["cores"] >= 1 and host["fit_s"] > 0 and len(z["times"]) == 5
