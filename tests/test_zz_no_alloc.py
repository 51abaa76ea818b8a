"""gap_predict_static, the allocation-free prediction entry point, against the
context-based gap_predict.

Callers such as a molecular-dynamics step loop whose allocator owns all GPU
memory cannot call cudaMalloc; gap_predict_static serves them with scratch in
a fixed device array compiled into the library.  This file is collected last
so that a run stopping at its first failure has run every other test.
"""
import ctypes

import numpy as np
import pytest

import gapgen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2207_03803_gb300 as gapgpu  # noqa: E402


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def _problem():
    r = gapgen.Recipe(n_cfg=29, atoms=(3, 90), d=45, n_sparse=(70,), zeta=3, neighbours=(0, 18), seed=77)
    p = gapgen.make_problem(r)
    return p, gapgpu.problem_from_arrays(p, np.zeros(p.n_rows), device="cuda")


def test_static_predictions_equal_gap_predict_on_two_calls():
    gapgpu.build()
    p, prob = _problem()
    ctx = gapgpu.Context("fp64")
    ctx.assemble(prob)  # the sparse set gap_predict uses
    for k in range(2):  # two calls in a row share (and reuse) the static scratch
        c = torch.from_numpy(gapgen.normals(300 + k, 1, p.n_sparse)).cuda()
        E1 = torch.empty(p.n_cfg, dtype=torch.float64, device="cuda")
        F1 = torch.empty(3 * p.n_atoms, dtype=torch.float64, device="cuda")
        ctx.predict(prob, c, E1, F1)
        E2 = torch.full_like(E1, float("nan"))
        F2 = torch.full_like(F1, float("nan"))
        gapgpu.predict_static(prob, c, E2, F2)
        torch.cuda.synchronize()
        assert rel(E2.cpu().numpy(), E1.cpu().numpy()) < 1e-12
        assert rel(F2.cpu().numpy(), F1.cpu().numpy()) < 1e-12
        # and both against the oracle, the same tolerance as the other prediction tests
        E_or, F_or = oracle.predict(p, c.cpu().numpy())
        assert rel(E2.cpu().numpy(), E_or) < 1e-12 and rel(F2.cpu().numpy(), F_or) < 1e-12
    ctx.close()


def test_static_prediction_rejects_targets_beyond_its_scratch():
    gapgpu.build()
    lib = gapgpu.load()
    st = gapgpu.gap_problem()
    st.n_cfg, st.n_atoms, st.d, st.n_pairs, st.n_sparse = 1, 200000, 512, 10, 4000
    st.zeta, st.delta, st.memory = 2, 1.0, gapgpu.GAP_MEM_DEVICE
    st.cfg_ptr = st.X = st.Xs = st.pair_ptr = st.pair_src = st.J = 8  # never dereferenced
    err = ctypes.create_string_buffer(256)
    rc = lib.gap_predict_static(ctypes.byref(st), 8, 8, 8, None, err, len(err))
    assert rc == gapgpu.GAP_ERR_INVALID
    assert b"bytes of scratch" in err.value
