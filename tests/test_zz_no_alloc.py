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


CASES = {
    # forces of one species
    "forces": dict(n_cfg=29, atoms=(3, 90), d=45, n_sparse=(70,), zeta=3, neighbours=(0, 18), seed=77),
    # energies only: no pair data at all
    "energies only": dict(n_cfg=31, atoms=(2, 60), d=33, n_sparse=(50,), zeta=2, neighbours=None, seed=78),
    # three species (the kernel vanishes across species), with forces
    "species": dict(n_cfg=24, atoms=(6, 70), d=29, n_sparse=(30, 25, 20), zeta=4, neighbours=(1, 12),
                    n_species=3, seed=79),
}


def _problem(case):
    p = gapgen.make_problem(gapgen.Recipe(**CASES[case]))
    return p, gapgpu.problem_from_arrays(p, np.zeros(p.n_rows), device="cuda")


@pytest.mark.parametrize("case", sorted(CASES))
def test_static_predictions_equal_gap_predict_on_two_calls(case):
    gapgpu.build()
    p, prob = _problem(case)
    ctx = gapgpu.Context("fp64")
    ctx.assemble(prob)  # the sparse set gap_predict uses
    nF = 3 * p.n_atoms
    for k in range(2):  # two calls in a row share (and reuse) the static scratch
        c = torch.from_numpy(gapgen.normals(300 + k, 1, p.n_sparse)).cuda()
        E1 = torch.empty(p.n_cfg, dtype=torch.float64, device="cuda")
        F1 = torch.empty(nF, dtype=torch.float64, device="cuda") if p.has_forces else None
        ctx.predict(prob, c, E1, F1)
        E2 = torch.full_like(E1, float("nan"))
        F2 = torch.full((nF,), float("nan"), dtype=torch.float64, device="cuda")
        gapgpu.predict_static(prob, c, E2, F2 if p.has_forces else None)
        torch.cuda.synchronize()
        assert rel(E2.cpu().numpy(), E1.cpu().numpy()) < 1e-12
        # and against the oracle, the same tolerance as the other FP64 prediction tests
        E_or, F_or = oracle.predict(p, c.cpu().numpy())
        assert rel(E2.cpu().numpy(), E_or) < 1e-12
        if p.has_forces:
            assert rel(F2.cpu().numpy(), F1.cpu().numpy()) < 1e-12
            assert rel(F2.cpu().numpy(), F_or) < 1e-12
    ctx.close()


def test_static_forces_of_targets_without_pairs_are_zero():
    """Targets given no pair data (n_pairs = 0) with a force buffer: the forces are
    written as zeros, over whatever the buffer held."""
    gapgpu.build()
    p, prob = _problem("energies only")
    c = torch.from_numpy(gapgen.normals(5, 1, p.n_sparse)).cuda()
    E = torch.full((p.n_cfg,), float("nan"), dtype=torch.float64, device="cuda")
    F = torch.full((3 * p.n_atoms,), float("nan"), dtype=torch.float64, device="cuda")
    gapgpu.predict_static(prob, c, E, F)
    torch.cuda.synchronize()
    assert torch.count_nonzero(F).item() == 0
    E_or, _ = oracle.predict(p, c.cpu().numpy())
    assert rel(E.cpu().numpy(), E_or) < 1e-12


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
    # a descriptor length whose byte count would wrap a 64-bit size is rejected as well
    st.n_atoms, st.d = 1000, (1 << 62)
    rc = lib.gap_predict_static(ctypes.byref(st), 8, 8, 8, None, err, len(err))
    assert rc == gapgpu.GAP_ERR_INVALID
    assert b"bytes of scratch" in err.value
