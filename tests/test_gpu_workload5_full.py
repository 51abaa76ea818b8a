"""Workload 5 at full size (6000 configurations in three species, 335,097 atoms, 5,365,085
pairs, d = 1024, M = 16,000; 1,011,291 data rows), through the calls and the launch
configuration the benchmark times: a host problem whose 132 GB of FP64 Jacobians reach the
force pass through a J ring of 524,288 rows.  It is checked on what the oracle can compute
at this size:
- sampled rows: every column of the design rows of four configurations against the
  oracle's rows of those configurations, computed here.  They are the first and the last
  configurations, one in the middle, and the one whose pairs cross the first chunk
  boundary of the ring.  A configuration's rows depend only on its own atoms and the
  sparse set; ``gapgen.make_part`` draws exactly the full problem's values.
- sampled predictions: the fitted model's energies and forces of those configurations
  (gap_predict of the fitted problem: its design rows times c) against the oracle's
  predictions with the same weights;
- the same weights through the plain FP64 GPU prediction path (the SIMT kernels of the
  FP64 precision, Eqs. 1, 2) on those configurations;
- a property of the fit that holds at any size: the targets carry noise of the stated
  sigmas, so the squared weighted residual is close to N - M.

The test needs about 140 GB of host memory and is skipped on a host with less."""
import numpy as np
import pytest

import gapgen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2207_03803_gb300 as gapgpu  # noqa: E402

RING = 128 * 4096


def rel(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def mem_available():
    for ln in open("/proc/meminfo"):
        if ln.startswith("MemAvailable:"):
            return int(ln.split()[1]) * 1024
    return 0


def sampled_configurations(r):
    cfg_ptr, pair_ptr = gapgen.structure(r)
    a = int(np.searchsorted(pair_ptr, RING // 128 * 42, side="right")) - 1
    A = int(np.searchsorted(cfg_ptr, a, side="right")) - 1
    return sorted({0, A, r.n_cfg // 2, r.n_cfg - 1})


def test_workload5_mixed_bf16_full_size():
    r = gapgen.RECIPES[5]
    n_atoms, n_pairs = gapgen.count_shape(r)
    if mem_available() < (n_pairs * 3 + n_atoms) * r.d * 8 + 16e9:
        pytest.skip("workload 5 needs about 150 GB of host memory")
    gapgpu.build()
    gapgpu.load()
    cfgs = sampled_configurations(r)
    parts = [gapgen.make_part(r, A, A + 1) for A in cfgs]
    p = gapgen.make_problem(r)
    y = gapgen.load_targets(p, 5)
    N, M = p.n_rows, p.n_sparse
    prob = gapgpu.problem_from_arrays(p, y, device="cpu")
    ctx = gapgpu.Context("mixed_bf16")
    ctx.set_option("j_ring_rows", RING)
    ctx.assemble(prob)
    ctx.factor()
    c = torch.empty(M, dtype=torch.float64, device="cuda")
    info = ctx.solve(c)
    assert info["converged"]
    E = torch.empty(p.n_cfg, dtype=torch.float64, device="cuda")
    F = torch.empty(3 * p.n_atoms, dtype=torch.float64, device="cuda")
    ctx.predict(None, c, E, F)
    E, F, cw = E.cpu().numpy(), F.cpu().numpy(), c.cpu().numpy()
    # the fit: weighted residual close to N - M
    res = (y - np.concatenate([E, F])) / np.concatenate([p.sigma_e, p.sigma_f])
    chi2 = float(res @ res) / (N - M)
    print("workload 5: %d iterations, chi2/dof %.4f" % (info["iterations"], chi2))
    assert 0.95 < chi2 < 1.05
    # sampled rows and predictions against the oracle's
    for A, q in zip(cfgs, parts):
        a0, a1 = int(p.cfg_ptr[A]), int(p.cfg_ptr[A + 1])
        ref = oracle.design(q)
        o = torch.empty((1 + 3 * (a1 - a0), M), dtype=torch.float64, device="cuda")
        ctx.read_design(1, A, 1, o[:1])
        ctx.read_design(1, p.n_cfg + 3 * a0, 3 * (a1 - a0), o[1:])
        got = o.cpu().numpy()
        scale = np.abs(ref).max(axis=1, keepdims=True) + 1e-300
        Eo, Fo = oracle.predict(q, cw)
        print("configuration %d (%d atoms): rows energy %.2e force %.2e (max %.2e); predictions E %.2e F %.2e"
              % (A, a1 - a0, rel(got[:1], ref[:1]), rel(got[1:], ref[1:]), np.max(np.abs(got - ref) / scale),
                 rel(E[A:A + 1], Eo), rel(F[3 * a0:3 * a1], Fo)))
        assert rel(got[:1], ref[:1]) < 2e-7 and rel(got[1:], ref[1:]) < 2e-6
        assert np.max(np.abs(got - ref) / scale) < 1e-5
        assert rel(E[A:A + 1], Eo) < 1e-6 and rel(F[3 * a0:3 * a1], Fo) < 1e-6
    ctx.close()
    # the same weights through the FP64 GPU prediction path, on the sampled configurations
    sub = gapgen.select_configurations(p, np.array(cfgs))
    del p, prob
    ctx64 = gapgpu.Context("fp64")
    ctx64.assemble(gapgpu.problem_from_arrays(sub, np.zeros(sub.n_rows), device="cuda"))
    E64 = torch.empty(sub.n_cfg, dtype=torch.float64, device="cuda")
    F64 = torch.empty(3 * sub.n_atoms, dtype=torch.float64, device="cuda")
    ctx64.predict(None, c, E64, F64)
    # the sub-problem holds the sampled configurations in order, their atoms in order
    cfg_ptr, _ = gapgen.structure(r)
    Es = E[cfgs]
    Fs = np.concatenate([F[3 * int(cfg_ptr[A]):3 * int(cfg_ptr[A + 1])] for A in cfgs])
    print("FP64 GPU predictions of the sampled configurations: E %.2e F %.2e"
          % (rel(Es, E64.cpu().numpy()), rel(Fs, F64.cpu().numpy())))
    assert rel(Es, E64.cpu().numpy()) < 1e-6 and rel(Fs, F64.cpu().numpy()) < 1e-6
    ctx64.close()
