"""The J ring (option "j_ring_rows", mixed precisions): the tensor-core force pass packs and
multiplies one chunk of pair tiles at a time through one operand slot, and a host problem's
Jacobians are copied chunk by chunk through two FP64 slots instead of being staged whole
(the layout that fits workload 5's 132 GB of Jacobians, Sec. IV, on one GPU).

Checked against the oracle (design rows, fits, predictions) and against the whole layout:
- chunks that cut targets' pair runs;
- targets of more pairs than one chunk;
- host and device problems;
- predictions through the ring;
- the reductions of workload 5 (three species, d = 1024): 60 configurations against a fresh
  oracle fit, and 600 configurations against the stored oracle fit of
  tests/golden/make_workload5_reduced_fit.py;
- the refusals."""
import os

import numpy as np
import pytest

import gapgen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2207_03803_gb300 as gapgpu  # noqa: E402

MIXED = ["mixed_bf16", "mixed_fp16", "mixed_tf32"]
GOLDEN_600 = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "workload5_reduced_oracle_fit.npz")


@pytest.fixture(scope="module", autouse=True)
def built():
    gapgpu.build()
    gapgpu.load()


def rel(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


_cache = {}


def problem():
    """37 configurations of 3-128 atoms, 0-80 pairs per atom (targets of up to two pair
    tiles), d = 47, M = 150: with 256-row chunks (84 pairs) most targets' pair runs are cut
    by a chunk boundary, and some targets span three chunks."""
    if "base" not in _cache:
        r = gapgen.Recipe(n_cfg=37, atoms=(3, 128), d=47, n_sparse=(150,), zeta=4, neighbours=(0, 80), seed=23)
        p = gapgen.make_problem(r)
        y = oracle.targets(p)
        c, _ = oracle.fit(p, y)
        _cache["base"] = (p, y, c, oracle.predict(p, c))
    return _cache["base"]


def fit(p, y, precision, device, ring, n_w=None):
    prob = gapgpu.problem_from_arrays(p, y, device=device)
    ctx = gapgpu.Context(precision)
    if ring:
        ctx.set_option("j_ring_rows", ring)
    ctx.assemble(prob)
    ctx.factor()
    c = torch.empty(n_w or p.n_sparse, dtype=torch.float64, device="cuda")
    info = ctx.solve(c)
    return ctx, prob, c, info


def predict(ctx, p, c, device):
    tgt = gapgpu.problem_from_arrays(p, np.zeros(p.n_rows), device=device)
    E = torch.empty(p.n_cfg, dtype=torch.float64, device="cuda")
    F = torch.empty(3 * p.n_atoms, dtype=torch.float64, device="cuda")
    ctx.predict(tgt, c, E, F)
    return E.cpu().numpy(), F.cpu().numpy()


@pytest.mark.parametrize("device", ["cuda", "cpu"])
@pytest.mark.parametrize("precision", MIXED)
def test_ring_design_rows_match_oracle_and_whole_layout(precision, device):
    p, y, *_ = problem()
    ref = oracle.design(p)
    rows = {}
    for ring in (0, 256):
        ctx = gapgpu.Context(precision)
        if ring:
            ctx.set_option("j_ring_rows", ring)
        ctx.assemble(gapgpu.problem_from_arrays(p, y, device=device))
        for which in (0, 1):
            out = torch.empty((p.n_rows, p.n_sparse), dtype=torch.float64, device="cuda")
            ctx.read_design(which, 0, p.n_rows, out)
            rows[(ring, which)] = out.cpu().numpy()
        ctx.close()
    acc = rows[(256, 1)]
    print(precision, device, "ring vs oracle: energy %.2e force %.2e; ring vs whole %.2e"
          % (rel(acc[:p.n_cfg], ref[:p.n_cfg]), rel(acc[p.n_cfg:], ref[p.n_cfg:]), rel(acc, rows[(0, 1)])))
    assert rel(acc[:p.n_cfg], ref[:p.n_cfg]) < 2e-7
    assert rel(acc[p.n_cfg:], ref[p.n_cfg:]) < 2e-6
    scale = np.abs(ref).max(axis=1, keepdims=True) + 1e-300
    assert np.max(np.abs(acc - ref) / scale) < 1e-5
    # the same sums as the whole layout, added in another order (FP32 reduce-adds)
    assert rel(acc, rows[(0, 1)]) < 1e-6
    assert rel(rows[(256, 0)], rows[(0, 0)]) < 1e-6
    assert np.array_equal(acc[:p.n_cfg], rows[(0, 1)][:p.n_cfg])  # energy rows do not use J


@pytest.mark.parametrize("precision", MIXED)
def test_ring_fits_and_predictions_match_oracle(precision):
    """Host and device problems through a 1024-row ring; the predictions of a host problem
    through the ring equal those of the device problem bit for bit (the same per-atom sums,
    the Jacobians of each run of atoms read from a slot instead of in place)."""
    p, y, c_or, (E_or, F_or) = problem()
    for device in ("cuda", "cpu"):
        ctx, _, c, info = fit(p, y, precision, device, 1024)
        E1, F1 = oracle.predict(p, c.cpu().numpy())
        print(precision, device, "fit E %.2e F %.2e" % (rel(E1, E_or), rel(F1, F_or)), info["iterations"])
        assert rel(E1, E_or) < 1e-6 and rel(F1, F_or) < 1e-6
        Eh, Fh = predict(ctx, p, c, "cpu")
        Ed, Fd = predict(ctx, p, c, "cuda")
        assert np.array_equal(Eh, Ed) and np.array_equal(Fh, Fd)
        assert rel(Ed, E_or) < 1e-6 and rel(Fd, F_or) < 1e-6
        ctx.close()


@pytest.mark.parametrize("precision", MIXED)
def test_predictions_of_the_last_ring_problem_from_its_design_rows(precision):
    """After a ring assembly of a host problem its Jacobians are not on the device:
    gap_predict(NULL) gives sigma times the design rows times c (Eq. 7), energies from the
    FP64 energy rows, forces from the FP32-accurate rows.  Against the predictions through
    the ring and against the oracle's predictions with the same weights."""
    p, y, c_or, (E_or, F_or) = problem()
    ctx, prob, c, info = fit(p, y, precision, "cpu", 512)
    E = torch.empty(p.n_cfg, dtype=torch.float64, device="cuda")
    F = torch.empty(3 * p.n_atoms, dtype=torch.float64, device="cuda")
    ctx.predict(None, c, E, F)
    Ed, Fd = E.cpu().numpy(), F.cpu().numpy()
    # energies only
    E2 = torch.empty(p.n_cfg, dtype=torch.float64, device="cuda")
    ctx.predict(None, c, E2)
    assert np.array_equal(E2.cpu().numpy(), Ed)
    Er, Fr = predict(ctx, p, c, "cpu")  # host targets: the last problem's copies are replaced
    E1, F1 = oracle.predict(p, c.cpu().numpy())
    print(precision, "design rows vs oracle E %.2e F %.2e; vs ring predictions E %.2e F %.2e"
          % (rel(Ed, E1), rel(Fd, F1), rel(Ed, Er), rel(Fd, Fr)))
    assert rel(Ed, E1) < 1e-7 and rel(Fd, F1) < 1e-6
    assert rel(Ed, Er) < 1e-7 and rel(Fd, Fr) < 1e-6
    ctx.close()


_w5 = {}


@pytest.mark.parametrize("precision", MIXED)
def test_workload5_reduced_through_ring(precision):
    """The workload-5 recipe with 60 configurations and 54 + 53 + 53 sparse points (three
    species, d = 1024: two K-chunks per ring chunk) from host memory through a ring of 4096
    rows (1344 pairs; 40 chunks)."""
    import dataclasses
    if not _w5:
        r = dataclasses.replace(gapgen.RECIPES[5], n_cfg=60, n_sparse=(54, 53, 53))
        p = gapgen.make_problem(r)
        y = oracle.targets(p)
        c, _ = oracle.fit(p, y)
        _w5.update(p=p, y=y, EF=oracle.predict(p, c))
    p, y, (E_or, F_or) = _w5["p"], _w5["y"], _w5["EF"]
    ctx, _, c, info = fit(p, y, precision, "cpu", 4096)
    E1, F1 = oracle.predict(p, c.cpu().numpy())
    E2, F2 = predict(ctx, p, c, "cpu")
    print("workload 5 reduced, ring", precision, "E %.2e F %.2e" % (rel(E1, E_or), rel(F1, F_or)), info["iterations"])
    assert rel(E1, E_or) < 1e-6 and rel(F1, F_or) < 1e-6
    assert rel(E2, E_or) < 1e-6 and rel(F2, F_or) < 1e-6
    ctx.close()


_w600 = {}


@pytest.mark.parametrize("precision", MIXED)
def test_workload5_600_configurations_against_stored_oracle_fit(precision):
    """The 600-configuration reduction of workload 5 (32,929 atoms, 527,258 pairs, 13 GB of
    FP64 Jacobians in host memory, M = 1600) through a ring of 32,768 rows (50 chunks)
    against the oracle's stored fit: predictions of the fitted weights to 1e-6."""
    import dataclasses
    if not _w600:
        z = np.load(GOLDEN_600)
        r = dataclasses.replace(gapgen.RECIPES[5], n_cfg=600, n_sparse=(534, 533, 533))
        p = gapgen.make_problem(r)
        assert str(z["fingerprint"]) == gapgen.fingerprint(p)
        _w600.update(p=p, y=np.ascontiguousarray(z["y"]), E=z["E"], F=z["F"])
    p, y, E_or, F_or = _w600["p"], _w600["y"], _w600["E"], _w600["F"]
    ctx, _, c, info = fit(p, y, precision, "cpu", 32768)
    E = torch.empty(p.n_cfg, dtype=torch.float64, device="cuda")
    F = torch.empty(3 * p.n_atoms, dtype=torch.float64, device="cuda")
    ctx.predict(None, c, E, F)  # from the design rows
    E3, F3 = E.cpu().numpy(), F.cpu().numpy()
    E2, F2 = predict(ctx, p, c, "cpu")  # from the descriptors, J through the ring
    print("workload 5, 600 configurations, ring", precision, "E %.2e F %.2e; from the design rows E %.2e F %.2e"
          % (rel(E2, E_or), rel(F2, F_or), rel(E3, E_or), rel(F3, F_or)), info["iterations"])
    assert rel(E2, E_or) < 1e-6 and rel(F2, F_or) < 1e-6
    assert rel(E3, E_or) < 1e-6 and rel(F3, F_or) < 1e-6
    ctx.close()


@pytest.mark.parametrize("precision", MIXED)
def test_ring_reads_page_locked_host_J_in_place(precision):
    """j_ring_direct: a pinned host J read in place by the packing and prediction kernels
    gives the same design rows as the copies through the FP64 slots, up to the order of the
    FP32 reduce-adds, and the same predictions bit for bit (the same per-atom sums)."""
    p, y, c_or, (E_or, F_or) = problem()
    out = {}
    for direct in (0, 1):
        prob = gapgpu.problem_from_arrays(p, y, device="cpu", pinned=True)
        ctx = gapgpu.Context(precision)
        ctx.set_option("j_ring_rows", 512)
        ctx.set_option("j_ring_direct", direct)
        ctx.assemble(prob)
        rows = torch.empty((p.n_rows, p.n_sparse), dtype=torch.float64, device="cuda")
        ctx.read_design(1, 0, p.n_rows, rows)
        ctx.factor()
        c = torch.empty(p.n_sparse, dtype=torch.float64, device="cuda")
        ctx.solve(c)
        E = torch.empty(p.n_cfg, dtype=torch.float64, device="cuda")
        F = torch.empty(3 * p.n_atoms, dtype=torch.float64, device="cuda")
        ctx.predict(prob, torch.from_numpy(c_or).cuda(), E, F)
        out[direct] = (rows.cpu().numpy(), E.cpu().numpy(), F.cpu().numpy(), c.cpu().numpy())
        ctx.close()
    assert rel(out[1][0], out[0][0]) < 1e-6
    assert np.array_equal(out[1][1], out[0][1]) and np.array_equal(out[1][2], out[0][2])
    E1, F1 = oracle.predict(p, out[1][3])
    assert rel(E1, E_or) < 1e-6 and rel(F1, F_or) < 1e-6
    # pageable host memory cannot be read in place
    ctx = gapgpu.Context(precision)
    ctx.set_option("j_ring_rows", 512)
    ctx.set_option("j_ring_direct", 1)
    with pytest.raises(gapgpu.GapError) as e:
        ctx.assemble(gapgpu.problem_from_arrays(p, y, device="cpu"))
    assert e.value.status == gapgpu.GAP_ERR_INVALID
    ctx.close()


def test_ring_refusals():
    p, y, c_or, _ = problem()
    ctx = gapgpu.Context("fp64")
    with pytest.raises(gapgpu.GapError) as e:
        ctx.set_option("j_ring_rows", 1024)
    assert e.value.status == gapgpu.GAP_ERR_INVALID
    ctx.close()
    ctx = gapgpu.Context("mixed_bf16")
    for bad in (100, -128, 128.5):
        with pytest.raises(gapgpu.GapError) as e:
            ctx.set_option("j_ring_rows", bad)
        assert e.value.status == gapgpu.GAP_ERR_INVALID
    # a virial problem
    rv = gapgen.Recipe(n_cfg=9, atoms=(3, 20), d=31, n_sparse=(40,), zeta=3, neighbours=(1, 9), virials=True, seed=5)
    pv = gapgen.make_problem(rv)
    ctx.set_option("j_ring_rows", 256)
    with pytest.raises(gapgpu.GapError) as e:
        ctx.assemble(gapgpu.problem_from_arrays(pv, np.zeros(pv.n_rows)))
    assert e.value.status == gapgpu.GAP_ERR_INVALID
    ctx.set_option("j_ring_rows", 128)
    ctx.assemble(gapgpu.problem_from_arrays(p, y, device="cpu"))
    ctx.factor()
    c = torch.empty(p.n_sparse, dtype=torch.float64, device="cuda")
    ctx.solve(c)
    # a 128-row ring holds 42 pairs: an atom with more cannot be predicted through it
    assert np.diff(p.pair_ptr).max() > 42
    with pytest.raises(gapgpu.GapError) as e:
        predict(ctx, p, c, "cpu")
    assert e.value.status == gapgpu.GAP_ERR_INVALID
    ctx.close()
