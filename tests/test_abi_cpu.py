"""The C-ABI library builds, loads and exports every symbol include/gap.h
declares; its host-only calls (sizes, validation, errors) work without a GPU."""
import ctypes
import json
import os
import re

import numpy as np
import pytest

import paper_2207_03803_gb300 as gapgpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    gapgpu.build()
    return gapgpu.load()


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "gap.h")).read()
    return sorted(set(re.findall(r"^\s*(?:gap_status|void|const char \*|int64_t|int)\s*\**\s*(gap_\w+)\s*\(", src, re.M)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_symbols()
    assert len(names) >= 12
    assert set(names) == set(gapgpu.EXPORTS)
    for n in names:
        assert hasattr(lib, n), n


def _host_problem(N_cfg=3, n_atoms=7, d=4, M=5, forces=True):
    cfg_ptr = np.array([0, 2, 5, 7], np.int64)
    X = np.ones((n_atoms, d)) / 2.0
    Xs = np.ones((M, d)) / 2.0
    kw = dict(cfg_ptr=cfg_ptr, X=X, Xs=Xs, delta=1.0, zeta=2)
    N = N_cfg
    if forces:
        pair_ptr = np.arange(n_atoms + 1, dtype=np.int64)
        pair_src = np.array([0, 1, 2, 3, 4, 5, 6], np.int64)
        kw.update(pair_ptr=pair_ptr, pair_src=pair_src, J=np.zeros((n_atoms, 3, d)))
        N += 3 * n_atoms
    kw.update(y=np.zeros(N), sigma=np.ones(N))
    return kw


def test_design_rows_and_workspace_reproduce_paper_sizes(lib):
    """(N + M) x M elements of Eq. (7) for the printed HEA and SiC sizes (Sec. IV)."""
    g = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_sizes.json")))
    for name in ("HEA", "SiC"):
        s = g[name]
        st = gapgpu.gap_problem()
        # N targets as energy rows only (the library counts rows, not their kind)
        st.n_cfg, st.n_atoms, st.d, st.n_pairs, st.n_sparse = s["N"], 1, 1, 0, s["M"]
        st.zeta, st.delta = 2, 1.0
        st.cfg_ptr = st.X = st.Xs = 1  # non-NULL placeholders; never dereferenced
        rows = lib.gap_design_rows(ctypes.byref(st))
        assert rows * s["M"] == s["n_A"]
        out = ctypes.c_size_t()
        assert lib.gap_workspace_size(ctypes.byref(st), 0, ctypes.byref(out)) == 0
        assert out.value >= s["n_A"] * 8  # the FP64 design matrix alone
    # a force problem: one energy row per configuration and three per atom
    p = gapgpu.Problem(**_host_problem())
    assert p.n_rows == 3 + 21 + 5


def test_j_ring_workspace_fits_workload5_on_one_gpu(lib):
    """Workload 5 (6000 configurations, 335,097 atoms, 5,365,085 pairs, d = 1024,
    M = 16000, a host problem): the whole mixed layout (every pair's converted Jacobian
    rows resident) needs more than the 298 GB of a GB300.  With the J ring the converted
    rows count once per slot, plus the two FP64 slots."""
    import gapgen
    r = gapgen.RECIPES[5]
    n_atoms, n_pairs = gapgen.count_shape(r)
    assert (n_atoms, n_pairs) == (335097, 5365085)
    st = gapgpu.gap_problem()
    st.n_cfg, st.n_atoms, st.d, st.n_pairs, st.n_sparse = r.n_cfg, n_atoms, r.d, n_pairs, sum(r.n_sparse)
    st.zeta, st.delta, st.jitter, st.memory = r.zeta, 1.0, 1e-8, gapgpu.GAP_MEM_HOST
    st.cfg_ptr = st.X = st.Xs = st.pair_ptr = st.pair_src = st.J = 1  # placeholders; never dereferenced
    whole, ring = ctypes.c_size_t(), ctypes.c_size_t()
    bf16 = gapgpu.PRECISIONS["mixed_bf16"]
    assert lib.gap_workspace_size(ctypes.byref(st), bf16, ctypes.byref(whole)) == 0
    rows = 128 * 4096
    assert lib.gap_workspace_size_ring(ctypes.byref(st), bf16, rows, ctypes.byref(ring)) == 0
    assert whole.value > 298e9 > 200e9 > ring.value
    # the difference: every pair's 3 rows x 1024 converted (8 bytes per element counted)
    # against one slot, and the two FP64 slots of 4096 x 42 pairs
    packed = (-(-n_pairs // 42) * 128 - rows) * 1024 * 8
    slots = 2 * 4096 * 42 * 3 * 1024 * 8
    assert abs((whole.value - ring.value) - (packed - slots)) < 1e6
    # a device problem's J is read in place: no FP64 slots
    st.memory = gapgpu.GAP_MEM_DEVICE
    dev = ctypes.c_size_t()
    assert lib.gap_workspace_size_ring(ctypes.byref(st), bf16, rows, ctypes.byref(dev)) == 0
    assert ring.value - dev.value == slots
    st.memory = gapgpu.GAP_MEM_HOST
    for bad in (100, -128):
        assert lib.gap_workspace_size_ring(ctypes.byref(st), bf16, bad, ctypes.byref(ring)) == gapgpu.GAP_ERR_INVALID
    fp64 = gapgpu.PRECISIONS["fp64"]
    assert lib.gap_workspace_size_ring(ctypes.byref(st), fp64, rows, ctypes.byref(ring)) == gapgpu.GAP_ERR_INVALID


def test_invalid_arguments_are_rejected_on_the_host(lib):
    st = gapgpu.gap_problem()
    out = ctypes.c_size_t()
    assert lib.gap_workspace_size(ctypes.byref(st), 0, ctypes.byref(out)) == gapgpu.GAP_ERR_INVALID
    p = gapgpu.Problem(**_host_problem())
    p.struct.zeta = 0
    assert lib.gap_workspace_size(ctypes.byref(p.struct), 0, ctypes.byref(out)) == gapgpu.GAP_ERR_INVALID
    h = ctypes.c_void_p()
    assert lib.gap_create(ctypes.byref(h), 7, None) == gapgpu.GAP_ERR_INVALID
    assert lib.gap_last_error(None) == b"ctx is NULL"
    assert lib.gap_tsqr_blocks(None) == -1
    assert lib.gap_set_option(None, b"tsqr_shards", 4.0) == gapgpu.GAP_ERR_INVALID


def test_library_fails_loudly_when_missing(monkeypatch, tmp_path):
    monkeypatch.setattr(gapgpu, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(gapgpu, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        gapgpu.load()


def test_tsqr_plan_blocks_cover_the_data_rows(lib):
    """The TSQR plan (host logic of gap_factor's "tsqr_shards"): contiguous blocks from
    row 0 to N that start on 128-row tiles, each at least M + 128 rows, at most the
    requested count and as many as fit; none when N (or the padded column) is too short."""
    cases = [(441968, 4000, 4), (7237, 150, 7), (5730, 300, 3), (64, 64, 4), (1000, 10, 64),
             (20000, 4000, 9), (4128, 4000, 2), (4300, 4000, 2), (1090, 10, 5)]
    for N, M, want in cases:
        blocks = gapgpu.tsqr_plan(N, M, want)
        ld = -(-(N + M) // 128) * 128
        if N < M + 128 or ld < N + 128:
            assert blocks == [], (N, M, want)
            continue
        G = len(blocks)
        assert 1 <= G <= min(want, 64), (N, M, want, G)
        assert blocks[0][0] == 0 and sum(n for _, n in blocks) == N
        for (r0, n), (r1, _) in zip(blocks, blocks[1:]):
            assert r1 == r0 + n
        assert all(r0 % 128 == 0 and n >= M + 128 for r0, n in blocks), (N, M, want, blocks)
        if G < min(want, 64):  # one more block would be too short
            assert (N // (G + 1)) // 128 * 128 < M + 128, (N, M, want, G)
    assert gapgpu.tsqr_plan(441968, 4000, 0) == []
    assert lib.gap_tsqr_plan(-1, 4, 2, None, None) == -1


def test_scalar_validation_rejects_each_bad_field(lib):
    """Host-side checks of a problem's scalars and pointers (no GPU needed): each
    single bad field gives GAP_ERR_INVALID; the unmodified problem is accepted."""
    out = ctypes.c_size_t()

    def status(**bad):
        p = gapgpu.Problem(**_host_problem())
        for k, v in bad.items():
            setattr(p.struct, k, v)
        return lib.gap_workspace_size(ctypes.byref(p.struct), 0, ctypes.byref(out))

    assert status() == gapgpu.GAP_OK and out.value > 0
    for bad in (dict(n_cfg=0), dict(n_atoms=0), dict(d=0), dict(n_sparse=0), dict(n_pairs=-1),
                dict(zeta=0), dict(zeta=64), dict(delta=float("nan")), dict(jitter=-1e-8),
                dict(jitter=float("inf")), dict(memory=7), dict(cfg_ptr=None), dict(X=None), dict(Xs=None),
                dict(pair_src=None), dict(J=None)):
        assert status(**bad) == gapgpu.GAP_ERR_INVALID, bad
    p = gapgpu.Problem(**_host_problem(forces=False))
    assert lib.gap_workspace_size(ctypes.byref(p.struct), 0, ctypes.byref(out)) == gapgpu.GAP_OK
    p.struct.n_pairs = 5  # pairs without pair_ptr
    assert lib.gap_workspace_size(ctypes.byref(p.struct), 0, ctypes.byref(out)) == gapgpu.GAP_ERR_INVALID


def test_allocation_free_predictions_name_no_allocator():
    """gap_predict_static and the prediction kernels it launches (its own file and the
    SIMT prediction file) call no device allocator: no cudaMalloc of any kind, no
    cudaFree, no allocating stream-ordered call."""
    csrc = os.path.join(ROOT, "paper_2207_03803_gb300", "csrc")
    for fn in ("gap_static.cu", "k_predict.cu"):
        code = open(os.path.join(csrc, fn)).read()
        code = re.sub(r"//[^\n]*", "", code)  # comments may name what the code avoids
        for bad in ("cudaMalloc", "cudaFree", "cuMemAlloc", "cuMemFree", "DevBuf", ".ensure("):
            assert bad not in code, (fn, bad)
