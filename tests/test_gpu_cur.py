"""CUR choice of the sparse set on the GPU (gap_select_cur) against the oracle
(oracle/cur.py) on the same seeded inputs: leverage scores element by element, and the
drawn atoms exactly, except where two keys are closer than the scores' rounding (there
either atom is a correct draw, and the two sets may differ only in such atoms)."""
import numpy as np
import pytest

import gapgen
from oracle import cur

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2207_03803_gb300 as gapgpu  # noqa: E402

LEV_TOL = 1e-9  # max |pi_gpu - pi_oracle| / max pi


@pytest.fixture(scope="module", autouse=True)
def lib():
    gapgpu.build()
    gapgpu.load()


def _run(X, species, n_select, k, l, q, seed):
    omega, u = gapgen.cur_draws(seed, X.shape[0], X.shape[1], l)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    sel, lev = gapgpu.select_cur(dev(X), n_select, k, l, dev(omega), dev(u), power_iters=q,
                                 atom_species=None if species is None else dev(species.astype(np.int32)),
                                 leverage=True)
    torch.cuda.synchronize()
    sel_or, lev_or = cur.select_cur(X, species, n_select, k, l, q, omega, u)
    return sel.cpu().numpy(), lev.cpu().numpy(), sel_or, lev_or, u


def _check(X, species, n_select, k, l, q, seed):
    sel, lev, sel_or, lev_or, u = _run(X, species, n_select, k, l, q, seed)
    done = ~np.isnan(lev_or)
    assert np.array_equal(np.isnan(lev), ~done)
    err = np.abs(lev[done] - lev_or[done]).max() / lev_or[done].max()
    assert err < LEV_TOL, err
    assert len(sel) == len(sel_or) == sum(n_select)
    spec = np.zeros(X.shape[0], np.int64) if species is None else species
    o = 0
    for t, m in enumerate(n_select):
        a, b = sel[o:o + m], sel_or[o:o + m]
        o += m
        assert (spec[a] == t).all() and (np.diff(a) > 0).all()
        if np.array_equal(a, b):
            continue
        # differing atoms must sit at the draw's threshold, within the scores' rounding
        atoms = np.nonzero(spec == t)[0]
        pi = lev_or[atoms]
        key = np.where(pi > 0, np.log(u[atoms]) / np.where(pi > 0, pi, 1), -np.inf)
        thr = np.sort(key)[::-1][m - 1]
        diff = np.setxor1d(a, b)
        kd = np.log(u[diff]) / lev_or[diff]
        assert np.all(np.abs(kd - thr) <= 1e-7 * np.abs(thr)), (diff, kd, thr)
    return err


@pytest.mark.parametrize("n,d,k,l,q,m", [
    (3000, 64, 8, 24, 2, 150),     # several row tiles and slabs, a ragged tail
    (1037, 37, 7, 23, 1, 61),      # odd l, d not a multiple of the tile
    (700, 130, 16, 128, 1, 40),    # the largest l
    (257, 9, 1, 1, 0, 5),          # k = l = 1, no power iteration
    (90, 16, 3, 8, 3, 90),         # every atom drawn
])
def test_cur_matches_oracle(n, d, k, l, q, m):
    X = gapgen.clustered_descriptors(31 + n, n, d, 40)
    _check(X, None, [m], k, l, q, 31 + n)


def test_cur_species_blocks_match_oracle():
    n, d = 5000, 96
    X = gapgen.clustered_descriptors(77, n, d, 60)
    species = gapgen.uniform_ints(77, 911, n, 0, 3).astype(np.int32)
    _check(X, species, [120, 0, 300, 17], 12, 40, 2, 77)


@pytest.mark.parametrize("w", [2, 5])
def test_cur_workload_descriptors_full_size(w):
    """The workloads' own descriptor rows, their sparse points by CUR with k = 64, l = 96
    and two power iterations: workload 2 (about 144,000 atoms, d = 512, 4000 points) and
    workload 5 (three species, about 336,000 atoms, d = 1024, 5334 + 5333 + 5333)."""
    r = gapgen.RECIPES[w]
    X, species = gapgen.recipe_descriptors(r)
    err = _check(X, species, list(r.n_sparse), 64, 96, 2, r.seed)
    print("workload %d CUR leverage error %.2e" % (w, err))


def test_cur_rank_deficient_rows():
    """Rows spanning 5 < l = 8 directions: the range basis holds them all (the shifted
    first CholeskyQR pass keeps the factor finite), so the rank-4 scores are exact and
    match the oracle's."""
    A = gapgen.normals(5, 912, 300 * 5).reshape(300, 5) @ gapgen.normals(5, 913, 5 * 16).reshape(5, 16)
    try:
        _check(A, None, [10], 4, 8, 1, 5)
    except gapgpu.GapError as e:  # a later plain pass may still meet a non-positive pivot
        assert e.status == gapgpu.GAP_ERR_RANK


def test_cur_errors_are_reported():
    X = gapgen.clustered_descriptors(5, 200, 16, 10)
    om, u = gapgen.cur_draws(5, 200, 16, 8)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    Xd, omd, ud = dev(X), dev(om), dev(u)
    with pytest.raises(gapgpu.GapError) as e:
        gapgpu.select_cur(Xd, [201], 4, 8, omd, ud)
    assert e.value.status == gapgpu.GAP_ERR_INVALID
    with pytest.raises(gapgpu.GapError) as e:  # l > d
        om2, _ = gapgen.cur_draws(5, 200, 16, 20)
        gapgpu.select_cur(Xd, [10], 4, 20, dev(om2), ud)
    assert e.value.status == gapgpu.GAP_ERR_INVALID
    with pytest.raises(gapgpu.GapError) as e:  # a species value out of range
        gapgpu.select_cur(Xd, [10, 10], 4, 8, omd, ud, atom_species=dev(np.full(200, 2, np.int32)))
    assert e.value.status == gapgpu.GAP_ERR_INVALID
    # rows that span no direction at all: CholeskyQR meets a zero pivot even after its shift
    with pytest.raises(gapgpu.GapError) as e:
        gapgpu.select_cur(torch.zeros_like(Xd), [10], 4, 8, omd, ud)
    assert e.value.status == gapgpu.GAP_ERR_RANK
    # the library stays usable after the errors
    sel = gapgpu.select_cur(Xd, [10], 4, 8, omd, ud)
    assert sel.shape == (10,)
