"""The part-by-part drawing of the synthetic inputs (``gapgen.make_part``,
``fingerprint_of_recipe``, ``structure``) that lets the oracle handle workload 5 (132 GB of
Jacobians) on a host that cannot hold it, and the stored records written that way.

A part must equal the same configurations cut out of the whole drawn problem, and the
fingerprint computed without drawing the whole problem must equal the whole problem's."""
import dataclasses
import os

import numpy as np
import pytest

import gapgen

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")

FIELDS = ("cfg_ptr", "X", "sparse_idx", "Xs", "c_star", "noise_e", "sigma_e", "atom_species", "sparse_species",
          "pair_ptr", "pair_src", "J", "noise_f", "sigma_f")

RECIPES = [
    dataclasses.replace(gapgen.RECIPES[5], n_cfg=40, n_sparse=(20, 21, 19)),  # three species, d = 1024
    dataclasses.replace(gapgen.RECIPES[2], n_cfg=30, n_sparse=(50,), d=64),
    gapgen.RECIPES[1],  # energies only
]


@pytest.mark.parametrize("r", RECIPES, ids=["species", "forces", "energies"])
def test_parts_equal_the_whole_problem_cut(r):
    p = gapgen.make_problem(r)
    for c0, c1 in [(0, r.n_cfg), (3, 17), (r.n_cfg - 1, r.n_cfg)]:
        q = gapgen.select_configurations(p, np.arange(c0, c1))
        t = gapgen.make_part(r, c0, c1)
        for f in FIELDS:
            a, b = getattr(q, f), getattr(t, f)
            assert (a is None) == (b is None), f
            if a is not None:
                assert np.array_equal(a, b), (f, c0, c1)
    empty = gapgen.make_part(r, 5, 5)
    assert empty.n_cfg == 0 and empty.n_atoms == 0


@pytest.mark.parametrize("r", RECIPES, ids=["species", "forces", "energies"])
def test_fingerprint_and_structure_without_the_whole_problem(r):
    p = gapgen.make_problem(r)
    assert gapgen.fingerprint_of_recipe(r) == gapgen.fingerprint(p)
    cfg_ptr, pair_ptr = gapgen.structure(r)
    assert np.array_equal(cfg_ptr, p.cfg_ptr)
    assert (pair_ptr is None) == (p.pair_ptr is None)
    if pair_ptr is not None:
        assert np.array_equal(pair_ptr, p.pair_ptr)


def test_parts_refuse_what_they_do_not_draw():
    with pytest.raises(ValueError):
        gapgen.make_part(dataclasses.replace(gapgen.RECIPES[2], n_cfg=10, virials=True), 0, 5)
    with pytest.raises(ValueError):
        gapgen.make_part(gapgen.RECIPES[2], 5, 3)


def test_workload5_records_belong_to_workload5():
    """The stored targets and sampled oracle rows of workload 5 carry the fingerprint of the
    drawn workload, and the rows cover the configurations the record names."""
    r = gapgen.RECIPES[5]
    fp = gapgen.fingerprint_of_recipe(r)
    z = np.load(gapgen.targets_path(5))
    assert str(z["fingerprint"]) == fp
    n_atoms, _ = gapgen.count_shape(r)
    assert int(z["n_rows"]) == len(z["y"]) == r.n_cfg + 3 * n_atoms
    rows = np.load(os.path.join(GOLDEN, "workload5_sampled_rows.npz"))
    assert str(rows["fingerprint"]) == fp
    cfg_ptr, _ = gapgen.structure(r)
    n = sum(1 + 3 * int(cfg_ptr[A + 1] - cfg_ptr[A]) for A in rows["cfgs"])
    assert rows["rows"].shape == (n, len(rows["cols"]))
    assert rows["cols"][-1] == sum(r.n_sparse) - 1
    # the sampled configurations include the last one and one across the first ring chunk
    assert int(rows["cfgs"][0]) == 0 and int(rows["cfgs"][-1]) == r.n_cfg - 1


def test_workload2_inputs_follow_the_recipe():
    """The workload-2 inputs have the stated shapes and value distributions: configurations of
    16-128 atoms, 8-24 pairs per atom from the atom's own configuration, unit-length
    non-negative descriptors, sparse points that are distinct atoms, N(0, 0.1^2) Jacobians,
    sigma_A = 1e-3 sqrt(n_A), sigma_F = 1e-2, and target noise of those sigmas."""
    r = gapgen.RECIPES[2]
    p = gapgen.make_problem(r, max_cfg=4)
    n_at = np.diff(p.cfg_ptr)
    assert n_at.min() >= 16 and n_at.max() <= 128
    n_nb = np.diff(p.pair_ptr)
    assert n_nb.min() >= 8 and n_nb.max() <= 24
    cfg_of = np.repeat(np.arange(p.n_cfg), n_at)
    tgt = np.repeat(np.arange(p.n_atoms), n_nb)
    assert np.array_equal(cfg_of[p.pair_src], cfg_of[tgt])
    for Y in (p.X, p.Xs):
        assert (Y >= 0).all() and np.abs(np.linalg.norm(Y, axis=1) - 1.0).max() < 1e-14
    assert p.Xs.shape == (4000, 512) and len(np.unique(p.sparse_idx)) == 4000
    n_full, _ = gapgen.count_shape(r)
    assert p.sparse_idx.min() >= 0 and p.sparse_idx.max() < n_full
    assert abs(p.J.std() / 0.1 - 1) < 0.01 and abs(p.J.mean()) < 1e-3
    assert np.allclose(p.sigma_e, 1e-3 * np.sqrt(n_at), rtol=1e-15, atol=0)
    assert (p.sigma_f == 1e-2).all()
    assert abs(p.noise_f.std() / 1e-2 - 1) < 0.05


def test_workload5_species_and_sizes():
    r = gapgen.RECIPES[5]
    p = gapgen.make_problem(r, max_cfg=3)
    assert sorted(np.unique(p.atom_species).tolist()) == [0, 1, 2]
    assert np.bincount(p.sparse_species).tolist() == [5334, 5333, 5333]
    assert p.Xs.shape == (16000, 1024)
    cfg_ptr, pair_ptr = gapgen.structure(r)
    n_at = np.diff(cfg_ptr)
    assert len(n_at) == 6000 and n_at.min() >= 16 and n_at.max() <= 96
    n_atoms, n_pairs = gapgen.count_shape(r)
    assert (n_atoms, n_pairs) == (335097, 5365085)
    assert 6000 + 3 * n_atoms == 1011291


def test_workload4_sweep_recipes():
    """The 64 sweep fits: rows ~ logU[2000, 40000] in whole configurations, M ~ logU[200, 2000],
    zeta in {2, 3, 4}, sigma_E in {1e-4, 1e-3, 1e-2}; 866,798 rows of the stacked matrices
    (817,574 data rows and 49,224 rows of U) in all."""
    rs = gapgen.sweep_recipes()
    assert len(rs) == 64
    total = 0
    for r in rs:
        n_atoms, _ = gapgen.count_shape(r)
        rows = r.n_cfg + 3 * n_atoms
        assert 2000 <= rows < 40000 + 1 + 3 * 128
        assert 200 <= r.n_sparse[0] <= 2000 and r.zeta in (2, 3, 4) and r.sigma_e_atom in (1e-4, 1e-3, 1e-2)
        assert r.d == 256 and r.neighbours == (8, 24)
        total += rows + r.n_sparse[0]
    assert total == 866798
    assert {r.zeta for r in rs} == {2, 3, 4} and {r.sigma_e_atom for r in rs} == {1e-4, 1e-3, 1e-2}
