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
