"""Design rows of sampled configurations of workload 5 at full size, from the FP64 oracle.

Workload 5 (6000 configurations, three species, d=1024, M=16000; 1,011,291 data rows)
is too large for an oracle fit, but the rows of any configuration are cheap: they depend
only on its own atoms, pairs and Jacobians and on the sparse set (Eqs. 6, 7).  This
script draws configurations of the full problem on their own (``gapgen.make_part``),
computes their energy and force rows with the oracle, and stores a fixed subset of the
columns (every 31st sparse point and the last one, across all three species blocks):

  cfgs         the configurations: the first, the one holding the first pair of the
               second 524,288-row chunk of the J ring (its pairs straddle the chunk
               boundary), one in the middle, the last
  cols         the stored columns
  rows         [sum over cfgs of (1 + 3 n_atoms), len(cols)]: each configuration's
               energy row, then its atoms' force rows (x, y, z), Sigma^-1/2 scaled
  fingerprint  gapgen.fingerprint_of_recipe of workload 5

The full-size benchmark (bench.py --workload 5) compares the library's rows of a
fit of the whole problem against these.

    python tests/golden/make_workload5_rows.py
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import gapgen  # noqa: E402
import oracle  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "workload5_sampled_rows.npz")
RING_PAIRS = 4096 * 42  # pairs of one 524,288-row chunk of the J ring


def sample_configurations(r):
    """The sampled configurations of recipe r (integer structure only)."""
    cfg_ptr, pair_ptr = gapgen.structure(r)
    a = int(np.searchsorted(pair_ptr, RING_PAIRS, side="right")) - 1  # atom holding pair RING_PAIRS
    A = int(np.searchsorted(cfg_ptr, a, side="right")) - 1
    return sorted({0, A, r.n_cfg // 2, r.n_cfg - 1})


def main():
    r = gapgen.RECIPES[5]
    M = sum(r.n_sparse)
    cols = np.unique(np.concatenate([np.arange(0, M, 31), [M - 1]])).astype(np.int64)
    cfgs = sample_configurations(r)
    t0 = time.time()
    rows = []
    for A in cfgs:
        q = gapgen.make_part(r, A, A + 1)
        d = oracle.design(q)  # its energy row, then 3 rows per atom
        rows.append(d[:, cols])
    rows = np.concatenate(rows)
    np.savez_compressed(OUT, cfgs=np.array(cfgs, np.int64), cols=cols, rows=rows,
                        fingerprint=np.array(gapgen.fingerprint_of_recipe(r)))
    print("configurations %s: %d rows x %d columns (%.1f s)" % (cfgs, rows.shape[0], len(cols), time.time() - t0))


if __name__ == "__main__":
    main()
