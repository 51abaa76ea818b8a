"""Write the hidden-weight targets of workload 2 with the FP64 oracle.

Workload 2 (2000 configurations of 16-128 atoms, d=512, M=4000, zeta=4,
8-24 neighbours per atom) is the synthetic stand-in for the paper's HEA/SiC
training sets (Sec. IV).  Its targets y = K c* + noise need the model's
forward pass over 2.3 M pairs, too slow to redo before every benchmark run,
so this script computes them once with the oracle (and nothing else) and
stores them with a fingerprint of the generated inputs they belong to.

Workload 5 (6000 configurations, three species, d=1024, M=16000; 132 GB of FP64
Jacobians) does not fit in this host's memory at once: its targets are computed
configuration range by configuration range (``gapgen.make_part``; the model's
energies and forces of a configuration depend only on its own atoms and the
sparse set), and stored with ``gapgen.fingerprint_of_recipe``, which equals the
fingerprint of the whole drawn problem.

    python tests/golden/make_workload_targets.py [workload]   (2, 5, or 4: the 64-fit sweep)
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import gapgen  # noqa: E402
import oracle  # noqa: E402




def main(workload: int = 2):
    if workload == 4:
        return main_sweep()
    if workload == 5:
        return main_parts(workload)
    t0 = time.time()
    p = gapgen.make_problem(gapgen.RECIPES[workload])
    t1 = time.time()
    y = oracle.targets(p)
    t2 = time.time()
    np.savez(gapgen.targets_path(workload), y=y, fingerprint=np.array(gapgen.fingerprint(p)),
             n_rows=np.array(p.n_rows))
    print("workload %d: %d rows, generation %.1f s, oracle targets %.1f s" % (workload, p.n_rows, t1 - t0, t2 - t1))


def main_parts(workload: int, cfgs_per_part: int = 100):
    """Targets of a workload drawn and predicted in parts of configurations: energies of
    every configuration first, then the three force rows of every atom (the full
    problem's row order)."""
    r = gapgen.RECIPES[workload]
    t0 = time.time()
    E, F = [], []
    for c0 in range(0, r.n_cfg, cfgs_per_part):
        p = gapgen.make_part(r, c0, min(r.n_cfg, c0 + cfgs_per_part))
        e, f, _ = oracle.predict_all(p, p.c_star)
        E.append(e + p.noise_e)
        F.append(f + p.noise_f)
        del p
    y = np.concatenate(E + F)
    fp = gapgen.fingerprint_of_recipe(r)
    n_atoms, _ = gapgen.count_shape(r)
    assert len(y) == r.n_cfg + 3 * n_atoms
    np.savez(gapgen.targets_path(workload), y=y, fingerprint=np.array(fp), n_rows=np.array(len(y)))
    print("workload %d: %d rows in parts of %d configurations, %.1f s" % (workload, len(y), cfgs_per_part,
                                                                        time.time() - t0))


def main_sweep():
    """Workload 4: the targets of the 64 sweep fits, concatenated, with per-fit offsets
    and fingerprints."""
    ys, fps, offs = [], [], [0]
    t0 = time.time()
    for r in gapgen.sweep_recipes():
        p = gapgen.make_problem(r)
        ys.append(oracle.targets(p))
        fps.append(gapgen.fingerprint(p))
        offs.append(offs[-1] + p.n_rows)
    np.savez(gapgen.targets_path(4), y=np.concatenate(ys), offsets=np.array(offs, dtype=np.int64),
             fingerprints=np.array(fps))
    print("workload 4: %d fits, %d rows, %.1f s" % (len(ys), offs[-1], time.time() - t0))


if __name__ == "__main__":
    main(int(sys.argv[1]) if len(sys.argv) > 1 else 2)
