"""Write the hidden-weight targets of workload 2 with the FP64 oracle.

Workload 2 (2000 configurations of 16-128 atoms, d=512, M=4000, zeta=4,
8-24 neighbours per atom) is the synthetic stand-in for the paper's HEA/SiC
training sets (Sec. IV).  Its targets y = K c* + noise need the model's
forward pass over 2.3 M pairs, too slow to redo before every benchmark run,
so this script computes them once with the oracle (and nothing else) and
stores them with a fingerprint of the generated inputs they belong to.

    python tests/golden/make_workload_targets.py [workload]   (2, or 4: the 64-fit sweep)
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
    t0 = time.time()
    p = gapgen.make_problem(gapgen.RECIPES[workload])
    t1 = time.time()
    y = oracle.targets(p)
    t2 = time.time()
    np.savez(gapgen.targets_path(workload), y=y, fingerprint=np.array(gapgen.fingerprint(p)),
             n_rows=np.array(p.n_rows))
    print("workload %d: %d rows, generation %.1f s, oracle targets %.1f s" % (workload, p.n_rows, t1 - t0, t2 - t1))


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
