"""Fit the 600-configuration reduction of workload 5 with the FP64 oracle and store it.

Workload 5 (three species, d=1024, zeta=4) is the largest synthetic stand-in for the
paper's training sets (Sec. IV).  This reduction keeps its shape at a size the oracle
fits in minutes: 600 configurations of 16-96 atoms (32,929 atoms, 99,387 data rows,
527,258 pairs, 13 GB of FP64 Jacobians) with 534 + 533 + 533 sparse points.  The
script draws it (generator only), computes its hidden-weight targets, fits it and
predicts with the oracle (the assembly of Eq. (7), the Cholesky of K_MM, the
Householder QR and back substitution of Eq. (12), all in plain FP64 loops), and stores:

  y            the targets
  c            the oracle's weights [M]
  E, F         the oracle's predictions with those weights (Eqs. 1, 2)
  fingerprint  of the generated inputs the record belongs to
  times        per-phase seconds: assembly, K_MM + Cholesky, QR, Q^T b + solve, predict
  host         machine, core count and date of the run

The GPU test of the J ring (the force pass fed chunk by chunk from host memory)
compares the library's fits of this instance against the record in every precision.

    python tests/golden/make_workload5_reduced_fit.py
"""
import dataclasses
import datetime
import json
import os
import platform
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import gapgen  # noqa: E402
import oracle  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "workload5_reduced_oracle_fit.npz")


def recipe():
    """The reduction: workload 5's recipe with 600 configurations and 1600 sparse points."""
    return dataclasses.replace(gapgen.RECIPES[5], n_cfg=600, n_sparse=(534, 533, 533))


def main():
    t0 = time.time()
    p = gapgen.make_problem(recipe())
    print("generated: %d configurations, %d atoms, %d rows, %d pairs (%.1f s)"
          % (p.n_cfg, p.n_atoms, p.n_rows, p.n_pairs, time.time() - t0), flush=True)
    t0 = time.time()
    y = oracle.targets(p)
    t_y = time.time() - t0
    t0 = time.time()
    c, times = oracle.fit(p, y)
    t_fit = time.time() - t0
    print("targets %.1f s; oracle fit %.1f s: assembly %.1f, K_MM + Cholesky %.1f, QR %.1f, solve %.1f"
          % (t_y, t_fit, *times), flush=True)
    t0 = time.time()
    E, F = oracle.predict(p, c)
    t_pred = time.time() - t0
    host = {"machine": platform.machine(), "cores": os.cpu_count(),
            "omp_num_threads": os.environ.get("OMP_NUM_THREADS", ""),
            "date": datetime.datetime.now(datetime.timezone.utc).strftime("%Y-%m-%dT%H:%M:%SZ"),
            "targets_s": t_y, "fit_s": t_fit, "predict_s": t_pred}
    np.savez_compressed(OUT, y=y, c=c, E=E, F=F, fingerprint=np.array(gapgen.fingerprint(p)),
                        times=np.array(list(times) + [t_pred]), host=np.array(json.dumps(host)))
    print("wrote", OUT, json.dumps(host), flush=True)


if __name__ == "__main__":
    main()
