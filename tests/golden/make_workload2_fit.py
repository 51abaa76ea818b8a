"""Fit workload 2 at full size with the FP64 oracle and store its weights and predictions.

Workload 2 (2000 configurations of 16-128 atoms, d=512, M=4000, zeta=4, 8-24
neighbours per atom; 441,968 design rows) is the synthetic stand-in for the
paper's HEA/SiC training sets (Sec. IV).  Its oracle fit -- the assembly of
Eq. (7), the Cholesky of K_MM, the Householder QR and back substitution of
Eq. (12), all in plain FP64 loops -- takes hours of host time, so this script
runs it once (oracle and generator only) and stores:

  c            the oracle's weights [M]
  E, F         the oracle's predictions with those weights (Eqs. 1, 2)
  fingerprint  of the generated inputs the record belongs to
  times        per-phase seconds: assembly, K_MM + Cholesky, QR, Q^T b + solve, predict
  host         machine, core count and date of the run

The full-size GPU parity test compares the library's fits against this record
in every precision, and the benchmark reports its errors against it.

    python tests/golden/make_workload2_fit.py
"""
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

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "workload2_oracle_fit.npz")


def main():
    t0 = time.time()
    p = gapgen.make_problem(gapgen.RECIPES[2])
    y = gapgen.load_targets(p, 2)
    t_gen = time.time() - t0
    print("generated workload 2: %d rows, %d pairs (%.1f s)" % (p.n_rows, p.n_pairs, t_gen), flush=True)
    t0 = time.time()
    c, times = oracle.fit(p, y)
    t_fit = time.time() - t0
    print("oracle fit %.1f s: assembly %.1f, K_MM + Cholesky %.1f, QR %.1f, solve %.1f"
          % (t_fit, *times), flush=True)
    t0 = time.time()
    E, F = oracle.predict(p, c)
    t_pred = time.time() - t0
    print("oracle predictions %.1f s" % t_pred, flush=True)
    host = {"machine": platform.machine(), "cores": os.cpu_count(),
            "omp_num_threads": os.environ.get("OMP_NUM_THREADS", ""),
            "date": datetime.datetime.now(datetime.timezone.utc).strftime("%Y-%m-%dT%H:%M:%SZ"),
            "fit_s": t_fit, "predict_s": t_pred}
    np.savez_compressed(OUT, c=c, E=E, F=F, fingerprint=np.array(gapgen.fingerprint(p)),
                        times=np.array(list(times) + [t_pred]), host=np.array(json.dumps(host)))
    print("wrote", OUT, json.dumps(host), flush=True)


if __name__ == "__main__":
    main()
