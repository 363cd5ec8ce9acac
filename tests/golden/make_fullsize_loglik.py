"""Write fullsize_loglik_n40000.json: the exact l(theta) (Eq. 1.2) of the
benchmark's full-size workload, from the oracle alone.

Workload: n = 40,000 locations of synth.jittered_grid(40000, seed=1) in
generation order, Z = synth.standard_normal(40000, seed=2), theta = (sigma2 1,
beta 0.1, nu 0.5).  Exact l does not depend on the order of the locations
(Sec. 3), so the value checks the TLR likelihood under any ordering.  The
oracle builds the dense 40,000 x 40,000 covariance (12.8 GB) and factors it
with LAPACK, single-threaded (a threaded OpenBLAS build of this size of
problem crashed); about fifteen minutes.

Usage: python tests/golden/make_fullsize_loglik.py
"""
import json
import os
import sys
import time

os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")  # before numpy loads OpenBLAS

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402

N, THETA, LOC_SEED, Z_SEED = 40000, (1.0, 0.1, 0.5), 1, 2


def main():
    t0 = time.time()
    xy = synth.jittered_grid(N, seed=LOC_SEED)
    z = synth.standard_normal(N, seed=Z_SEED)
    r = oracle.loglik_dense(xy, z, THETA)
    out = {"n": N, "theta": list(THETA), "loc_seed": LOC_SEED, "z_seed": Z_SEED,
           "z": "synth.standard_normal(n, seed=z_seed)", "order": "generation",
           "loglik": r["loglik"], "logdet": r["logdet"], "quad": r["quad"],
           "source": "oracle.loglik_dense (dense FP64 covariance, LAPACK Cholesky)",
           "seconds": round(time.time() - t0, 1)}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "fullsize_loglik_n40000.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
