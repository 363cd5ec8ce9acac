"""Write the full-size golden files of the benchmark workload, from the oracle alone:

* fullsize_z_n40000.npy: the observations Z = L w (float64, generation order),
  L the dense FP64 Cholesky factor of Sigma(theta) for the locations in
  generation order and w = synth.standard_normal(n, seed=z_seed): the
  workload's data drawn from the model, as its configuration states;
* fullsize_loglik_n40000.json: the exact l(theta) (Eq. 1.2) of that Z and
  its two terms log|Sigma| and Z' Sigma^-1 Z, from the same factor.

Workload: n = 40,000 locations of synth.jittered_grid(40000, seed=1) in
generation order, theta = (sigma2 1, beta 0.1, nu 0.5).  Exact l does not
depend on the order of the locations (Sec. 3), so the values check the TLR
likelihood under any ordering and at any accuracy eps.  The oracle builds
the dense 40,000 x 40,000 covariance (12.8 GB) and factors it with LAPACK,
single-threaded (a threaded OpenBLAS build of this size of problem crashed);
about fifteen minutes and 26 GB of host memory.

Usage: python tests/golden/make_fullsize_loglik.py
"""
import json
import os
import sys
import time

os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")  # before numpy loads OpenBLAS

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import synth  # noqa: E402

N, THETA, LOC_SEED, Z_SEED = 40000, (1.0, 0.1, 0.5), 1, 2


def main():
    here = os.path.dirname(os.path.abspath(__file__))
    t0 = time.time()
    xy = synth.jittered_grid(N, seed=LOC_SEED)
    w = synth.standard_normal(N, seed=Z_SEED)
    sigma = oracle.cov_matrix(xy, THETA)
    L = np.linalg.cholesky(sigma)
    del sigma
    z = L @ w
    r = oracle.loglik_from_factor(L, z)
    np.save(os.path.join(here, "fullsize_z_n40000.npy"), z)
    out = {"n": N, "theta": list(THETA), "loc_seed": LOC_SEED, "z_seed": Z_SEED,
           "z": "fullsize_z_n40000.npy: Z = L w, L = chol(Sigma(theta)) in generation order, "
                "w = synth.standard_normal(n, seed=z_seed)",
           "order": "generation",
           "loglik": r["loglik"], "logdet": r["logdet"], "quad": r["quad"],
           "w_sumsq": float(w @ w),
           "source": "oracle.cov_matrix + LAPACK Cholesky + oracle.loglik_from_factor (dense FP64)",
           "seconds": round(time.time() - t0, 1)}
    with open(os.path.join(here, "fullsize_loglik_n40000.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
