"""CPU FP64 oracle for the TLR Matern log-likelihood of arXiv 2402.09356.

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
cpu_baseline / reference leg of bench.py may import, call or execute anything
in this package.  The product path (paper_2402_09356_gb300) never imports it,
and this package never imports the product: the two share no code; the only
module both use is `synth`, the seeded input generator, which holds none of the
method's arithmetic.

What it computes, each in the plainest form that follows the paper:
  covariance  K_nu by quadrature of its integral representation and the
              Matern covariance of Eq. 4.2 (matern_ref.c); dense Sigma (Eq. 1.1).
  ordering    identity, random, Morton, Hilbert, KD-tree and max-min (Sec. 3).
  likelihood  exact Eq. 1.2 by dense Cholesky (LAPACK) and a triangular solve.
  ranks       SVD rank of every off-diagonal tile at accuracy eps * sigma2
              (Sec. 2-3) and the memory accounting of Table 1.

Every function is pinned in tests/test_oracle_*.py against facts the paper
and the mathematics fix (closed forms, the Hilbert figure, Table 1's dense
column, brute-force determinants, invariances).
"""
from ._clib import build  # noqa: F401
from .covariance import besselk, besselk_scaled, matern, cov_matrix, cov_block, permute_xy  # noqa: F401
from .ordering import (IDENTITY, RANDOM, MORTON, HILBERT, KDTREE, MAXMIN, NAMES,  # noqa: F401
                       quantize, dequantize, morton_code, hilbert_code, random_keys,
                       sort_codes, kdtree_perm, maxmin_perm, order, decode_xy)
from .likelihood import (loglik_dense, loglik_from_cov, loglik_from_factor, simulate_z, tile_bounds,  # noqa: F401
                         tile_singular_values, ranks_from_singular_values, tile_ranks,
                         factor_tile_ranks, dense_offdiag_bytes, tlr_offdiag_bytes)
