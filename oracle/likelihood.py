"""Oracle: the exact Gaussian log-likelihood (Eq. 1.2), data simulation, and the
reference tile ranks of the TLR representation (Sec. 2, Sec. 3, Table 1).
Test infrastructure only.

* loglik_dense: l = -n/2 log(2 pi) - 1/2 log|Sigma| - 1/2 Z' Sigma^-1 Z with
  Sigma built by the oracle's own Matern code, factored by LAPACK's Cholesky
  (a library primitive), log|Sigma| = 2 sum log L_ii and Z' Sigma^-1 Z = |L^-1 Z|^2
  (loglik_from_factor: the same two terms from a factor already computed).
* simulate_z: Z = L w with L the dense Cholesky factor of Sigma(theta) in the
  order the locations are given (generation order for the workloads).
* tile_ranks: for every off-diagonal tile of Sigma the number of singular
  values above eps * sigma2 (Sec. 3: the accuracy threshold decides how many
  singular values are kept; the threshold is absolute and scales with sigma2).
* factor_tile_ranks: the same count for the tiles L_ij L_jj' of the exact
  factor, i.e. for the off-diagonal tiles of the Schur complement at the step
  where column j is factored (the quantity a right- or left-looking TLR
  Cholesky truncates before its triangular solve).
* Memory accounting as in Table 1: dense off-diagonal storage is the number
  of lower off-diagonal tiles times nb^2 doubles; TLR storage is
  (m_i + m_j) * r_ij doubles per tile (U is m_i x r, V is m_j x r).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg

from .covariance import cov_matrix


def loglik_from_factor(L: np.ndarray, z: np.ndarray) -> dict:
    """Eq. 1.2 from the lower Cholesky factor L of Sigma (Sigma = L L'):
    log|Sigma| = 2 sum log L_ii, Z' Sigma^-1 Z = |L^-1 Z|^2."""
    n = L.shape[0]
    logdet = 2.0 * float(np.sum(np.log(np.diag(L))))
    y = scipy.linalg.solve_triangular(L, z, lower=True)
    quad = float(y @ y)
    ll = -0.5 * n * math.log(2.0 * math.pi) - 0.5 * logdet - 0.5 * quad
    return {"loglik": ll, "logdet": logdet, "quad": quad}


def loglik_from_cov(sigma: np.ndarray, z: np.ndarray) -> dict:
    return loglik_from_factor(np.linalg.cholesky(sigma), z)


def loglik_dense(xy: np.ndarray, z: np.ndarray, theta) -> dict:
    """Exact Eq. 1.2 for SoA locations xy and observations z in the same order."""
    return loglik_from_cov(cov_matrix(xy, theta), np.asarray(z, dtype=np.float64))


def simulate_z(xy: np.ndarray, theta, w: np.ndarray) -> np.ndarray:
    """Z = L w, L the Cholesky factor of Sigma(theta) for the given location order."""
    L = np.linalg.cholesky(cov_matrix(xy, theta))
    return L @ np.asarray(w, dtype=np.float64)


def tile_bounds(n: int, nb: int):
    nt = (n + nb - 1) // nb
    return [(t * nb, min(n, (t + 1) * nb)) for t in range(nt)]


def tile_singular_values(sigma: np.ndarray, nb: int) -> dict:
    """Singular values (descending) of every lower off-diagonal tile, keyed (i, j)."""
    b = tile_bounds(sigma.shape[0], nb)
    out = {}
    for i in range(len(b)):
        for j in range(i):
            blk = sigma[b[i][0]:b[i][1], b[j][0]:b[j][1]]
            out[(i, j)] = np.linalg.svd(blk, compute_uv=False)
    return out


def ranks_from_singular_values(sv: dict, n: int, nb: int, thresh: float) -> np.ndarray:
    b = tile_bounds(n, nb)
    nt = len(b)
    r = np.zeros((nt, nt), dtype=np.int64)
    for i in range(nt):
        r[i, i] = b[i][1] - b[i][0]          # diagonal tiles stay dense (full rank)
    for (i, j), s in sv.items():
        r[i, j] = int(np.count_nonzero(s > thresh))
        r[j, i] = r[i, j]
    return r


def tile_ranks(sigma: np.ndarray, nb: int, eps: float, sigma2: float = 1.0):
    """Rank map of the TLR compression of Sigma at absolute accuracy eps * sigma2."""
    sv = tile_singular_values(sigma, nb)
    return ranks_from_singular_values(sv, sigma.shape[0], nb, eps * sigma2), sv


def factor_tile_ranks(sigma: np.ndarray, nb: int, eps: float, sigma2: float = 1.0):
    """Rank map of the tiles L_ij L_jj' (i > j) of the exact Cholesky factor."""
    L = np.linalg.cholesky(sigma)
    b = tile_bounds(sigma.shape[0], nb)
    sv = {}
    for i in range(len(b)):
        for j in range(i):
            lij = L[b[i][0]:b[i][1], b[j][0]:b[j][1]]
            ljj = L[b[j][0]:b[j][1], b[j][0]:b[j][1]]
            sv[(i, j)] = np.linalg.svd(lij @ ljj.T, compute_uv=False)
    return ranks_from_singular_values(sv, sigma.shape[0], nb, eps * sigma2), sv


def dense_offdiag_bytes(n: int, nb: int) -> int:
    """Table 1 "Dense": lower off-diagonal tiles x nb^2 x 8 bytes (full tiles)."""
    nt = (n + nb - 1) // nb
    return nt * (nt - 1) // 2 * nb * nb * 8


def tlr_offdiag_bytes(ranks: np.ndarray, n: int, nb: int) -> int:
    """Table 1 TLR storage: U (m_i x r) plus V (m_j x r) doubles per off-diagonal tile."""
    b = tile_bounds(n, nb)
    total = 0
    for i in range(len(b)):
        for j in range(i):
            total += ((b[i][1] - b[i][0]) + (b[j][1] - b[j][0])) * int(ranks[i, j]) * 8
    return total
