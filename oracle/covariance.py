"""Oracle: K_nu and the Matern covariance (Eq. 4.2, Eq. 1.1).  Test infrastructure only.

The arithmetic lives in matern_ref.c (trapezoid quadrature of the integral
representation of K_nu); these wrappers only marshal numpy arrays.
"""
from __future__ import annotations

import numpy as np

from ._clib import lib, ptr


def besselk(nu: float, x) -> np.ndarray:
    """K_nu(x) for x > 0 (integral representation, trapezoid rule)."""
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    f = lib().oracle_besselk
    return np.array([f(float(nu), float(v)) for v in x])


def besselk_scaled(nu: float, x) -> np.ndarray:
    """exp(x) K_nu(x)."""
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    f = lib().oracle_besselk_scaled
    return np.array([f(float(nu), float(v)) for v in x])


def matern(d, theta) -> np.ndarray:
    """C(d; sigma2, beta, nu) of Eq. 4.2 for an array of distances d >= 0."""
    s2, beta, nu = (float(t) for t in theta)
    d = np.ascontiguousarray(np.atleast_1d(np.asarray(d, dtype=np.float64)))
    out = np.empty_like(d)
    lib().oracle_matern_vec(d.size, ptr(d), s2, beta, nu, ptr(out))
    return out


def cov_matrix(xy: np.ndarray, theta) -> np.ndarray:
    """Dense Sigma_ij = C(||s_i - s_j||) (Eq. 1.1) for SoA locations xy (length 2n)."""
    xy = np.ascontiguousarray(xy, dtype=np.float64)
    n = xy.size // 2
    out = np.empty((n, n), dtype=np.float64)
    s2, beta, nu = (float(t) for t in theta)
    lib().oracle_matern_matrix(n, ptr(xy), s2, beta, nu, ptr(out))
    return out


def cov_block(rxy: np.ndarray, cxy: np.ndarray, theta) -> np.ndarray:
    """Covariance block between row locations rxy and column locations cxy (both SoA)."""
    rxy = np.ascontiguousarray(rxy, dtype=np.float64)
    cxy = np.ascontiguousarray(cxy, dtype=np.float64)
    nr, nc = rxy.size // 2, cxy.size // 2
    out = np.empty((nr, nc), dtype=np.float64)
    s2, beta, nu = (float(t) for t in theta)
    lib().oracle_matern_block(nr, ptr(rxy), nc, ptr(cxy), s2, beta, nu, ptr(out))
    return out


def permute_xy(xy: np.ndarray, perm: np.ndarray) -> np.ndarray:
    """SoA locations reordered so that position k holds original point perm[k]."""
    n = xy.size // 2
    return np.concatenate([xy[:n][perm], xy[n:][perm]])
