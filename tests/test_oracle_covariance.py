"""Pins for the oracle's K_nu and Matern covariance (Eq. 4.2, Eq. 1.1).

The oracle evaluates K_nu by quadrature of its integral representation.  It is
checked against facts fixed independently of that formula: the closed forms
for half-integer orders, the three-term recurrence and the Wronskian (DLMF
10.29.1, 10.28.2), the small-argument limit, and scipy's K_nu as a library
comparator.  A dropped term, a wrong exponent or a wrong scale fails one of them.
"""
import math

import numpy as np
import pytest
from scipy import special

import oracle
import synth

XS = np.concatenate([np.logspace(-6, 0, 13), np.linspace(1.5, 60.0, 12), [100.0, 300.0, 700.0]])


def rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)) / np.abs(np.asarray(b))


def test_besselk_half_integer_closed_forms():
    # K_{1/2}, K_{3/2}, K_{5/2} in elementary form (DLMF 10.47.9 with 10.49.12)
    pref = np.sqrt(np.pi / (2 * XS))
    ks = oracle.besselk_scaled  # exp(x) K_nu(x): no underflow at x = 700
    assert rel(ks(0.5, XS), pref).max() < 1e-13
    assert rel(ks(1.5, XS), pref * (1 + 1 / XS)).max() < 1e-13
    assert rel(ks(2.5, XS), pref * (1 + 3 / XS + 3 / XS ** 2)).max() < 1e-13


@pytest.mark.parametrize("nu", [0.3, 0.75, 1.2, 2.0, 3.4])
def test_besselk_recurrence(nu):
    # K_{nu+1}(x) = K_{nu-1}(x) + (2 nu / x) K_nu(x)
    x = XS[XS < 200]
    lhs = oracle.besselk_scaled(nu + 1, x)
    rhs = oracle.besselk_scaled(nu - 1, x) + 2 * nu / x * oracle.besselk_scaled(nu, x)
    assert rel(rhs, lhs).max() < 1e-13


@pytest.mark.parametrize("nu", [0.1, 0.5, 1.0, 1.7, 2.5])
def test_besselk_wronskian(nu):
    # I_nu K_{nu+1} + I_{nu+1} K_nu = 1/x, with I_nu from scipy (scaled forms)
    x = np.logspace(-3, 2, 21)
    w = special.ive(nu, x) * oracle.besselk_scaled(nu + 1, x) + \
        special.ive(nu + 1, x) * oracle.besselk_scaled(nu, x)
    assert rel(w, 1 / x).max() < 1e-13


def test_besselk_against_scipy():
    rng = np.random.default_rng(0)
    for nu in rng.uniform(0.05, 6.0, 12):
        v = oracle.besselk_scaled(nu, XS)
        assert rel(v, special.kve(nu, XS)).max() < 2e-13, nu


def test_besselk_small_argument_limit():
    # K_nu(x) ~ Gamma(nu) 2^(nu-1) x^-nu as x -> 0 (nu > 0)
    for nu in (0.5, 1.0, 2.5):
        x = 1e-7
        lim = math.gamma(nu) * 2 ** (nu - 1) * x ** (-nu)
        assert abs(oracle.besselk(nu, x)[0] / lim - 1) < 1e-5


def test_matern_closed_forms():
    d = np.linspace(0.0, 1.5, 61)
    for s2, beta in ((1.0, 0.1), (2.5, 0.03), (0.7, 0.3)):
        x = d / beta
        assert rel(oracle.matern(d, (s2, beta, 0.5)), s2 * np.exp(-x)).max() < 1e-13
        assert rel(oracle.matern(d, (s2, beta, 1.5)), s2 * (1 + x) * np.exp(-x)).max() < 1e-13
        assert rel(oracle.matern(d, (s2, beta, 2.5)),
                   s2 * (1 + x + x * x / 3) * np.exp(-x)).max() < 1e-13


def test_matern_zero_distance_and_monotone():
    for nu in (0.4, 1.0, 2.2):
        c = oracle.matern(np.array([0.0, 1e-13, 1e-3, 1e-2, 0.1, 0.5]), (1.7, 0.1, nu))
        assert c[0] == 1.7                       # no nugget: C(0) = sigma2
        assert abs(c[1] - 1.7) < 1e-9            # continuous at 0
        assert np.all(np.diff(c[1:]) < 0)        # decreasing in d


def test_cov_matrix_symmetric_spd():
    xy = synth.jittered_grid(300, seed=11)
    for theta in ((1.0, 0.1, 0.5), (1.3, 0.05, 1.0), (0.8, 0.3, 1.5)):
        s = oracle.cov_matrix(xy, theta)
        assert np.array_equal(s, s.T)
        assert np.all(np.diag(s) == theta[0])
        assert np.all(s > 0) and np.all(s <= theta[0])
        np.linalg.cholesky(s)                    # positive definite


def test_cov_block_matches_matrix():
    xy = synth.jittered_grid(120, seed=5)
    n = 120
    s = oracle.cov_matrix(xy, (1.0, 0.1, 1.3))
    r = np.r_[xy[:n][10:40], xy[n:][10:40]]
    c = np.r_[xy[:n][70:120], xy[n:][70:120]]
    b = oracle.cov_block(r, c, (1.0, 0.1, 1.3))
    assert np.array_equal(b, s[10:40, 70:120])
