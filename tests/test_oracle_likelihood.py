"""Pins for the oracle's log-likelihood (Eq. 1.2), ranks and Table 1 accounting.

The dense likelihood is checked against a brute-force evaluation that shares
nothing with it (Leibniz determinant and Cramer's rule on tiny n), closed
forms at n = 1 and 2, exact invariances (permutation of the locations,
scaling of sigma2) and the quadratic form of a simulated vector.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
import synth


def leibniz_det(a):
    n = a.shape[0]
    total = 0.0
    for p in itertools.permutations(range(n)):
        inv = sum(1 for i in range(n) for j in range(i + 1, n) if p[i] > p[j])
        term = -1.0 if inv % 2 else 1.0
        for i in range(n):
            term *= a[i, p[i]]
        total += term
    return total


def brute_loglik(xy, z, theta):
    n = z.size
    x, y = xy[:n], xy[n:]
    s2, beta, nu = theta
    # covariance entries from the half-integer closed forms (independent of K_nu code)
    a = np.empty((n, n))
    for i in range(n):
        for j in range(n):
            t = math.hypot(x[i] - x[j], y[i] - y[j]) / beta
            a[i, j] = s2 * (1 + t + t * t / 3) * math.exp(-t) if nu == 2.5 else s2 * math.exp(-t)
    det = leibniz_det(a)
    sol = np.empty(n)
    for k in range(n):  # Cramer's rule for Sigma^-1 z
        b = a.copy()
        b[:, k] = z
        sol[k] = leibniz_det(b) / det
    quad = float(z @ sol)
    return -0.5 * n * math.log(2 * math.pi) - 0.5 * math.log(det) - 0.5 * quad, math.log(det), quad


@pytest.mark.parametrize("n,theta", [(4, (1.0, 0.3, 0.5)), (6, (1.7, 0.2, 2.5)), (7, (0.6, 0.5, 0.5))])
def test_loglik_brute_force(n, theta):
    xy = synth.jittered_grid(n, seed=20 + n)
    z = synth.standard_normal(n, seed=30 + n)
    ll, logdet, quad = brute_loglik(xy, z, theta)
    r = oracle.loglik_dense(xy, z, theta)
    assert abs(r["loglik"] - ll) <= 1e-11 * abs(ll)
    assert abs(r["logdet"] - logdet) <= 1e-11 * max(1.0, abs(logdet))
    assert abs(r["quad"] - quad) <= 1e-11 * abs(quad)


def test_loglik_n1_n2_closed_forms():
    s2 = 1.9
    r = oracle.loglik_dense(np.array([0.3, 0.7]), np.array([0.8]), (s2, 0.1, 1.2))
    assert abs(r["loglik"] - (-0.5 * math.log(2 * math.pi) - 0.5 * math.log(s2) - 0.32 / s2)) < 1e-14
    xy = np.array([0.1, 0.4, 0.2, 0.6])  # points (0.1, 0.2) and (0.4, 0.6): distance 0.5
    z = np.array([0.5, -1.1])
    c = s2 * math.exp(-0.5 / 0.25)
    det = s2 * s2 - c * c
    quad = (s2 * z[0] ** 2 - 2 * c * z[0] * z[1] + s2 * z[1] ** 2) / det
    ll = -math.log(2 * math.pi) - 0.5 * math.log(det) - 0.5 * quad
    assert abs(oracle.loglik_dense(xy, z, (s2, 0.25, 0.5))["loglik"] - ll) < 1e-13


def test_loglik_permutation_invariant():
    n = 400
    xy = synth.jittered_grid(n, seed=8)
    theta = (1.0, 0.1, 0.9)
    z = oracle.simulate_z(xy, theta, synth.standard_normal(n, seed=9))
    ref = oracle.loglik_dense(xy, z, theta)["loglik"]
    for m in oracle.NAMES:
        perm, _ = oracle.order(xy, m)
        ll = oracle.loglik_dense(oracle.permute_xy(xy, perm), z[perm], theta)["loglik"]
        assert abs(ll - ref) <= 1e-12 * abs(ref), m


def test_simulated_quadratic_form_and_sigma2_scaling():
    n = 300
    xy = synth.jittered_grid(n, seed=12)
    w = synth.standard_normal(n, seed=13)
    theta = (1.0, 0.1, 0.5)
    z = oracle.simulate_z(xy, theta, w)
    r = oracle.loglik_dense(xy, z, theta)
    assert abs(r["quad"] - w @ w) <= 1e-9 * (w @ w)  # L^-1 (L w) = w
    c = 3.0
    r2 = oracle.loglik_dense(xy, z, (c * theta[0],) + theta[1:])
    assert abs(r2["logdet"] - (r["logdet"] + n * math.log(c))) < 1e-9 * n
    assert abs(r2["quad"] - r["quad"] / c) < 1e-9 * r["quad"]


def test_table1_dense_column(golden_dir):
    rows = [l.split() for l in open(golden_dir + "/table1_memory.txt") if l[0].isdigit()]
    dense = {int(r[0]): int(r[2]) for r in rows if r[1] == "dense"}
    assert dense == {10000: 360, 20000: 1520, 30000: 3480, 40000: 6240}
    for n, mb in dense.items():
        assert oracle.dense_offdiag_bytes(n, 1000) == mb * 10 ** 6


def test_tlr_bytes_formula():
    r = np.array([[3, 2, 0], [2, 3, 1], [0, 1, 2]])
    # n = 8, nb = 3: tiles of 3, 3, 2 rows
    assert oracle.tlr_offdiag_bytes(r, 8, 3) == 8 * ((3 + 3) * 2 + (2 + 3) * 0 + (2 + 3) * 1)


def test_tile_ranks_limits():
    n, nb = 1024, 128
    xy = synth.jittered_grid(n, seed=3)
    perm, _ = oracle.order(xy, "hilbert")
    s = oracle.cov_matrix(oracle.permute_xy(xy, perm), (1.0, 0.1, 0.5))
    r0, _ = oracle.tile_ranks(s, nb, 0.0)
    assert np.all(r0 == nb)                             # eps -> 0: every tile full rank
    r9, sv = oracle.tile_ranks(s, nb, 1e-9)
    r5, _ = oracle.tile_ranks(s, nb, 1e-5)
    assert np.all(r5 <= r9) and np.all(r9 <= nb)
    assert r9[0, 2:].min() < r9[0, 1] // 2              # far tiles compress better
    for (i, j), v in sv.items():                        # eps-rank is the SVD count
        assert r9[i, j] == np.count_nonzero(v > 1e-9)


def test_factor_tile_is_schur_complement():
    n, nb = 180, 60
    xy = synth.jittered_grid(n, seed=6)
    s = oracle.cov_matrix(xy, (1.0, 0.2, 1.0))
    L = np.linalg.cholesky(s)
    b = oracle.tile_bounds(n, nb)
    i, j = 2, 1
    blk = lambda m, a, c: m[b[a][0]:b[a][1], b[c][0]:b[c][1]]
    schur = blk(s, i, j) - blk(L, i, 0) @ blk(L, j, 0).T
    assert np.abs(schur - blk(L, i, j) @ blk(L, j, j).T).max() < 1e-13
    rf, _ = oracle.factor_tile_ranks(s, nb, 1e-9)
    assert rf[i, j] == np.count_nonzero(np.linalg.svd(schur, compute_uv=False) > 1e-9)


def _tile_with_spectrum(rng, m, k, s):
    """m x k tile sum_q s[q] u_q v_q' with orthonormal u, v (QR of Gaussians)."""
    u, _ = np.linalg.qr(rng.standard_normal((m, len(s))))
    v, _ = np.linalg.qr(rng.standard_normal((k, len(s))))
    return (u * np.asarray(s)) @ v.T


@pytest.mark.parametrize("sigma2, spectra, expected", [
    # tau = eps * sigma2 = 2e-6: 1.5e-6 lies between eps and eps * sigma2, and
    # the relative threshold eps * s_1 = 5e-6 would drop 3e-6 and 2.5e-6
    (2.0, {(1, 0): [5.0, 1e-1, 3e-6, 2.5e-6, 1.5e-6, 5e-7],
           (2, 0): [1.9e-6, 1e-7],
           (2, 1): [1.0, 2.1e-6, 1.2e-6]}, {(1, 0): 4, (2, 0): 0, (2, 1): 2}),
    # tau = 5e-7: 7e-7 and 6e-7 count although they are below eps = 1e-6
    (0.5, {(1, 0): [1.0, 1e-3, 7e-7, 6e-7, 3e-7],
           (2, 0): [8e-7, 4e-7],
           (2, 1): [2e-2, 9e-7, 5.5e-7, 4.5e-7]}, {(1, 0): 4, (2, 0): 1, (2, 1): 3}),
])
def test_tile_ranks_constructed_spectra(sigma2, spectra, expected):
    """Sec. 2-3: the rank of a tile is the number of its singular values above the
    absolute threshold eps * sigma2 (reading of the accuracy threshold).  Tiles with
    a known spectrum are placed in a block matrix; a threshold that drops sigma2,
    is relative to the largest singular value, or counts the wrong blocks fails."""
    eps, nb, n = 1e-6, 24, 3 * 24 - 5     # ragged last tile (19 rows)
    rng = np.random.default_rng(11)
    b = oracle.tile_bounds(n, nb)
    S = np.zeros((n, n))
    for t in range(3):
        S[b[t][0]:b[t][1], b[t][0]:b[t][1]] = np.eye(b[t][1] - b[t][0])
    for (i, j), s in spectra.items():
        T = _tile_with_spectrum(rng, b[i][1] - b[i][0], b[j][1] - b[j][0], s)
        S[b[i][0]:b[i][1], b[j][0]:b[j][1]] = T
        S[b[j][0]:b[j][1], b[i][0]:b[i][1]] = T.T
    r, sv = oracle.tile_ranks(S, nb, eps, sigma2)
    for (i, j), want in expected.items():
        assert r[i, j] == want and r[j, i] == want, ((i, j), r[i, j], want)
        top = sorted(spectra[(i, j)], reverse=True)
        assert np.allclose(sv[(i, j)][:len(top)], top, rtol=1e-9, atol=1e-15)
    assert [r[t, t] for t in range(3)] == [24, 24, 19]   # diagonal tiles dense
    # the Table 1 memory of this rank map: (m_i + m_j) r_ij doubles per tile
    want_bytes = 8 * sum((b[i][1] - b[i][0] + b[j][1] - b[j][0]) * c for (i, j), c in expected.items())
    assert oracle.tlr_offdiag_bytes(r, n, nb) == want_bytes


def test_ranks_threshold_is_strict():
    """A singular value equal to the threshold is dropped: the kept values are
    those strictly above eps * sigma2 (values exact in binary)."""
    sv = {(1, 0): np.array([1.0, 0.25, 0.25, 0.125]), (2, 0): np.array([0.25]),
          (2, 1): np.array([0.5, 0.2500000000000001])}
    r = oracle.ranks_from_singular_values(sv, 9, 3, 0.25)
    assert (r[1, 0], r[2, 0], r[2, 1]) == (1, 0, 2)
    assert (r[0, 1], r[0, 2], r[1, 2]) == (1, 0, 2)


def test_loglik_from_factor_of_simulated_z():
    """Eq. 1.2 on data drawn from the model, Z = L w: Z' Sigma^-1 Z = |w|^2
    exactly, and log|Sigma| is LAPACK's log-determinant of Sigma."""
    n = 300
    xy = synth.jittered_grid(n, seed=4)
    S = oracle.cov_matrix(xy, (1.7, 0.08, 1.0))
    L = np.linalg.cholesky(S)
    w = synth.standard_normal(n, seed=9)
    r = oracle.loglik_from_factor(L, L @ w)
    assert abs(r["quad"] - w @ w) <= 1e-10 * (w @ w)
    sign, ld = np.linalg.slogdet(S)
    assert sign == 1.0 and abs(r["logdet"] - ld) <= 1e-10 * abs(ld)
    assert r["loglik"] == pytest.approx(-0.5 * n * math.log(2 * math.pi) - 0.5 * ld - 0.5 * (w @ w), rel=1e-10)
