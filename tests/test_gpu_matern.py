"""Device K_nu / Matern covariance (Eq. 4.2) and tile generation (Eq. 1.1)
against the oracle: entries within 1e-12 relative (absolute floor 1e-300)."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL = 1e-12


def close(a, b):
    err = np.abs(a - b)
    return np.all(err <= TOL * np.abs(b) + 1e-300), float(np.max(err / np.maximum(np.abs(b), 1e-300)))


@pytest.mark.parametrize("nu", [0.05, 0.3, 0.5, 0.77, 1.0, 1.5, 1.9999, 2.2, 2.5, 3.7, 6.3])
def test_matern_entries(ctx, nu):
    import torch
    import paper_2402_09356_gb300 as tlr
    beta = 0.1
    x = np.concatenate([np.logspace(-9, 3, 700), np.linspace(0.01, 40, 500),
                        [1.999999, 2.0, 2.000001, 24.99999, 25.0, 25.00001, 700.0, 760.0, 900.0]])
    d = np.concatenate([[0.0], x * beta])
    theta = (1.3, beta, nu)
    dev = tlr.tlr_matern(ctx, torch.from_numpy(d).cuda(), theta).cpu().numpy()
    ok, worst = close(dev, oracle.matern(d, theta))
    assert ok, worst
    assert dev[0] == 1.3


def test_matern_small_mu(ctx):
    # nu within 1e-9 of an integer exercises the small-|mu| branch of Temme's constants
    import torch
    import paper_2402_09356_gb300 as tlr
    d = np.logspace(-4, 0.5, 300)
    for nu in (1.0 + 1e-9, 2.0 - 3e-8, 1e-3 + 1.0, 0.9999):
        dev = tlr.tlr_matern(ctx, torch.from_numpy(d).cuda(), (1.0, 0.05, nu)).cpu().numpy()
        ok, worst = close(dev, oracle.matern(d, (1.0, 0.05, nu)))
        assert ok, (nu, worst)


@pytest.mark.parametrize("n,nb,theta,order", [(1600, 200, (1.0, 0.1, 0.5), "morton"),
                                              (1000, 96, (1.3, 0.05, 1.7), "hilbert"),
                                              (37, 16, (0.8, 0.3, 2.5), "kdtree")])
def test_generate_tiles(ctx, n, nb, theta, order):
    import torch
    import paper_2402_09356_gb300 as tlr
    xy = synth.jittered_grid(n, seed=2)
    perm, _ = oracle.order(xy, order)
    xyp = oracle.permute_xy(xy, perm)
    tiles = tlr.tlr_generate(ctx, torch.from_numpy(xyp).cuda(), nb, theta).cpu().numpy()
    S = oracle.cov_matrix(xyp, theta)
    nt = (n + nb - 1) // nb
    for i in range(nt):
        for j in range(i + 1):
            t = tiles[(i * (i + 1) // 2 + j) * nb * nb:][:nb * nb].reshape(nb, nb).T  # column major
            mi, mj = min(nb, n - i * nb), min(nb, n - j * nb)
            ok, worst = close(t[:mi, :mj], S[i * nb:i * nb + mi, j * nb:j * nb + mj])
            assert ok, (i, j, worst)
            assert np.all(t[mi:, :] == 0) and np.all(t[:, mj:] == 0)
