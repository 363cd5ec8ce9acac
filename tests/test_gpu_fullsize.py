"""Parity at the full benchmark size (n = 40,000, tile 800, the bench's launch
configuration), where the dense oracle likelihood is too slow to run in a test:

* sampled tiles of L L' against the oracle's covariance tiles.  In the
  left-looking factorisation tile (i, j) of L L' equals Sigma_ij minus the one
  truncation made when T_ij = Sigma_ij - sum_k L_ik L_jk' was compressed
  (Sec. 2: singular values <= eps sigma2 dropped), so its spectral-norm error
  is at most eps sigma2 (small slack for the randomised range finder and
  rounding); diagonal tiles are exact up to the covariance entries' own
  1e-12 relative accuracy (spectral norm <= nb 1e-12 sigma2) and rounding.
* the log-determinant equals 2 sum log diag(L_jj) read back from the factor.
* exact l is invariant under any permutation of the locations (Sec. 3): the
  Hilbert and Morton results agree within twice the 10 eps |l| bound each
  meets, and the mixed path stays within 1e-6 |l| of the FP64 path.
* l, log|Sigma| and Z' Sigma^-1 Z of both paths, at eps = 1e-7 and 1e-9,
  each within 10 eps of its own magnitude from the exact values the dense
  oracle computed once for this workload with the data drawn from the model,
  Z = L w (tests/golden/fullsize_loglik_n40000.json and fullsize_z_n40000.npy,
  written by make_fullsize_loglik.py).
"""
import json
import os

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

N, NB, EPS, THETA = 40000, 800, 1e-7, (1.0, 0.1, 0.5)
SAMPLED = [(0, 0), (1, 0), (2, 1), (25, 24), (30, 10), (49, 0), (49, 48)]


def golden_z(golden_dir):
    return np.load(os.path.join(golden_dir, "fullsize_z_n40000.npy"))


def factor(ctx, order, precision, eps=EPS, z=None):
    """TLR factor of the workload; z (generation order) defaults to white noise,
    which the tests that only look at the factor use."""
    import torch
    import paper_2402_09356_gb300 as tlr
    xy = synth.jittered_grid(N, seed=1)
    w = synth.standard_normal(N, seed=2) if z is None else z
    xy_d = torch.from_numpy(xy).cuda()
    xyo = torch.empty_like(xy_d)
    perm = tlr.tlr_order(ctx, xy_d, order, xy_out=xyo)
    zo = tlr.tlr_gather(ctx, perm, torch.from_numpy(np.ascontiguousarray(w)).cuda())
    L = tlr.TlrMatrix(ctx, N, NB)
    r = tlr.tlr_loglik(L, xyo, zo, THETA, tlr.Options(nb=NB, eps=eps, precision=precision))
    return L, r, xyo.cpu().numpy()


class Tiles:
    """Factor tiles read back to the host: L_jj dense, L_ij = U_ij V_ij'."""

    def __init__(self, L):
        import paper_2402_09356_gb300 as tlr
        self.L, self.tlr, self.cache = L, tlr, {}

    def get(self, i, j):
        if (i, j) not in self.cache:
            t = self.tlr.tlr_mat_tile(self.L, i, j)
            self.cache[(i, j)] = t.cpu().numpy() if i == j else (t[0].cpu().numpy(), t[1].cpu().numpy())
        return self.cache[(i, j)]

    def llt(self, i, j):
        """Tile (i, j), i >= j, of L L'."""
        acc = 0.0
        for k in range(j):
            Ui, Vi = self.get(i, k)
            Uj, Vj = self.get(j, k)
            acc = acc + Ui @ ((Vi.T @ Vj) @ Uj.T)
        Ljj = self.get(j, j)
        if i == j:
            return acc + Ljj @ Ljj.T
        Ui, Vi = self.get(i, j)
        return acc + Ui @ (Vi.T @ Ljj.T)


def block_xy(xy, t):
    n = xy.size // 2
    a, b = t * NB, min(n, (t + 1) * NB)
    return np.concatenate([xy[:n][a:b], xy[n:][a:b]])


@pytest.fixture(scope="module")
def hilbert64(ctx):
    import paper_2402_09356_gb300 as tlr
    L, r, xyo = factor(ctx, "hilbert", tlr.TLR_PREC_FP64)
    yield L, r, xyo
    L.close()


def test_fullsize_sampled_tiles_of_llt(ctx, hilbert64):
    L, r, xyo = hilbert64
    tiles = Tiles(L)
    for i, j in SAMPLED:
        S = oracle.cov_block(block_xy(xyo, i), block_xy(xyo, j), THETA)
        err = np.linalg.norm(tiles.llt(i, j) - S, 2)
        if i == j:
            assert err <= 2.5 * NB * 1e-12 * THETA[0], (i, j, err)
        else:
            assert err <= 1.5 * EPS * THETA[0], (i, j, err)


def test_fullsize_logdet_from_diagonal(ctx, hilbert64):
    L, r, _ = hilbert64
    tiles = Tiles(L)
    nt = (N + NB - 1) // NB
    s = sum(np.log(np.diag(tiles.get(t, t))).sum() for t in range(nt))
    assert abs(2 * s - r["logdet"]) <= 1e-11 * abs(r["logdet"])


def test_fullsize_ordering_invariance_and_mixed(ctx, golden_dir):
    import paper_2402_09356_gb300 as tlr
    z = golden_z(golden_dir)
    L6, r64, _ = factor(ctx, "hilbert", tlr.TLR_PREC_FP64, z=z)
    L6.close()
    Lm, rm, _ = factor(ctx, "morton", tlr.TLR_PREC_FP64, z=z)
    Lm.close()
    Lt, rt, _ = factor(ctx, "hilbert", tlr.TLR_PREC_TENSOR, z=z)
    Lt.close()
    Lx, rx, xyo = factor(ctx, "hilbert", tlr.TLR_PREC_MIXED, z=z)
    ref = abs(r64["loglik"])
    assert abs(rm["loglik"] - r64["loglik"]) <= 20 * EPS * ref, (rm["loglik"], r64["loglik"])
    assert abs(rx["loglik"] - r64["loglik"]) <= 1e-6 * ref, (rx["loglik"], r64["loglik"])
    assert abs(rt["loglik"] - r64["loglik"]) <= 1e-6 * ref, (rt["loglik"], r64["loglik"])
    # the mixed factor meets the same tile bound
    tiles = Tiles(Lx)
    for i, j in SAMPLED[1:4]:
        S = oracle.cov_block(block_xy(xyo, i), block_xy(xyo, j), THETA)
        assert np.linalg.norm(tiles.llt(i, j) - S, 2) <= 1.5 * EPS * THETA[0]
    Lx.close()


@pytest.mark.parametrize("eps", [1e-7, 1e-9])
@pytest.mark.parametrize("precision", ["fp64", "mixed", "tensor"])
def test_fullsize_loglik_terms_against_exact_oracle(ctx, golden_dir, eps, precision):
    """Eq. 1.2 term by term at full size: l, log|Sigma| and Z' Sigma^-1 Z each
    within 10 eps of its own magnitude from the dense oracle's exact values."""
    import paper_2402_09356_gb300 as tlr
    gold = json.load(open(os.path.join(golden_dir, "fullsize_loglik_n40000.json")))
    assert gold["n"] == N and tuple(gold["theta"]) == THETA and gold["loc_seed"] == 1 and gold["z_seed"] == 2
    z = golden_z(golden_dir)
    assert z.shape == (N,)
    prec = {"fp64": tlr.TLR_PREC_FP64, "mixed": tlr.TLR_PREC_MIXED, "tensor": tlr.TLR_PREC_TENSOR}[precision]
    L, r, _ = factor(ctx, "hilbert", prec, eps=eps, z=z)
    L.close()
    for term in ("loglik", "logdet", "quad"):
        assert abs(r[term] - gold[term]) <= 10 * eps * abs(gold[term]), (term, r[term], gold[term])
