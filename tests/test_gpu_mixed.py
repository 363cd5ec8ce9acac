"""Mixed precision: the off-diagonal dense products in paired-FP32 arithmetic
(TLR_PREC_MIXED) or as BF16-slice products on the tensor cores
(TLR_PREC_TENSOR), everything else FP64.

The products carry about 46 (paired FP32) or 40 (five BF16 slices)
significant bits, so the factor differs from the
FP64 path only by rounding far below the compression threshold: the mixed
likelihood must stay within the FP64 path's own bound against the exact dense
oracle (10 eps |l|), within 1e-6 |l| of the FP64 path, and the rank maps of
the two paths may differ only where a singular value sits at the threshold.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def run(ctx, xy, z, theta, order, nb, eps, maxrank, precision):
    import torch
    import paper_2402_09356_gb300 as tlr
    n = z.size
    xy_d = torch.from_numpy(xy).cuda()
    xyo = torch.empty_like(xy_d)
    perm = tlr.tlr_order(ctx, xy_d, order, xy_out=xyo)
    zo = tlr.tlr_gather(ctx, perm, torch.from_numpy(z).cuda())
    L = tlr.TlrMatrix(ctx, n, nb, maxrank)
    r = tlr.tlr_loglik(L, xyo, zo, theta, tlr.Options(nb=nb, eps=eps, maxrank=maxrank, precision=precision))
    return r, tlr.tlr_mat_ranks(L), perm.cpu().numpy()


CASES = [
    # n, nb, order, theta, eps, maxrank
    (1600, 200, "morton", (1.0, 0.1, 0.5), 1e-9, 0),
    (3000, 256, "hilbert", (1.5, 0.1, 1.0), 1e-7, 0),
    (2113, 128, "kdtree", (0.7, 0.05, 1.5), 1e-5, 0),
    (1600, 200, "random", (1.0, 0.3, 0.5), 1e-9, 200),
]


@pytest.mark.parametrize("path", ["mixed", "tensor"])
@pytest.mark.parametrize("n,nb,order,theta,eps,maxrank", CASES)
def test_mixed_matches_fp64_and_oracle(ctx, n, nb, order, theta, eps, maxrank, path):
    """Both mixed paths: paired-FP32 products (TLR_PREC_MIXED) and BF16-slice
    products on the tensor cores (TLR_PREC_TENSOR)."""
    import paper_2402_09356_gb300 as tlr
    prec = tlr.TLR_PREC_MIXED if path == "mixed" else tlr.TLR_PREC_TENSOR
    xy = synth.jittered_grid(n, seed=n)
    z = oracle.simulate_z(xy, theta, synth.standard_normal(n, seed=n + 1))
    r64, rk64, perm = run(ctx, xy, z, theta, order, nb, eps, maxrank, tlr.TLR_PREC_FP64)
    rmx, rkmx, _ = run(ctx, xy, z, theta, order, nb, eps, maxrank, prec)
    assert rmx["precision_used"] == prec
    ref = oracle.loglik_dense(oracle.permute_xy(xy, perm), z[perm], theta)["loglik"]
    assert abs(rmx["loglik"] - ref) <= 10 * eps * abs(ref), (rmx["loglik"], ref)
    assert abs(rmx["loglik"] - r64["loglik"]) <= 1e-6 * abs(r64["loglik"])
    d = np.abs(rkmx.astype(np.int64) - rk64)
    assert d.max() <= 1 and (d > 0).mean() <= 0.05, (d.max(), (d > 0).mean())


@pytest.mark.parametrize("path", ["mixed", "tensor"])
def test_mixed_eps_to_zero_is_dense(ctx, path):
    import paper_2402_09356_gb300 as tlr
    prec = tlr.TLR_PREC_MIXED if path == "mixed" else tlr.TLR_PREC_TENSOR
    n, nb, theta = 1600, 200, (1.0, 0.1, 0.5)
    xy = synth.jittered_grid(n)
    z = oracle.simulate_z(xy, theta, synth.standard_normal(n, seed=2))
    r, _, perm = run(ctx, xy, z, theta, "morton", nb, 0.0, nb, prec)
    ref = oracle.loglik_dense(oracle.permute_xy(xy, perm), z[perm], theta)["loglik"]
    # tensor: ~40-bit products, amplified by the conditioning of Sigma
    assert abs(r["loglik"] - ref) <= (1e-10 if path == "mixed" else 1e-8) * abs(ref)


@pytest.mark.parametrize("path", ["mixed", "tensor"])
@pytest.mark.parametrize("n,nb", [(1, 16), (17, 16), (1000, 96)])
def test_mixed_ragged_and_tiny(ctx, n, nb, path):
    import paper_2402_09356_gb300 as tlr
    prec = tlr.TLR_PREC_MIXED if path == "mixed" else tlr.TLR_PREC_TENSOR
    theta, eps = (1.2, 0.08, 0.8), 1e-9
    xy = synth.jittered_grid(n, seed=n)
    z = oracle.simulate_z(xy, theta, synth.standard_normal(n, seed=n + 1))
    r, _, perm = run(ctx, xy, z, theta, "hilbert", nb, eps, nb, prec)
    ref = oracle.loglik_dense(oracle.permute_xy(xy, perm), z[perm], theta)["loglik"]
    assert abs(r["loglik"] - ref) <= 10 * eps * abs(ref) + 1e-12


AUTO_CASES = [
    # n, nb, theta: rough to very smooth, short to long range
    (1600, 200, (1.0, 0.1, 0.5)),
    (900, 128, (1.0, 0.2, 2.0)),
    (1200, 160, (1.5, 0.25, 2.5)),
]


def test_auto_precision_takes_mixed_or_fp64(ctx):
    """TLR_PREC_AUTO returns, bit for bit, the mixed result when the factor's
    smallest squared pivot is at least TLR_AUTO_PIVOT2 sigma2, else the FP64
    result (both started from the same, empty, rank map)."""
    import paper_2402_09356_gb300 as tlr
    seen = set()
    for n, nb, theta in AUTO_CASES:
        xy = synth.jittered_grid(n, seed=n)
        z = synth.standard_normal(n, seed=n + 3)
        out = {}
        for name, prec in (("fp64", tlr.TLR_PREC_FP64), ("mixed", tlr.TLR_PREC_MIXED), ("auto", tlr.TLR_PREC_AUTO)):
            try:
                out[name] = run(ctx, xy, z, theta, "hilbert", nb, 1e-7, nb, prec)[0]
            except tlr.TlrError as e:
                out[name] = e.code
        m = out["mixed"]
        fallback = isinstance(m, int) or m["min_pivot2"] < tlr.TLR_AUTO_PIVOT2 * theta[0]
        want = out["fp64"] if fallback else m
        got = out["auto"]
        if isinstance(want, int):
            assert got == want, (n, theta, got, want)
        else:
            assert got["loglik"] == want["loglik"] and got["logdet"] == want["logdet"], (n, theta)
            assert got["precision_used"] == (tlr.TLR_PREC_FP64 if fallback else tlr.TLR_PREC_MIXED)
        seen.add(fallback)
        if not isinstance(out["fp64"], int):
            assert out["fp64"]["min_pivot2"] > 0
    assert seen == {True, False}, "the cases should exercise both paths"
