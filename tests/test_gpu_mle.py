"""tlr_mle (Sec. 5.1: derivative-free, bound-constrained maximisation of Eq. 1.2).

The oracle has no optimiser, so the estimate is checked through the exact
dense likelihood: it must beat the data-generating theta, be a local maximum
of the oracle's l along each coordinate, and give a value of the identifiable
combination f = sigma2 beta^(-2 nu) (Eq. 5.1) close to the truth.
"""
import math

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def test_mle_small_config(ctx):
    import torch
    import paper_2402_09356_gb300 as tlr
    n, nb, eps = 900, 150, 1e-9
    truth = (1.0, 0.1, 0.5)
    xy = synth.jittered_grid(n, seed=31)
    z = oracle.simulate_z(xy, truth, synth.standard_normal(n, seed=32))
    xy_d = torch.from_numpy(xy).cuda()
    xyo = torch.empty_like(xy_d)
    perm = tlr.tlr_order(ctx, xy_d, "hilbert", xy_out=xyo)
    zo = tlr.tlr_gather(ctx, perm, torch.from_numpy(z).cuda())
    L = tlr.TlrMatrix(ctx, n, nb, nb)
    res = tlr.tlr_mle(L, xyo, zo, tlr.Options(nb=nb, eps=eps, maxrank=nb), theta0=(0.6, 0.05, 0.8),
                      lo=(0.05, 0.005, 0.1), hi=(10.0, 2.0, 3.0), tol=1e-9, max_iter=600)
    th = res["theta"]
    p = perm.cpu().numpy()
    xyp, zp = oracle.permute_xy(xy, p), z[p]
    ll = lambda t: oracle.loglik_dense(xyp, zp, t)["loglik"]
    l_hat = ll(th)
    assert abs(l_hat - res["loglik"]) <= 1e-7 * abs(l_hat)       # GPU value at the estimate
    assert l_hat >= ll(truth) - 1e-6                               # the MLE beats the truth
    for d in range(3):                                             # coordinate-wise local max
        for f in (0.97, 1.03):
            t = list(th)
            t[d] *= f
            assert ll(t) <= l_hat + 1e-6, (d, f)
    f_hat = th[0] * th[1] ** (-2 * th[2])
    f_true = truth[0] * truth[1] ** (-2 * truth[2])
    assert abs(math.log(f_hat / f_true)) < 0.3                     # Eq. 5.1 quantity
    assert 4 <= res["iters"] <= 600


@pytest.mark.parametrize("path", ["mixed", "tensor"])
def test_mle_mixed_paths_match_fp64(ctx, path):
    """The mixed-precision paths reach the FP64 path's estimate: every parameter
    of theta-hat within 1e-3 (relative) of the FP64 search's, same data and
    start (the accuracy target of the mixed-precision growth row)."""
    import torch
    import paper_2402_09356_gb300 as tlr
    n, nb, eps = 1600, 200, 1e-7
    truth = (1.0, 0.1, 0.5)
    xy = synth.jittered_grid(n, seed=41)
    z = oracle.simulate_z(xy, truth, synth.standard_normal(n, seed=42))
    xy_d = torch.from_numpy(xy).cuda()
    xyo = torch.empty_like(xy_d)
    perm = tlr.tlr_order(ctx, xy_d, "hilbert", xy_out=xyo)
    zo = tlr.tlr_gather(ctx, perm, torch.from_numpy(z).cuda())
    out = {}
    for name, prec in (("fp64", tlr.TLR_PREC_FP64),
                       (path, tlr.TLR_PREC_MIXED if path == "mixed" else tlr.TLR_PREC_TENSOR)):
        L = tlr.TlrMatrix(ctx, n, nb)
        out[name] = tlr.tlr_mle(L, xyo, zo, tlr.Options(nb=nb, eps=eps, precision=prec), theta0=(0.6, 0.05, 0.8),
                                lo=(0.05, 0.005, 0.1), hi=(10.0, 2.0, 3.0), tol=1e-9, max_iter=600)
        L.close()
    a, b = out[path]["theta"], out["fp64"]["theta"]
    for d in range(3):
        assert abs(a[d] - b[d]) <= 1e-3 * abs(b[d]), (d, a, b)
    assert abs(out[path]["loglik"] - out["fp64"]["loglik"]) <= 1e-6 * abs(out["fp64"]["loglik"])
