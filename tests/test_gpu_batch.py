"""tlr_loglik_batch: several factorisations advanced together on one context.

Every step of a tile column is one launch for all entries (panel products
with the Matern generation, the diagonal POTRF clusters, the compression's
launch classes, V <- L^-1 V, Gram matrices, solve); each entry must still
compute exactly what tlr_loglik computes for it alone: the same l, log|Sigma|,
Z' Sigma^-1 Z and rank map bit for bit, on every precision path, on a first
evaluation and on one that starts from the previous rank map.  Entries that
fail (a rank above maxrank, non-finite locations) report their own status,
and the others are unaffected.  The grouped results are also checked against
the exact dense oracle (Eq. 1.2) at 10 eps.
"""
import math

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

# uneven datasets: ragged last tiles, different tile counts, different theta
CASES = [(900, 200, (1.0, 0.1, 0.5), 11), (1500, 200, (0.7, 0.05, 1.0), 12), (2300, 256, (1.5, 0.2, 0.5), 13),
         (640, 128, (1.0, 0.03, 0.8), 14), (1, 16, (1.0, 0.1, 0.5), 15)]


def dataset(ctx, n, theta, seed, order="hilbert"):
    import torch
    import paper_2402_09356_gb300 as tlr
    xy = synth.jittered_grid(n, seed=seed)
    z = oracle.simulate_z(xy, theta, synth.standard_normal(n, seed=seed + 100))
    xy_d = torch.from_numpy(xy).cuda()
    xyo = torch.empty_like(xy_d)
    perm = tlr.tlr_order(ctx, xy_d, order, xy_out=xyo)
    zo = tlr.tlr_gather(ctx, perm, torch.from_numpy(z).cuda())
    return xy, z, xyo, zo, perm.cpu().numpy()


def same(a, b):
    return all(a[k] == b[k] for k in ("loglik", "logdet", "quad", "max_rank", "mean_rank", "offdiag_bytes",
                                      "precision_used", "min_pivot2"))


@pytest.mark.parametrize("prec", ["fp64", "mixed", "tensor", "auto"])
def test_batch_bitwise_equals_single(ctx, prec):
    import paper_2402_09356_gb300 as tlr
    p = {"fp64": tlr.TLR_PREC_FP64, "mixed": tlr.TLR_PREC_MIXED, "tensor": tlr.TLR_PREC_TENSOR,
         "auto": tlr.TLR_PREC_AUTO}[prec]
    data = [dataset(ctx, n, th, sd) for n, nb, th, sd in CASES]
    opts = [tlr.Options(nb=nb, eps=1e-7, precision=p) for n, nb, th, sd in CASES]
    single = [tlr.TlrMatrix(ctx, n, nb) for n, nb, th, sd in CASES]
    group = [tlr.TlrMatrix(ctx, n, nb) for n, nb, th, sd in CASES]
    # two evaluations each: the second starts from the first one's rank map
    for step, scale in enumerate((1.0, 1.1)):
        thetas = [(th[0] * scale, th[1] * scale, th[2]) for n, nb, th, sd in CASES]
        alone = [tlr.tlr_loglik(L, d[2], d[3], t, o) for L, d, t, o in zip(single, data, thetas, opts)]
        res, st = tlr.tlr_loglik_batch(group, [d[2] for d in data], [d[3] for d in data], thetas, opts)
        assert st == [tlr.TLR_OK] * len(CASES)
        for g in range(len(CASES)):
            assert same(res[g], alone[g]), (step, g, res[g], alone[g])
            assert np.array_equal(tlr.tlr_mat_ranks(group[g]), tlr.tlr_mat_ranks(single[g]))


def test_batch_against_dense_oracle(ctx):
    """The grouped results, entry by entry, within 10 eps of the exact l (Eq. 1.2)."""
    import paper_2402_09356_gb300 as tlr
    eps = 1e-9
    cases = CASES[:4]
    data = [dataset(ctx, n, th, sd) for n, nb, th, sd in cases]
    mats = [tlr.TlrMatrix(ctx, n, nb) for n, nb, th, sd in cases]
    opts = [tlr.Options(nb=nb, eps=eps, precision=tlr.TLR_PREC_MIXED) for n, nb, th, sd in cases]
    res, st = tlr.tlr_loglik_batch(mats, [d[2] for d in data], [d[3] for d in data], [c[2] for c in cases], opts)
    assert st == [tlr.TLR_OK] * len(cases)
    for (n, nb, th, sd), d, r in zip(cases, data, res):
        xy, z, _, _, perm = d
        ex = oracle.loglik_dense(oracle.permute_xy(xy, perm), z[perm], th)
        for key in ("loglik", "logdet", "quad"):
            assert abs(r[key] - ex[key]) <= 10 * eps * abs(ex[key]), (n, key, r[key], ex[key])


def test_batch_failures_stay_with_their_entry(ctx):
    import paper_2402_09356_gb300 as tlr
    n, nb, th = 1600, 200, (1.0, 0.1, 0.5)
    good = [dataset(ctx, n, th, 21), dataset(ctx, 1000, th, 22)]
    xy_bad, z_bad, _, _, _ = dataset(ctx, 400, th, 23, order="identity")
    import torch
    xy_bad = xy_bad.copy()
    xy_bad[150] = np.nan
    xyb = torch.from_numpy(xy_bad).cuda()
    zb = torch.from_numpy(z_bad).cuda()
    rank_fail = dataset(ctx, n, th, 24, order="random")
    entries = [good[0], (None, None, xyb, zb, None), rank_fail, good[1]]
    sizes = [(n, nb, 0), (400, 100, 0), (n, nb, 4), (1000, nb, 0)]
    opts = [tlr.Options(nb=b, eps=1e-9, maxrank=mr) for _, b, mr in sizes]
    mats = [tlr.TlrMatrix(ctx, m, b, mr) for m, b, mr in sizes]
    res, st = tlr.tlr_loglik_batch(mats, [e[2] for e in entries], [e[3] for e in entries], [th] * 4, opts)
    assert st[0] == tlr.TLR_OK and st[3] == tlr.TLR_OK
    assert st[1] in (tlr.TLR_ERR_NAN, tlr.TLR_ERR_NOT_SPD)
    assert st[2] == tlr.TLR_ERR_RANK
    # the same status and info as alone, and the good entries as alone
    for g, e in enumerate(entries):
        m, b, mr = sizes[g]
        L = tlr.TlrMatrix(ctx, m, b, mr)
        if st[g] == tlr.TLR_OK:
            assert same(res[g], tlr.tlr_loglik(L, e[2], e[3], th, opts[g]))
        else:
            with pytest.raises(tlr.TlrError) as err:
                tlr.tlr_loglik(L, e[2], e[3], th, opts[g])
            assert err.value.code == st[g]
            assert err.value.info == res[g]["info"]
    # the context stays usable
    r = tlr.tlr_loglik(tlr.TlrMatrix(ctx, n, nb), good[0][2], good[0][3], th, opts[0])
    assert math.isfinite(r["loglik"])


def test_batch_bad_arguments(ctx):
    import paper_2402_09356_gb300 as tlr
    d = dataset(ctx, 400, (1.0, 0.1, 0.5), 31)
    L1, L2 = tlr.TlrMatrix(ctx, 400, 100), tlr.TlrMatrix(ctx, 400, 100)
    o64, omix = tlr.Options(nb=100), tlr.Options(nb=100, precision=tlr.TLR_PREC_MIXED)
    th = (1.0, 0.1, 0.5)
    for mats, opts in (([L1, L1], [o64, o64]),          # one L for two entries
                       ([L1, L2], [o64, omix])):        # two precisions
        with pytest.raises(tlr.TlrError) as e:
            tlr.tlr_loglik_batch(mats, [d[2]] * 2, [d[3]] * 2, [th] * 2, opts)
        assert e.value.code == tlr.TLR_ERR_ARG
    with pytest.raises(tlr.TlrError) as e:
        tlr.tlr_loglik_batch([L1] * 33, [d[2]] * 33, [d[3]] * 33, [th] * 33, o64)
    assert e.value.code == tlr.TLR_ERR_ARG


def test_buckets_roundtrip_and_validation(ctx):
    import paper_2402_09356_gb300 as tlr
    default = tlr.tlr_ctx_get_buckets(ctx)
    assert default["qr_size"] == [4, 8, 16, 16] and default["svd_size"] == [1, 4, 8, 16]
    assert default["qr_edge"][:2] == [64, 128] and default["svd_edge"][:3] == [48, 96, 160]
    bad = dict(default, qr_size=[3, 8, 16, 16])
    with pytest.raises(tlr.TlrError) as e:
        tlr.tlr_ctx_set_buckets(ctx, bad)
    assert e.value.code == tlr.TLR_ERR_ARG
    bad = dict(default, svd_edge=[96, 48, 160, 0])
    with pytest.raises(tlr.TlrError):
        tlr.tlr_ctx_set_buckets(ctx, bad)
    assert tlr.tlr_ctx_get_buckets(ctx) == default  # unchanged by a refused map
    mine = {"qr_edge": [32, 96, 200, 0], "qr_size": [2, 4, 8, 16], "svd_edge": [64, 128, 256, 0],
            "svd_size": [2, 4, 8, 8]}
    tlr.tlr_ctx_set_buckets(ctx, mine)
    got = tlr.tlr_ctx_get_buckets(ctx)
    assert got["qr_size"] == mine["qr_size"] and got["svd_size"] == mine["svd_size"]
    tlr.tlr_ctx_set_buckets(ctx, None)
    assert tlr.tlr_ctx_get_buckets(ctx) == default


@pytest.mark.parametrize("buckets", [
    {"qr_edge": [10 ** 6] * 4, "qr_size": [1] * 4, "svd_edge": [10 ** 6] * 4, "svd_size": [1] * 4},
    {"qr_edge": [32, 64, 96, 0], "qr_size": [2, 4, 8, 16], "svd_edge": [32, 64, 96, 0], "svd_size": [2, 4, 8, 16]},
])
def test_buckets_change_reduction_not_result(ctx, buckets):
    """Other cluster sizes change how a tile's QR and SVD are reduced: ranks
    equal the default map's (up to singular values within 1e-3 of the
    threshold) and l stays within 10 eps of the exact oracle."""
    import paper_2402_09356_gb300 as tlr
    n, nb, th, eps = 2000, 250, (1.0, 0.05, 0.5), 1e-9
    xy, z, xyo, zo, perm = dataset(ctx, n, th, 41)
    ex = oracle.loglik_dense(oracle.permute_xy(xy, perm), z[perm], th)
    L0 = tlr.TlrMatrix(ctx, n, nb)
    r0 = tlr.tlr_loglik(L0, xyo, zo, th, tlr.Options(nb=nb, eps=eps))
    try:
        tlr.tlr_ctx_set_buckets(ctx, buckets)
        L1 = tlr.TlrMatrix(ctx, n, nb)
        r1 = tlr.tlr_loglik(L1, xyo, zo, th, tlr.Options(nb=nb, eps=eps))
    finally:
        tlr.tlr_ctx_set_buckets(ctx, None)
    for key in ("loglik", "logdet", "quad"):
        assert abs(r1[key] - ex[key]) <= 10 * eps * abs(ex[key])
    k0, k1 = tlr.tlr_mat_ranks(L0), tlr.tlr_mat_ranks(L1)
    assert np.abs(k0.astype(int) - k1.astype(int)).max() <= 1
    assert abs(r1["loglik"] - r0["loglik"]) <= 20 * eps * abs(r0["loglik"])
