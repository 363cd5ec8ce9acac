"""Worker pool: many resident datasets evaluated by concurrent workers.

Each dataset's k-th result must be bit-for-bit the result of k tlr_loglik calls
on one context and one tlr_mat (the same ordered data, theta sequence, eps and
precision), whatever runs beside it; under a budget that forces evictions too.
The first result of each dataset is also checked against the dense oracle
(10 eps |l|, FP64 path) and its ordering against the oracle's (bit-exact).
"""
import threading

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

# rank slots: the whole tile (maxrank = nb), so that no request of these small
# cases stops at a rank cap
FULL = 1024
KEYS = ("loglik", "logdet", "quad", "max_rank", "mean_rank", "offdiag_bytes")


def make(n, seed, theta):
    xy = synth.jittered_grid(n, seed=seed)
    z = oracle.simulate_z(xy, theta, synth.standard_normal(n, seed=seed + 1))
    return xy, z


def alone(ctx, pool, did, seq):
    """The dataset's request sequence on one context and one tlr_mat (rank
    slots = the tile size, as in the pools below)."""
    import paper_2402_09356_gb300 as tlr
    d = tlr.tlr_pool_dataset(pool, did)
    maxrank = d["nb"]
    L = tlr.TlrMatrix(ctx, d["n"], d["nb"], maxrank)
    out = []
    for theta, eps, prec in seq:
        try:
            out.append(tlr.tlr_loglik(L, d["xy"], d["z"], theta, tlr.Options(nb=d["nb"], eps=eps, maxrank=maxrank,
                                                                             precision=prec)))
        except tlr.TlrError as e:
            out.append(e.code)
    L.close()
    return out


def same(a, b):
    if isinstance(a, int) or isinstance(b, int):
        return a == b
    return all(a[k] == b[k] for k in KEYS)


def run_mix(pool, seqs):
    """Submit every dataset's sequence interleaved round-robin; results per dataset."""
    import paper_2402_09356_gb300 as tlr
    tickets = {d: [] for d in seqs}
    longest = max(len(s) for s in seqs.values())
    for k in range(longest):
        for d, s in seqs.items():
            if k < len(s):
                theta, eps, prec = s[k]
                tickets[d].append(tlr.tlr_pool_submit(pool, d, theta, eps, prec))
    res = {}
    for d, ts in tickets.items():
        res[d] = []
        for t in ts:
            try:
                res[d].append(tlr.tlr_pool_wait(pool, t)[0])
            except tlr.TlrError as e:
                res[d].append(e.code)
    return res


def sequences(ids, steps, seed, precisions):
    seqs = {}
    for j, d in enumerate(ids):
        walk = synth.theta_walk((1.0, 0.1, 0.5 + 0.25 * (j % 3)), steps, seed=seed + j)
        seqs[d] = [(tuple(th), 1e-7, precisions[j % len(precisions)]) for th in walk]
    return seqs


@pytest.mark.parametrize("group", [1, 4])
def test_pool_identical_alone_and_in_the_mix(ctx, group):
    """group > 1: workers evaluate up to `group` queued requests of one
    precision together (tlr_loglik_batch); the results stay those of the
    dataset's sequence alone."""
    import paper_2402_09356_gb300 as tlr
    sizes = [700, 1500, 2300, 3100, 1201]
    pool = tlr.Pool(0, workers=3, nb=256, maxrank=FULL)
    tlr.tlr_pool_configure(pool, group)
    ids, data = [], {}
    for j, n in enumerate(sizes):
        xy, z = make(n, 11 * j + 1, (1.0, 0.1, 0.5))
        ids.append(tlr.tlr_pool_add(pool, xy, z, "morton", nb=256 if j != 4 else 160))
        data[ids[-1]] = (xy, z)
    seqs = sequences(ids, 4, 5, [tlr.TLR_PREC_FP64, tlr.TLR_PREC_MIXED])
    mix = run_mix(pool, seqs)
    st = tlr.tlr_pool_stats(pool)
    assert st["completed"] == sum(len(s) for s in seqs.values())
    assert st["max_running"] >= 2
    assert (st["grouped_requests"] > 0) == (group > 1)
    for d in ids:
        ref = alone(ctx, pool, d, seqs[d])
        for k, (a, b) in enumerate(zip(mix[d], ref)):
            assert same(a, b), (d, k, a, b)
        # ordering and the first result against the oracle
        xy, z = data[d]
        got = tlr.tlr_pool_dataset(pool, d)
        perm = got["perm"].cpu().numpy()
        assert np.array_equal(perm, oracle.order(xy, "morton")[0])
        theta, eps, prec = seqs[d][0]
        assert isinstance(mix[d][0], dict), ("first request failed", d, mix[d][0])
        exact = oracle.loglik_dense(oracle.permute_xy(xy, perm), z[perm], theta)["loglik"]
        assert abs(mix[d][0]["loglik"] - exact) <= 10 * eps * abs(exact), (d, mix[d][0]["loglik"], exact)
    pool.close()


@pytest.mark.parametrize("group", [1, 3])
def test_pool_tight_budget_evicts_and_stays_identical(ctx, group):
    import paper_2402_09356_gb300 as tlr
    sizes = [1800, 2600, 1000, 2600]
    nb = 200
    fps = [tlr.tlr_pool_footprint(n, nb, nb) for n in sizes]
    # room for the resident data and for the largest dataset to run alone: all
    # four factors (about 160 MB) plus any workspace (at least 64 MiB) do not
    # fit, so requests of different datasets evict one another
    budget = sum(f["base"] for f in fps) + max(f["factor"] + f["work"] for f in fps)
    pool = tlr.Pool(0, workers=2, nb=nb, maxrank=FULL, hbm_budget=budget)
    tlr.tlr_pool_configure(pool, group)
    ids = []
    for j, n in enumerate(sizes):
        xy, z = make(n, 7 * j + 3, (1.0, 0.1, 1.0))
        ids.append(tlr.tlr_pool_add(pool, xy, z, "hilbert"))
    seqs = sequences(ids, 3, 17, [tlr.TLR_PREC_MIXED])
    mix = run_mix(pool, seqs)
    st = tlr.tlr_pool_stats(pool)
    assert st["evictions"] > 0 and st["allocations"] > len(ids)
    assert st["peak"] <= budget
    for d in ids:
        ref = alone(ctx, pool, d, seqs[d])
        for k, (a, b) in enumerate(zip(mix[d], ref)):
            assert same(a, b), (d, k, a, b)
    pool.close()


def test_pool_batched_many_small_datasets(ctx):
    """A small batched workload: 24 datasets of uneven n on 8 workers."""
    import paper_2402_09356_gb300 as tlr
    rng = np.random.default_rng(4)
    sizes = rng.integers(300, 2500, 24)
    pool = tlr.Pool(0, workers=8, nb=192, maxrank=FULL)
    ids = []
    thetas = []
    for j, n in enumerate(sizes):
        xy, z = make(int(n), 100 + j, (1.0, 0.1, 0.5))
        ids.append(tlr.tlr_pool_add(pool, xy, z, "morton"))
        thetas.append((float(rng.uniform(0.5, 2.0)), float(rng.uniform(0.02, 0.3)), float(rng.uniform(0.5, 2.5))))
    res, status = tlr.tlr_pool_loglik(pool, ids, thetas, eps=1e-7, precision=tlr.TLR_PREC_MIXED)
    for d, th, r, s in zip(ids, thetas, res, status):
        ref = alone(ctx, pool, d, [(th, 1e-7, tlr.TLR_PREC_MIXED)])[0]
        if isinstance(ref, int):
            assert s == ref
        else:
            assert s == tlr.TLR_OK and same(r, ref), (d, r, ref)
    assert tlr.tlr_pool_stats(pool)["max_running"] >= 4
    pool.close()


def test_pool_mle_matches_tlr_mle_beside_other_traffic(ctx):
    import torch
    import paper_2402_09356_gb300 as tlr
    theta_true = (1.0, 0.1, 0.5)
    pool = tlr.Pool(0, workers=3, nb=200, maxrank=FULL)
    xy, z = make(1600, 41, theta_true)
    did = tlr.tlr_pool_add(pool, xy, z, "morton")
    others = [tlr.tlr_pool_add(pool, *make(n, 50 + n, theta_true), "morton") for n in (900, 1400)]
    lo, hi = (0.01, 0.005, 0.1), (5.0, 2.0, 3.0)
    start = (0.5, 0.2, 1.0)
    # other requests run while the MLE's evaluations go through the pool
    tickets = [tlr.tlr_pool_submit(pool, o, (1.0, 0.05 + 0.01 * k, 0.5), 1e-7) for k in range(6) for o in others]
    got = {}

    def mle():
        got["r"] = tlr.tlr_pool_mle(pool, did, start, lo, hi, eps=1e-7, tol=1e-7, max_iter=60)

    t = threading.Thread(target=mle)
    t.start()
    t.join()
    for tk in tickets:
        tlr.tlr_pool_wait(pool, tk)
    th, ll, it = got["r"]
    d = tlr.tlr_pool_dataset(pool, did)
    L = tlr.TlrMatrix(ctx, d["n"], d["nb"], d["nb"])
    ref = tlr.tlr_mle(L, d["xy"], d["z"], tlr.Options(nb=d["nb"], eps=1e-7, maxrank=d["nb"]), start, lo, hi,
                      tol=1e-7, max_iter=60)
    torch.cuda.synchronize()
    assert ref["theta"] == th and ref["loglik"] == ll and ref["iters"] == it
    L.close()
    pool.close()


def test_pool_tune_picks_a_candidate(ctx):
    import paper_2402_09356_gb300 as tlr
    pool = tlr.Pool(0, workers=2, nb=256, maxrank=FULL)
    xy, z = make(2400, 9, (1.0, 0.1, 0.5))
    did = tlr.tlr_pool_add(pool, xy, z, "hilbert")
    best, ms = tlr.tlr_pool_tune(pool, did, (1.0, 0.1, 0.5), [160, 240, 400])
    assert best in (160, 240, 400)
    assert all(v > 0 for v in ms.values())
    assert ms[best] == min(ms.values())
    d = tlr.tlr_pool_dataset(pool, did)
    assert d["nb"] == best and d["last_max_rank"] == 0  # rank map restarted
    r, _ = tlr.tlr_pool_wait(pool, tlr.tlr_pool_submit(pool, did, (1.0, 0.1, 0.5), 1e-7))
    exact = oracle.loglik_dense(oracle.permute_xy(xy, d["perm"].cpu().numpy()), z[d["perm"].cpu().numpy()],
                                (1.0, 0.1, 0.5))["loglik"]
    assert abs(r["loglik"] - exact) <= 1e-6 * abs(exact)
    pool.close()


def test_pool_errors_are_per_request(ctx):
    import paper_2402_09356_gb300 as tlr
    pool = tlr.Pool(0, workers=2, nb=128, maxrank=FULL)
    xy, z = make(500, 3, (1.0, 0.1, 0.5))
    did = tlr.tlr_pool_add(pool, xy, z, "morton")
    with pytest.raises(tlr.TlrError) as e:
        tlr.tlr_pool_submit(pool, did + 17, (1.0, 0.1, 0.5))
    assert e.value.code == tlr.TLR_ERR_ARG
    with pytest.raises(tlr.TlrError):
        tlr.tlr_pool_submit(pool, did, (1.0, 0.1, 0.5), eps=-1.0)
    bad = tlr.tlr_pool_submit(pool, did, (-1.0, 0.1, 0.5))
    good = tlr.tlr_pool_submit(pool, did, (1.0, 0.1, 0.5))
    with pytest.raises(tlr.TlrError) as e:
        tlr.tlr_pool_wait(pool, bad)
    assert e.value.code == tlr.TLR_ERR_ARG
    r, times = tlr.tlr_pool_wait(pool, good)
    assert np.isfinite(r["loglik"]) and times["latency_ms"] >= times["run_ms"] >= 0
    with pytest.raises(tlr.TlrError):
        tlr.tlr_pool_wait(pool, good)  # consumed
    with pytest.raises(tlr.TlrError) as e:
        tlr.tlr_pool_add(pool, xy[:10], z[:3], "morton")
    small = tlr.Pool(0, workers=1, nb=128, hbm_budget=1 << 20)
    with pytest.raises(tlr.TlrError) as e:
        tlr.tlr_pool_add(small, xy, z, "morton")
    assert e.value.code == tlr.TLR_ERR_OOM
    small.close()
    tlr.tlr_pool_remove(pool, did)
    with pytest.raises(tlr.TlrError):
        tlr.tlr_pool_submit(pool, did, (1.0, 0.1, 0.5))
    pool.close()


def test_pool_compact_slot_overflow_falls_back_to_uniform(ctx):
    """A request whose ranks outgrow the compact slots sized by the previous
    request (here: eps 1e-3, then 1e-9) is rerun from the same rank map on
    uniform slots; every result still equals the single-context sequence."""
    import paper_2402_09356_gb300 as tlr
    pool = tlr.Pool(0, workers=2, nb=256, maxrank=FULL)
    xy, z = make(2600, 77, (1.0, 0.1, 0.5))
    did = tlr.tlr_pool_add(pool, xy, z, "hilbert")
    seq = [((1.0, 0.1, 0.5), 1e-3, tlr.TLR_PREC_FP64), ((1.0, 0.1, 0.5), 1e-9, tlr.TLR_PREC_FP64),
           ((1.02, 0.1, 0.5), 1e-9, tlr.TLR_PREC_MIXED)]
    got = run_mix(pool, {did: seq})[did]
    ref = alone(ctx, pool, did, seq)
    for k, (a, b) in enumerate(zip(got, ref)):
        assert same(a, b), (k, a, b)
    st = tlr.tlr_pool_stats(pool)
    # uniform (first), compact, uniform (the overflow rerun), compact
    assert st["allocations"] >= 3, st
    pool.close()


def test_pool_autotune_keeps_the_fastest_candidate(ctx):
    """Rank-bucket and group-size tuning on a batch of uneven datasets: every
    candidate is timed, the pool keeps the fastest, and its results after
    tuning match the dense oracle."""
    import paper_2402_09356_gb300 as tlr
    sizes = [1200, 2500, 1800, 3000, 900, 2200]
    pool = tlr.Pool(0, workers=2, nb=256, maxrank=FULL)
    ids, data = [], []
    for j, n in enumerate(sizes):
        xy, z = make(n, 5 * j + 2, (1.0, 0.1, 0.5))
        ids.append(tlr.tlr_pool_add(pool, xy, z, "hilbert"))
        data.append((xy, z))
    thetas = [(1.0, 0.1, 0.5)] * len(ids)
    small = {"qr_edge": [48, 96, 160, 0], "qr_size": [2, 4, 8, 8], "svd_edge": [48, 96, 160, 0],
             "svd_size": [1, 2, 4, 8]}
    cands = [(1, None), (3, None), (3, small)]
    best, rates = tlr.tlr_pool_autotune(pool, ids, thetas, cands, eps=1e-9, precision=tlr.TLR_PREC_MIXED)
    assert 0 <= best < len(cands) and all(r > 0 for r in rates)
    assert rates[best] == max(rates)
    cfg = tlr.tlr_pool_get_config(pool)
    assert cfg["group"] == cands[best][0]
    if cands[best][1] is not None:
        assert cfg["buckets"]["qr_size"] == small["qr_size"]
    res, st = tlr.tlr_pool_loglik(pool, ids, thetas, eps=1e-9, precision=tlr.TLR_PREC_MIXED)
    assert st == [tlr.TLR_OK] * len(ids)
    for d, (xy, z), r in zip(ids, data, res):
        perm = tlr.tlr_pool_dataset(pool, d)["perm"].cpu().numpy()
        exact = oracle.loglik_dense(oracle.permute_xy(xy, perm), z[perm], thetas[0])["loglik"]
        assert abs(r["loglik"] - exact) <= 10 * 1e-9 * abs(exact)
    with pytest.raises(tlr.TlrError):
        tlr.tlr_pool_configure(pool, 0)
    with pytest.raises(tlr.TlrError):
        tlr.tlr_pool_autotune(pool, ids, thetas, [(40, None)])
    pool.close()
