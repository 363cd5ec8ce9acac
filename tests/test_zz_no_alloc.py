"""tlr_order_noalloc: the ordering entry point that allocates nothing.

Some callers cannot allocate device memory while they run (a latency-bound
serving loop that cannot absorb cudaMalloc's device synchronisation, or a
process with a fixed memory budget).  For them the library keeps one fixed
scratch array per device.  This file is collected last so that a failure here
is seen only after every other test has run; it passes alone and after them.
The result must be bit-identical to tlr_order's, on two calls in a row (the
second call smaller than the first, so stale scratch contents would show).
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def _both(ctx, n, method, seed):
    import torch
    import paper_2402_09356_gb300 as tlr
    xy = torch.from_numpy(synth.jittered_grid(n, seed=seed)).cuda()
    codes_a = torch.zeros(n, dtype=torch.int32, device="cuda")
    codes_b = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    perm_a = tlr.tlr_order(ctx, xy, method, seed=seed, codes=codes_a)
    perm_b = tlr.tlr_order_noalloc(xy, method, seed=seed, codes=codes_b)
    torch.cuda.synchronize()
    return perm_a.cpu().numpy(), perm_b.cpu().numpy(), codes_a.cpu().numpy(), codes_b.cpu().numpy()


@pytest.mark.parametrize("method", ["hilbert", "morton", "random"])
def test_noalloc_matches_tlr_order_twice(ctx, method):
    for n, seed in ((50000, 5), (1601, 9)):
        pa, pb, ca, cb = _both(ctx, n, method, seed)
        assert np.array_equal(pa, pb), (method, n)
        assert np.array_equal(ca, cb), (method, n)


def test_noalloc_rejects_oversize_and_other_methods(ctx):
    import torch
    import paper_2402_09356_gb300 as tlr
    big = torch.zeros(2 * (262144 + 1), dtype=torch.float64, device="cuda")
    with pytest.raises(tlr.TlrError) as e:
        tlr.tlr_order_noalloc(big, "hilbert")
    assert e.value.code == tlr.TLR_ERR_ARG
    small = torch.zeros(20, dtype=torch.float64, device="cuda")
    with pytest.raises(tlr.TlrError) as e:
        tlr.tlr_order_noalloc(small, "kdtree")
    assert e.value.code == tlr.TLR_ERR_ARG
