"""GPU ordering (Sec. 3) against the oracle: permutations and codes bit-exact."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

METHODS = ["identity", "random", "morton", "hilbert", "kdtree", "maxmin"]


def run(ctx, xy, method, seed=3, flags=0):
    import torch
    import paper_2402_09356_gb300 as tlr
    n = xy.size // 2
    d = torch.from_numpy(np.ascontiguousarray(xy)).cuda()
    codes = torch.zeros(n, dtype=torch.int32, device="cuda")
    out = torch.empty_like(d)
    perm = tlr.tlr_order(ctx, d, method, seed=seed, flags=flags, codes=codes, xy_out=out)
    torch.cuda.synchronize()
    return perm.cpu().numpy(), codes.cpu().numpy().view(np.uint32), out.cpu().numpy()


def check(ctx, xy, method, seed=3):
    perm_o, codes_o = oracle.order(xy, method, seed)
    perm, codes, out = run(ctx, xy, method, seed)
    assert np.array_equal(perm, perm_o), method
    if codes_o is not None:
        assert np.array_equal(codes, codes_o), method
    assert np.array_equal(out, oracle.permute_xy(xy, perm_o))


@pytest.mark.parametrize("method", METHODS)
@pytest.mark.parametrize("n", [1, 2, 3, 7, 100, 257, 1600, 4133])
def test_order_parity(ctx, method, n):
    check(ctx, synth.jittered_grid(n, seed=n + 17), method, seed=11)


@pytest.mark.parametrize("method", METHODS)
def test_order_ties_and_clamping(ctx, method):
    # an exact lattice (equal coordinates and equal codes everywhere), points
    # outside [0, 1] (clamped by the encoders) and duplicated locations
    g = np.arange(12) / 11.0
    xs, ys = np.meshgrid(g, g, indexing="ij")
    x = np.concatenate([xs.ravel(), [-0.3, 1.2, 0.5, 0.5], xs.ravel()[:20]])
    y = np.concatenate([ys.ravel(), [0.4, 1.7, -2.0, 0.5], ys.ravel()[:20]])
    check(ctx, np.concatenate([x, y]), method)


def test_quantize_decode(ctx):
    import paper_2402_09356_gb300 as tlr
    xy = synth.jittered_grid(999, seed=5)
    for m in ("morton", "hilbert"):
        perm, _, out = run(ctx, xy, m, flags=tlr.TLR_ORDER_QUANTIZE)
        assert np.array_equal(out, oracle.permute_xy(oracle.decode_xy(xy), perm))


@pytest.mark.parametrize("method", METHODS)
def test_order_full_size(ctx, method):
    # the 200 x 200 perturbed grid of the n = 40,000 ordering study
    check(ctx, synth.jittered_grid(40000, seed=1), method)
