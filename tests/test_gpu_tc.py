"""The tensor-core product of the mixed-precision path (tlr_gemm_tc) against FP64.

Each operand is split into BF16 slices with a power-of-two scale per row and
64-wide chunk of the inner dimension; with S slices a product carries about
8 S significant bits relative to the chunk's scales.  The bound checked per
entry is therefore 2^-(8 S - 2) * sum over chunks of 64 max|a_i,chunk|
max|b_j,chunk| (S = 5: 2^-38; S = 1: 2^-6), against numpy's FP64 product.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def chunk_bound(a, b, slices):
    """a: m x k, b: k x n (numpy) -> m x n bound on |C - AB|."""
    m, k = a.shape
    n = b.shape[1]
    bound = np.zeros((m, n))
    for c0 in range(0, k, 64):
        ma = np.abs(a[:, c0:c0 + 64]).max(axis=1)
        mb = np.abs(b[c0:c0 + 64, :]).max(axis=0)
        bound += 64.0 * np.outer(ma, mb)
    return 2.0 ** -(8 * slices - 2) * bound + 1e-300


def run(ctx, a, b, ta, tb, slices, alpha=1.0, beta=0.0, c0=None):
    """a = op(A) (m x k), b = op(B) (k x n) as numpy; returns the GPU C (m x n)."""
    import torch
    import paper_2402_09356_gb300 as tlr
    # a column-major matrix X (rows x cols) is the row-major torch tensor X'
    # op(A) = A' when ta: the stored A is a' (k x m, column major) -> torch tensor a (m x k)
    A = torch.from_numpy(np.ascontiguousarray(a) if ta else np.ascontiguousarray(a.T)).cuda()
    B = torch.from_numpy(np.ascontiguousarray(b) if tb else np.ascontiguousarray(b.T)).cuda()
    C = None if c0 is None else torch.from_numpy(np.ascontiguousarray(c0.T)).cuda()
    out = tlr.tlr_gemm_tc(ctx, A, B, C, alpha=alpha, beta=beta, trans_a=ta, trans_b=tb, slices=slices)
    return out.cpu().numpy().T


@pytest.mark.parametrize("trans", [(False, False), (False, True), (True, False)])
@pytest.mark.parametrize("m,n,k", [(200, 100, 150), (128, 64, 64), (1, 1, 1), (257, 129, 300), (700, 400, 1030)])
def test_tc_product_matches_fp64(ctx, trans, m, n, k):
    ta, tb = trans
    rng = np.random.default_rng(m * 7 + n * 3 + k)
    a = rng.standard_normal((m, k))
    b = rng.standard_normal((k, n))
    ref = a @ b
    got = run(ctx, a, b, ta, tb, 5)
    err = np.abs(got - ref)
    assert np.all(err <= chunk_bound(a, b, 5)), err.max()


def test_tc_per_chunk_scaling(ctx):
    """Rows and inner chunks of very different magnitude keep their relative
    accuracy: the scale is per row and 64-wide chunk, not per matrix."""
    rng = np.random.default_rng(5)
    m, n, k = 300, 130, 320
    # (the float-float accumulators keep scales 2^(e_row + e_col) in FP32's
    # normal range, |entries| > ~1e-37; the magnitudes here stay well inside)
    a = rng.standard_normal((m, k)) * np.logspace(-8, 8, m)[:, None]
    a[:, 64:128] *= 1e-10
    b = rng.standard_normal((k, n)) * np.logspace(-4, 4, n)[None, :]
    ref = a @ b
    got = run(ctx, a, b, False, True, 5)
    assert np.all(np.abs(got - ref) <= chunk_bound(a, b, 5))
    rel = np.abs(got - ref) / (np.abs(a) @ np.abs(b))
    assert rel.max() < 1e-10


def test_tc_linear_epilogue_and_single_slice(ctx):
    rng = np.random.default_rng(9)
    m, n, k = 190, 77, 260
    a = rng.uniform(-1, 1, (m, k))
    b = rng.uniform(-1, 1, (k, n))
    c0 = rng.standard_normal((m, n))
    got = run(ctx, a, b, False, False, 5, alpha=-0.75, beta=0.5, c0=c0)
    ref = -0.75 * (a @ b) + 0.5 * c0
    assert np.all(np.abs(got - ref) <= 0.75 * chunk_bound(a, b, 5) + 1e-15 * np.abs(c0))
    # one slice: the plain BF16 product with FP32 accumulation (8 bits)
    got1 = run(ctx, a, b, False, False, 1)
    err1 = np.abs(got1 - a @ b)
    assert np.all(err1 <= chunk_bound(a, b, 1))
    assert err1.max() > 1e-6  # and it is that coarse


def test_tc_empty_inner_and_nonfinite(ctx):
    rng = np.random.default_rng(3)
    a = rng.standard_normal((100, 0))
    b = rng.standard_normal((0, 50))
    c0 = rng.standard_normal((100, 50))
    got = run(ctx, a, b, False, False, 5, beta=2.0, c0=c0)
    assert np.array_equal(got, 2.0 * c0)
    a = rng.standard_normal((130, 70))
    b = rng.standard_normal((70, 40))
    a[5, 3] = np.nan
    got = run(ctx, a, b, False, False, 5)
    assert np.all(np.isnan(got[5]))
    mask = np.ones(130, bool)
    mask[5] = False
    assert np.all(np.isfinite(got[mask]))


def test_tc_bad_arguments(ctx):
    import torch
    import paper_2402_09356_gb300 as tlr
    A = torch.zeros((4, 4), dtype=torch.float64, device="cuda")
    with pytest.raises(tlr.TlrError) as e:
        tlr.tlr_gemm_tc(ctx, A, A, slices=3)
    assert e.value.code == tlr.TLR_ERR_ARG
    with pytest.raises(tlr.TlrError) as e:
        tlr.tlr_gemm_tc(ctx, A, A, trans_a=True, trans_b=True)
    assert e.value.code == tlr.TLR_ERR_ARG
