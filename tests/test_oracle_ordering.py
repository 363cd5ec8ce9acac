"""Pins for the oracle's orderings (Sec. 3).

Hilbert: the visit orders drawn in Figure 3 (tests/golden/hilbert_figure.txt).
Morton: the bit-interleave definition, checked against its recursive Z-shape.
KD-tree and max-min: hand-made cases and brute-force checkers that test the
rules of Sec. 3.2 / the max-min definition on the output, independently of
the way the oracle builds it.  Random: the published SplitMix64 output.
"""
import math

import numpy as np
import pytest

import oracle
import synth


def load_figure(golden_dir):
    seqs = {}
    with open(golden_dir + "/hilbert_figure.txt") as f:
        for line in f:
            if line.startswith("p="):
                head, *cells = line.split()
                seqs[int(head[2:])] = [tuple(map(int, c.split(","))) for c in cells]
    return seqs


def test_quantize_pins():
    q = oracle.quantize(np.array([0.0, 1.0, 0.5, -0.2, 1.7, 1 / 65535, 0.25]))
    # 0.5 * 65535 = 32767.5 rounds to the even neighbour 32768
    assert list(q) == [0, 65535, 32768, 0, 65535, 1, 16384]
    x = synth.uniform(3, 1000)
    assert np.all(np.abs(oracle.dequantize(oracle.quantize(x)) - x) <= 0.5 / 65535 + 1e-15)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_hilbert_matches_figure(golden_dir, p):
    seq = load_figure(golden_dir)[p]
    assert len(seq) == 4 ** p
    xs = np.array([c[0] for c in seq])
    ys = np.array([c[1] for c in seq])
    assert list(oracle.hilbert_code(xs, ys, bits=p)) == list(range(4 ** p))
    # the 16-bit curve refines the order-p one: its top 2p bits give the order-p index
    big = oracle.hilbert_code(xs << (16 - p), ys << (16 - p), bits=16)
    assert list(big >> np.uint32(2 * (16 - p))) == list(range(4 ** p))


@pytest.mark.parametrize("p", [4, 5])
def test_hilbert_is_a_continuous_bijection(p):
    g = 1 << p
    xs, ys = np.meshgrid(np.arange(g), np.arange(g), indexing="ij")
    c = oracle.hilbert_code(xs.ravel(), ys.ravel(), bits=p)
    assert sorted(c) == list(range(g * g))
    order = np.argsort(c)
    px, py = xs.ravel()[order], ys.ravel()[order]
    steps = np.abs(np.diff(px)) + np.abs(np.diff(py))
    assert np.all(steps == 1)                      # consecutive cells are grid neighbours
    assert (px[0], py[0]) == (0, 0) and (px[-1], py[-1]) == (g - 1, 0)


def test_morton_interleave():
    assert list(oracle.morton_code([0, 1, 0, 1], [0, 0, 1, 1])) == [0, 1, 2, 3]
    assert oracle.morton_code([65535], [0])[0] == 0x55555555
    assert oracle.morton_code([0], [65535])[0] == 0xAAAAAAAA
    # recursive Z shape on an 8 x 8 grid: quadrant order LL, LR, UL, UR at every level
    def z(x, y, m):
        if m == 0:
            return 0
        q = (1 if x >= m else 0) + (2 if y >= m else 0)
        return q * m * m + z(x % m, y % m, m // 2)
    for x in range(8):
        for y in range(8):
            assert oracle.morton_code([x], [y], bits=3)[0] == z(x, y, 4)


def test_sort_is_stable():
    codes = np.array([5, 3, 5, 1, 3, 5], dtype=np.uint32)
    assert list(oracle.sort_codes(codes)) == [3, 1, 4, 0, 2, 5]


def test_splitmix64_published_value():
    # first output of SplitMix64 from state 0 (Vigna's reference implementation)
    v = oracle.ordering._splitmix64(np.array([0], dtype=np.uint64))[0]
    assert int(v) == 0xE220A8397B1DCDAF
    k = oracle.random_keys(8, 3)
    assert list(k) == list(oracle.random_keys(8, 3))
    assert sorted(oracle.order(synth.jittered_grid(50), "random", 9)[0]) == list(range(50))


def test_kdtree_hand_made():
    x = np.array([0.9, 0.1, 0.5, 0.3])
    y = np.array([0.1, 0.2, 0.15, 0.12])
    assert list(oracle.kdtree_perm(x, y)) == [1, 3, 2, 0]
    # y has the larger range: split on y first
    x = np.array([0.1, 0.12, 0.11, 0.13, 0.1])
    y = np.array([0.9, 0.1, 0.5, 0.3, 0.7])
    # by y: 1(.1) 3(.3) 2(.5) 4(.7) 0(.9); left = first 3 = {1,3,2}, right = {4,0}
    # left {1,3,2}: ranges x .02, y .4 -> by y: 1,3 | 2 ; {1,3}: x .01 y .2 -> 1,3
    assert list(oracle.kdtree_perm(x, y)) == [1, 3, 2, 4, 0]
    # equal ranges: x wins
    x = np.array([0.0, 1.0, 0.0, 1.0])
    y = np.array([1.0, 0.0, 0.0, 1.0])
    assert list(oracle.kdtree_perm(x, y)) == [2, 0, 1, 3]


def kd_check(x, y, perm):
    """Brute-force check of Sec. 3.2 on an output order (independent of the builder)."""
    def check(seg):
        m = seg.size
        if m <= 1:
            return
        rx = x[seg].max() - x[seg].min()
        ry = y[seg].max() - y[seg].min()
        c = x if rx >= ry else y
        half = (m + 1) // 2
        left, right = seg[:half], seg[half:]
        assert c[left].max() <= c[right].min()
        check(left)
        check(right)
    check(np.asarray(perm))


@pytest.mark.parametrize("n", [1, 2, 3, 7, 37, 200])
def test_kdtree_rules(n):
    xy = synth.jittered_grid(n, seed=n)
    perm, _ = oracle.order(xy, "kdtree")
    assert sorted(perm) == list(range(n))
    kd_check(xy[:n], xy[n:], perm)


def maxmin_check(x, y, perm):
    n = x.size
    cx, cy = (x.min() + x.max()) * 0.5, (y.min() + y.max()) * 0.5
    d0 = [(x[i] - cx) ** 2 + (y[i] - cy) ** 2 for i in range(n)]
    assert perm[0] == min(range(n), key=lambda i: (d0[i], i))
    taken = [perm[0]]
    for k in range(1, n):
        rest = [i for i in range(n) if i not in taken]
        score = {i: min((x[i] - x[j]) ** 2 + (y[i] - y[j]) ** 2 for j in taken) for i in rest}
        best = max(score.values())
        assert perm[k] == min(i for i in rest if score[i] == best)
        taken.append(perm[k])


@pytest.mark.parametrize("n", [1, 2, 9, 30])
def test_maxmin_brute_force(n):
    xy = synth.jittered_grid(n, seed=100 + n)
    perm, _ = oracle.order(xy, "maxmin")
    maxmin_check(xy[:n], xy[n:], list(perm))


def test_maxmin_grid_ties():
    # exact 3x3 lattice: distances tie often; ties resolve to the lowest index
    g = np.arange(3) / 2.0
    xs, ys = np.meshgrid(g, g, indexing="ij")
    x, y = xs.ravel(), ys.ravel()
    perm = oracle.maxmin_perm(x, y)
    maxmin_check(x, y, list(perm))
    assert perm[0] == 4  # the centre


@pytest.mark.parametrize("method", list(oracle.NAMES))
def test_every_ordering_is_a_permutation(method):
    n = 257
    xy = synth.jittered_grid(n, seed=4)
    perm, codes = oracle.order(xy, method)
    assert perm.dtype == np.int64 and sorted(perm) == list(range(n))
    if codes is not None:
        assert np.all(np.diff(codes[perm].astype(np.int64)) >= 0)


def test_sfc_orders_are_local():
    # space-filling orders keep neighbours close: mean step much shorter than random
    n = 4096
    xy = synth.jittered_grid(n, seed=1)
    x, y = xy[:n], xy[n:]
    def mean_step(p):
        return np.mean(np.hypot(np.diff(x[p]), np.diff(y[p])))
    rnd = mean_step(oracle.order(xy, "random")[0])
    for m in ("morton", "hilbert", "kdtree"):
        assert mean_step(oracle.order(xy, m)[0]) < 0.1 * rnd
    # Hilbert steps between consecutive points stay ~one grid spacing
    assert mean_step(oracle.order(xy, "hilbert")[0]) < 2.0 / math.sqrt(n)
