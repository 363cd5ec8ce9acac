"""Oracle: spatial orderings of Sec. 3.  Test infrastructure only.

Every ordering returns a permutation `perm` (int64): position k of the
ordered problem holds original location perm[k].  Readings of the paper where
the text leaves a choice open:

* Quantisation (Sec. 3.1, "Encoding"): each coordinate, clamped to [0, 1],
  is multiplied by 65535 (the largest 16-bit unsigned value) in one FP64
  multiply and rounded to the nearest integer, ties to even.
* Morton (Sec. 3.1.1): the 32-bit code interleaves the bits of the two
  16-bit integers; bit 2k of the code is bit k of x, bit 2k+1 is bit k of y.
* Hilbert (Sec. 3.1.2, Figure 3): the orientation drawn in the figure: the
  order-p curve starts in cell (0, 0), ends in cell (2^p - 1, 0) and visits
  the quadrants lower-left, upper-left, upper-right, lower-right.  Codes use
  p = 16.
* Sorting (Sec. 3.1, "Sorting"): a stable sort of the codes, so that equal
  codes keep the original index order (the paper's quicksort is not stable;
  the total order (code, index) makes the result unique).
* KD-tree (Sec. 3.2): split on the dimension of largest range (x on a tie)
  at the median; after sorting the node's points by (coordinate, index) the
  first ceil(m/2) go left, which is exactly "<= median goes left" whenever
  the coordinates are distinct; in-order traversal of the leaves.
* Max-min (Sec. 3.3.1 cites Guinness 2018): the maximum-minimum-distance
  ordering: start at the point nearest the centre of the bounding box, then
  repeatedly take the point whose smallest squared distance to the points
  already taken is largest; ties go to the lowest index.  Squared distances
  are dx*dx + dy*dy with every operation rounded separately.
* Random ("no order" in Sec. 5 is the generation order, IDENTITY here):
  RANDOM sorts the keys splitmix64(seed XOR i) >> 32, stably.
"""
from __future__ import annotations

import math

import numpy as np

IDENTITY, RANDOM, MORTON, HILBERT, KDTREE, MAXMIN = 0, 1, 2, 3, 4, 5
NAMES = {"identity": IDENTITY, "random": RANDOM, "morton": MORTON,
         "hilbert": HILBERT, "kdtree": KDTREE, "maxmin": MAXMIN}

_U64 = np.uint64


def quantize(v: np.ndarray) -> np.ndarray:
    """Sec. 3.1 "Encoding": round(clamp(v, 0, 1) * 65535) as uint32 values in [0, 65535]."""
    c = np.clip(np.asarray(v, dtype=np.float64), 0.0, 1.0)
    return np.rint(c * 65535.0).astype(np.uint32)


def dequantize(q: np.ndarray) -> np.ndarray:
    """Sec. 3.1 "Decoding": the integer coordinate divided by 65535."""
    return np.asarray(q, dtype=np.float64) / 65535.0


def morton_code(qx: np.ndarray, qy: np.ndarray, bits: int = 16) -> np.ndarray:
    """Sec. 3.1.1: interleave the binary digits of the two integer coordinates."""
    qx = np.asarray(qx, dtype=np.uint64)
    qy = np.asarray(qy, dtype=np.uint64)
    code = np.zeros(qx.shape, dtype=np.uint64)
    for k in range(bits):
        code |= ((qx >> _U64(k)) & _U64(1)) << _U64(2 * k)
        code |= ((qy >> _U64(k)) & _U64(1)) << _U64(2 * k + 1)
    return code.astype(np.uint32)


def hilbert_code(qx: np.ndarray, qy: np.ndarray, bits: int = 16) -> np.ndarray:
    """Sec. 3.1.2: position of cell (qx, qy) along the order-`bits` Hilbert curve.

    Recursive definition, applied from the top level down.  At a level with
    half-width M the cell lies in quadrant q (0 lower-left, 1 upper-left,
    2 upper-right, 3 lower-right), which contributes q * M^2, and the cell is
    mapped into the frame in which that quadrant's sub-curve has the standard
    orientation (start (0,0), end (M-1,0)):
      lower-left  (x, y) -> (y, x)                (transpose)
      upper-left  (x, y) -> (x, y - M)
      upper-right (x, y) -> (x - M, y - M)
      lower-right (x, y) -> (M-1-y, 2M-1-x)       (anti-transpose)
    """
    x = np.asarray(qx, dtype=np.int64).copy()
    y = np.asarray(qy, dtype=np.int64).copy()
    d = np.zeros(x.shape, dtype=np.int64)
    m = 1 << (bits - 1)
    while m >= 1:
        right = x >= m
        up = y >= m
        ll = ~right & ~up
        ul = ~right & up
        ur = right & up
        lr = right & ~up
        q = np.where(ll, 0, np.where(ul, 1, np.where(ur, 2, 3)))
        d += q * m * m
        nx = np.where(ll, y, np.where(ul, x, np.where(ur, x - m, m - 1 - y)))
        ny = np.where(ll, x, np.where(ul, y - m, np.where(ur, y - m, 2 * m - 1 - x)))
        x, y = nx, ny
        m //= 2
    return d.astype(np.uint32)


def _splitmix64(v: np.ndarray) -> np.ndarray:
    """SplitMix64 output for state v (Steele, Lea, Flood 2014; Vigna's constants)."""
    z = np.asarray(v, dtype=np.uint64) + _U64(0x9E3779B97F4A7C15)
    z = (z ^ (z >> _U64(30))) * _U64(0xBF58476D1CE4E5B9)
    z = (z ^ (z >> _U64(27))) * _U64(0x94D049BB133111EB)
    return z ^ (z >> _U64(31))


def random_keys(n: int, seed: int) -> np.ndarray:
    """Keys of the RANDOM ordering: splitmix64(seed XOR i) >> 32 as uint32."""
    i = np.arange(n, dtype=np.uint64)
    return (_splitmix64(_U64(seed & 0xFFFFFFFFFFFFFFFF) ^ i) >> _U64(32)).astype(np.uint32)


def sort_codes(codes: np.ndarray) -> np.ndarray:
    """Sec. 3.1 "Sorting": stable sort, so ties keep the original index order."""
    return np.argsort(codes, kind="stable").astype(np.int64)


def kdtree_perm(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """Sec. 3.2: build the KD-tree (steps 1-4) and list its leaves in order."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    out = []

    def build(idx: np.ndarray) -> None:
        m = idx.size
        if m == 1:
            out.append(int(idx[0]))
            return
        xs, ys = x[idx], y[idx]
        rx = xs.max() - xs.min()
        ry = ys.max() - ys.min()
        c = xs if rx >= ry else ys          # step 1: dimension of largest range
        srt = idx[np.lexsort((idx, c))]     # by coordinate, then by index
        half = (m + 1) // 2                 # step 2: <= median goes left
        build(srt[:half])                   # step 3: left sub-tree first
        build(srt[half:])

    if x.size:
        build(np.arange(x.size, dtype=np.int64))
    return np.array(out, dtype=np.int64)


def maxmin_perm(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """Maximum-minimum-distance ordering (Sec. 3.3.1, after Guinness 2018)."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    n = x.size
    perm = np.empty(n, dtype=np.int64)
    if n == 0:
        return perm
    cx = (x.min() + x.max()) * 0.5
    cy = (y.min() + y.max()) * 0.5
    dx = x - cx
    dy = y - cy
    p = int(np.argmin(dx * dx + dy * dy))   # first occurrence: lowest index
    mind = np.full(n, np.inf)
    for k in range(n):
        perm[k] = p
        mind[p] = -1.0                      # taken
        dx = x - x[p]
        dy = y - y[p]
        dd = dx * dx + dy * dy
        np.minimum(mind, dd, out=mind)      # taken points stay at -1
        p = int(np.argmax(mind))
    return perm


def order(xy: np.ndarray, method, seed: int = 3):
    """Permutation (and the 32-bit codes, where the method has them) for SoA locations.

    Returns (perm, codes); codes is None for IDENTITY, KDTREE and MAXMIN.
    """
    if isinstance(method, str):
        method = NAMES[method]
    xy = np.asarray(xy, dtype=np.float64)
    n = xy.size // 2
    x, y = xy[:n], xy[n:]
    if method == IDENTITY:
        return np.arange(n, dtype=np.int64), None
    if method == RANDOM:
        codes = random_keys(n, seed)
        return sort_codes(codes), codes
    if method in (MORTON, HILBERT):
        qx, qy = quantize(x), quantize(y)
        codes = morton_code(qx, qy) if method == MORTON else hilbert_code(qx, qy)
        return sort_codes(codes), codes
    if method == KDTREE:
        return kdtree_perm(x, y), None
    if method == MAXMIN:
        return maxmin_perm(x, y), None
    raise ValueError("unknown ordering %r" % (method,))


def decode_xy(xy: np.ndarray) -> np.ndarray:
    """Sec. 3.1 "Decoding": coordinates replaced by their quantised values / 65535."""
    n = xy.size // 2
    return np.concatenate([dequantize(quantize(xy[:n])), dequantize(quantize(xy[n:]))])


def n_tiles(n: int, nb: int) -> int:
    return int(math.ceil(n / nb)) if n else 0
