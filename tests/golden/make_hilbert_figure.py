"""Write hilbert_figure.txt: the Hilbert-curve visit orders drawn in Figure 3 (Sec. 3.1.2).

Usage: python tests/golden/make_hilbert_figure.py <LaTeX source of the paper>

The figure is an inline TikZ drawing: one path segment per \\draw with a
`controls` clause, for the curves of order p = 1, 2 and 3 side by side.  The
drawn end points are hand placed (a few are off by a quarter cell), so each
is snapped to the nearest cell centre of its panel; the segments are then
chained into a path starting from the end at cell (0, 0).  Nothing here uses
the oracle or the CUDA path: the fixture is the paper's own data.
"""
import collections
import os
import re
import sys

# panel x-extent and cell-centre coordinates of the three drawings
PANELS = {
    1: ((0.0, 11.0), [1.25, 10.0], [4.25, 13.0]),
    2: ((11.0, 22.5), [12.5, 15.5, 18.25, 21.25], [4.25, 7.25, 10.0, 13.0]),
    3: ((22.5, 40.0), [23.75 + 1.25 * k for k in range(8)], [4.25 + 1.25 * k for k in range(8)]),
}


def segments(tex: str):
    out = []
    for line in tex.split("\n"):
        if "controls" in line and "short" in line:
            pts = re.findall(r"\(([\d.]+),([\d.]+)\)", line)
            out.append((tuple(map(float, pts[0])), tuple(map(float, pts[-1]))))
    return out


def nearest(v, grid):
    return min(range(len(grid)), key=lambda k: abs(v - grid[k]))


def visit_order(segs, p):
    (lo, hi), gx, gy = PANELS[p]
    adj = collections.defaultdict(set)
    for a, b in segs:
        if not lo <= a[0] < hi:
            continue
        ca = (nearest(a[0], gx), nearest(a[1], gy))
        cb = (nearest(b[0], gx), nearest(b[1], gy))
        adj[ca].add(cb)
        adj[cb].add(ca)
    assert len(adj) == 4 ** p
    seq, prev = [(0, 0)], None
    while len(seq) < 4 ** p:
        nxt = [c for c in adj[seq[-1]] if c != prev]
        assert len(nxt) == 1
        prev = seq[-1]
        seq.append(nxt[0])
    return seq


def main(src: str) -> None:
    segs = segments(open(src, encoding="utf-8").read())
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "hilbert_figure.txt")
    with open(path, "w") as f:
        f.write("# Visit order of the 2-d Hilbert curve of order p = 1, 2, 3, read off Figure 3\n")
        f.write("# (Sec. 3.1.2, the TikZ drawing adapted from Skilling 2004).  Cells are (x, y)\n")
        f.write("# with x to the right and y upwards, 0-based; the drawn segments were snapped\n")
        f.write("# to the nearest cell centre and chained from the end at cell (0, 0).\n")
        f.write("# Written by tests/golden/make_hilbert_figure.py from the paper's figure source.\n")
        for p in (1, 2, 3):
            f.write("p=%d " % p + " ".join("%d,%d" % c for c in visit_order(segs, p)) + "\n")


if __name__ == "__main__":
    main(sys.argv[1])
