"""Factor storage plans (host logic, no GPU): uniform slots hold nb * maxrank
columns per off-diagonal tile, as many doubles as the dense lower tiles at
maxrank = nb / 2; compact slots from a rank map hold r + max(8, r / 4)
columns rounded up to 8 (at most maxrank) plus an overflow area of
max(sum / 8, 4 maxrank) columns."""
import numpy as np
import pytest

import paper_2402_09356_gb300 as tlr
from paper_2402_09356_gb300 import build as tlr_build


@pytest.fixture(scope="module", autouse=True)
def lib():
    tlr_build.build()
    return tlr.load_library()


def plan(n, nb, maxrank, rmap=None):
    nt = -(-n // nb)
    noff = nt * (nt - 1) // 2
    if rmap is None:
        cols = max(noff, 1) * maxrank
    else:
        caps = [min(maxrank, (r + max(8, r // 4) + 7) // 8 * 8) for i in range(nt) for j in range(i)
                for r in [max(0, int(rmap[i, j]))]]
        cols = max(sum(caps) + max(sum(caps) // 8, 4 * maxrank), 1)
    return (nt * nb * nb + 2 * cols * nb) * 8 + nt * nt * 4


def test_uniform_plan_is_dense_sized():
    n, nb = 40000, 800
    b = tlr.tlr_mat_plan_bytes(n, nb)
    assert b == plan(n, nb, nb // 2)
    nt = n // nb
    dense_lower = nt * (nt - 1) // 2 * nb * nb * 8
    assert b - nt * nb * nb * 8 - nt * nt * 4 == dense_lower


@pytest.mark.parametrize("seed", range(4))
def test_compact_plan(seed):
    rng = np.random.default_rng(seed)
    n, nb, maxrank = int(rng.integers(2000, 30000)), int(rng.choice([128, 256, 800])), 0
    nt = -(-n // nb)
    rmap = np.zeros((nt, nt), dtype=np.int32)
    for i in range(nt):
        for j in range(i):
            rmap[i, j] = rmap[j, i] = min(nb // 2, int(rng.exponential(20)) + (60 if i == j + 1 else 0))
    got = tlr.tlr_mat_plan_bytes(n, nb, maxrank, rmap)
    assert got == plan(n, nb, nb // 2, rmap)
    assert got < tlr.tlr_mat_plan_bytes(n, nb)


def test_plan_rejects_bad_sizes():
    assert tlr.tlr_mat_plan_bytes(0, 256) == -1
    assert tlr.tlr_mat_plan_bytes(1000, 8) == -1
    assert tlr.tlr_mat_plan_bytes(1000, 256, 300) == -1
