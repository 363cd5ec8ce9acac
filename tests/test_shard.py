"""Sharding the batched workload by dataset (no collective on the data path).

tlr_shard_place (host only) puts the largest footprint first onto the
least-loaded rank with room; every rank computes the same placement.  Checked
against its definition on small cases, against the longest-processing-time
bound (heaviest rank <= 4/3 of the optimum's lower bound), for budgets, and on
two gloo ranks with the bench's own placement and throughput aggregation.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def place(fp, nranks, budget=None):
    import paper_2402_09356_gb300 as tlr
    return tlr.tlr_shard_place(fp, nranks, budget)


def test_place_small_cases_by_hand():
    # sorted 9, 7, 5, 4, 3 (index order on ties) onto 2 ranks:
    # 9 -> r0; 7 -> r1; 5 -> r1 (7 < 9); 4 -> r0 (9 < 12); 3 -> r1 (12 < 13)
    fp = [5, 9, 3, 7, 4]
    got = place(fp, 2)
    assert list(got) == [1, 0, 1, 1, 0]
    loads = [sum(f for f, r in zip(fp, got) if r == k) for k in range(2)]
    assert loads == [13, 15]
    # ties: equal footprints go to the lower index first and to the lower rank
    assert list(place([4, 4, 4], 3)) == [0, 1, 2]
    assert list(place([], 2)) == []


def test_place_lpt_bound_and_cover():
    rng = np.random.default_rng(7)
    for nranks in (2, 3, 4, 8):
        fp = rng.integers(1, 10 ** 9, 256)
        got = place(fp, nranks)
        assert set(got) <= set(range(nranks))
        loads = np.bincount(got, weights=fp, minlength=nranks)
        lower = max(fp.sum() / nranks, fp.max())
        assert loads.max() <= 4.0 / 3.0 * lower + 1


def test_place_respects_budgets():
    import paper_2402_09356_gb300 as tlr
    fp = [10, 10, 10, 10]
    got = place(fp, 2, budget=[30, 10])
    loads = np.bincount(got, weights=fp, minlength=2)
    assert loads[0] <= 30 and loads[1] <= 10
    with pytest.raises(tlr.TlrError) as e:
        place(fp, 2, budget=[15, 15])
    assert e.value.code == tlr.TLR_ERR_OOM
    with pytest.raises(tlr.TlrError) as e:
        place([1, -1], 2)
    assert e.value.code == tlr.TLR_ERR_ARG


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sizes, _ = bench.batched_datasets(256)
    rank_of, fp = bench.shard_batched(sizes, world)
    everyone = [None] * world
    dist.all_gather_object(everyone, [int(r) for r in rank_of])
    mine = [i for i in range(len(sizes)) if rank_of[i] == rank]
    # rank r pretends its evaluations took 10 (r + 1) s
    rate, units, secs = bench.aggregate_units(len(mine), 10.0 * (rank + 1), world)
    q.put((rank, everyone, mine, [int(f) for f in fp], rate, units, secs))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_sharded_batched_workload():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=180) for _ in range(world))
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    (_, ev0, mine0, fp, rate, units, secs), (_, ev1, mine1, _, rate1, _, _) = out
    assert ev0[0] == ev0[1] == ev1[0]                  # one placement, computed by each rank alone
    assert sorted(mine0 + mine1) == list(range(256))   # disjoint and complete
    loads = [sum(fp[i] for i in m) for m in (mine0, mine1)]
    assert max(loads) <= 4.0 / 3.0 * max(sum(fp) / 2, max(fp)) + 1
    assert units == 256 and secs == 20.0 and rate == pytest.approx(256 / 20.0) and rate1 == rate
