"""The multi-GPU bench path is replicas only (one dataset per rank, no
collective on the data path); its host logic — distinct datasets per rank and
the max-over-ranks timing of the whole job — runs here on two gloo ranks."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # rank r pretends its 4 steps took 1000 (r + 1) ms
    value, total = bench.aggregate(1000.0 * (rank + 1), 4, world)
    q.put((rank, value, total, bench.dataset_seeds(rank)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_replicas_aggregate_max_time():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    out.sort()
    for rank, value, total, seeds in out:
        assert total == 2000.0                  # the slowest rank's time
        assert value == pytest.approx(2 * 4 / 2.0)
        assert seeds == (1 + rank, 2 + rank)    # a different dataset per replica
    assert out[0][3] != out[1][3]
