"""World-size-2 gloo tests (CPU) of the replica logic used by bench.py for
N > 1 GPUs: sharding, distinct seeds, max-over-ranks timing and the combined
log-det estimate."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1312_1476_gb300 import replicas


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = replicas.max_over_ranks(1.5 + rank, dist)
        start, stop = replicas.shard(10, rank, world)
        qs = np.arange(start, stop, dtype=np.float64) ** 2
        est, se, n = replicas.combine_logdet(qs, shift=3.0, dist=dist)
        q.put((rank, t, (start, stop), est, se, n, replicas.replica_seed(7, rank)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    all_q = np.arange(10, dtype=np.float64) ** 2
    for rank, t, (start, stop), est, se, n, seed in out:
        assert t == 2.5                                  # max over ranks
        assert n == 10
        assert abs(est - (all_q.mean() + 3.0)) < 1e-12   # same global estimate on every rank
        assert abs(se - all_q.std(ddof=1) / np.sqrt(10)) < 1e-12
    assert [o[2] for o in out] == [(0, 5), (5, 10)]
    assert out[0][6] != out[1][6]


@pytest.mark.parametrize("count,world", [(10, 3), (1, 4), (0, 2), (7, 7)])
def test_shard_covers_units(count, world):
    got = [replicas.shard(count, r, world) for r in range(world)]
    assert got[0][0] == 0 and got[-1][1] == count
    for (a, b), (c, d) in zip(got, got[1:]):
        assert b == c and b >= a
    sizes = [b - a for a, b in got]
    assert max(sizes) - min(sizes) <= 1


def test_single_process_paths():
    assert replicas.max_over_ranks(3.0) == 3.0
    est, se, n = replicas.combine_logdet([1.0, 3.0], 0.5)
    assert est == 2.5 and n == 2 and abs(se - 1.0) < 1e-12
