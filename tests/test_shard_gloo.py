"""Multi-rank host logic on CPU (gloo, world size 2): the row-slab partition of one image and
the timing aggregate a multi-GPU benchmark reduces (slowest rank's time, summed attempts and
rays).  No GPU: ranks are processes on this host."""
import os
import socket

import pytest

from paper_1601_02063_gb300 import shard
from paper_1601_02063_gb300 import workloads as W


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        out = shard.aggregate(10.0 + 2.5 * rank, 100.0 * (rank + 1), 7.0 + rank, dist)
        sc = shard.row_shard(W.torus_512(), rank, world)
        q.put((rank, out, sc["n_beta"], sc["beta_min"], sc["beta_max"]))
    finally:
        dist.destroy_process_group()


def test_two_rank_aggregate_and_shards_gloo():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    got.sort()
    for rank, out, nb, b0, b1 in got:
        assert out == (12.5, 300.0, 15.0), out  # max time, summed attempts and rays
    assert [g[2] for g in got] == [256, 256]
    assert got[0][3] == -20.0 and got[1][4] == 20.0 and got[0][4] == got[1][3] == 0.0


@pytest.mark.parametrize("n_beta,world", [(512, 2), (512, 3), (7, 4), (5, 8), (1, 1)])
def test_row_slabs_cover_the_image_with_its_pixel_centres(n_beta, world):
    sc = W.scene(n_alpha=3, n_beta=n_beta, beta_min=-13.0, beta_max=17.0)
    db = (sc["beta_max"] - sc["beta_min"]) / n_beta
    rows = []
    for r in range(world):
        j0, j1 = shard.row_range(n_beta, r, world)
        rows += list(range(j0, j1))
        s = shard.row_shard(sc, r, world)
        if j1 == j0:
            assert s is None
            continue
        sdb = (s["beta_max"] - s["beta_min"]) / s["n_beta"]
        for jj in range(s["n_beta"]):
            full = sc["beta_min"] + (j0 + jj + 0.5) * db
            mine = s["beta_min"] + (jj + 0.5) * sdb
            assert abs(full - mine) <= 1e-12 * max(1.0, abs(full))
    assert rows == list(range(n_beta))  # disjoint, ordered, complete
    sizes = [shard.row_range(n_beta, r, world) for r in range(world)]
    lens = [b - a for a, b in sizes]
    assert max(lens) - min(lens) <= 1


def test_aggregate_without_process_group_is_identity():
    assert shard.aggregate(3.0, 4.0, 5.0, None) == (3.0, 4.0, 5.0)
