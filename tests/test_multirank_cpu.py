"""Two-rank (gloo, CPU) tests of the multi-rank host logic: work-balanced source
shards whose partial rate fields sum to the single-rank result, and whole-job
throughput over the slowest rank."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2311_01492_gb300 import sharding as SH
from paper_2311_01492_gb300 import synth as S


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import oracle as O
    n = 16
    w = S.lognormal_box(n, 10.0, 24, 1e50, 1e53, radius=None)
    w["radius"] = np.minimum(w["radius"], 7.0)
    owner = SH.lpt_shards(w["radius"], world)
    mine = owner == rank
    tab = O.make_table("bb")
    part = O.raytrace(n, w["cell_cm"], w["nH"], w["xHI"], w["pos"][mine], w["ndot"][mine],
                      w["radius"][mine], tab)["gamma"]
    g = torch.tensor(part)
    SH.sum_rates(g, dist)
    ms, value = SH.aggregate(10.0 * (rank + 1), 100.0, dist)
    if rank == 0:
        full = O.raytrace(n, w["cell_cm"], w["nH"], w["xHI"], w["pos"], w["ndot"], w["radius"],
                          tab)["gamma"]
        q.put((g.numpy(), full, ms, value))
    dist.destroy_process_group()


def test_sharded_rates_sum_to_the_full_field():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got, full, ms, value = q.get(timeout=300)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    nz = full != 0
    assert np.array_equal(got != 0, nz)
    np.testing.assert_allclose(got[nz], full[nz], rtol=1e-13)
    assert ms == 20.0 and value == pytest.approx(200.0 / 0.02)


def test_lpt_shards_balance_work():
    R = 5.0 * (10 ** np.random.default_rng(1).uniform(0, 5, 10000) / 1.0) ** 0.2
    for world in (2, 4, 8):
        owner = SH.lpt_shards(R, world)
        loads = SH.shard_loads(R, owner, world)
        assert set(np.unique(owner)) == set(range(world))
        assert loads.max() / loads.mean() < 1.001
