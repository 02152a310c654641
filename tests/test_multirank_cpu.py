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


def _bench_path_worker(rank, world, port, q):
    """The sharded step bench.py runs, with the oracle as each rank's tracer."""
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import oracle as O
    n = 16
    w = S.lognormal_box(n, 10.0, 30, 1e50, 1e53, radius=None)
    w["radius"] = np.minimum(w["radius"], 7.0)
    pos, ndot, R = SH.shard(w["pos"], w["ndot"], w["radius"], rank, world)
    tab = O.make_table("bb")
    x0 = np.zeros(n ** 3)
    dt = 5 * S.MYR_S

    def trace(gamma):
        gamma.copy_(torch.tensor(O.raytrace(n, w["cell_cm"], w["nH"], w["xHI"], pos, ndot, R,
                                            tab)["gamma"]))

    def chemistry(gamma):
        return O.chemistry(w["nH"], x0, x0, gamma.numpy(), dt)

    step = SH.ShardedStep(trace, chemistry, dist, world)
    gamma = torch.zeros(n ** 3, dtype=torch.float64)
    xa, xn, cnt = step(gamma)
    if rank == 0:
        full = O.raytrace(n, w["cell_cm"], w["nH"], w["xHI"], w["pos"], w["ndot"], w["radius"],
                          tab)["gamma"]
        xa_f, xn_f, cnt_f = O.chemistry(w["nH"], x0, x0, full, dt)
        q.put((len(pos), gamma.numpy(), full, xn, xn_f, cnt, cnt_f))
    else:
        q.put((len(pos),))
    dist.destroy_process_group()


def test_bench_sharded_step_matches_single_rank():
    """Each rank traces its longest-first share of the catalogue, the partial rate
    fields are summed (the one exchange of the paper's MPI mode, Sec. 3.2-3.3) and
    the chemistry runs on the sum: the same rates and ionised fractions as one rank
    tracing every source."""
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_bench_path_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    r0 = [r for r in res if len(r) > 1][0]
    nsrc_total = sum(r[0] for r in res)
    assert nsrc_total == 30 and all(r[0] > 0 for r in res)
    _, got, full, xn, xn_f, cnt, cnt_f = r0
    nz = full != 0
    assert np.array_equal(got != 0, nz)
    np.testing.assert_allclose(got[nz], full[nz], rtol=1e-13)
    np.testing.assert_allclose(xn, xn_f, rtol=1e-12, atol=1e-300)
    assert abs(cnt - cnt_f) <= 1
