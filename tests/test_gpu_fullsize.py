"""Parity at the benchmark workloads' full sizes, in the launch configuration
the benchmark times (autotuned batched schedule): the complete rate field of
the 128^3 / 1e4-source and 250^3 / 1e6-source workloads against the OpenMP
oracle (identical zero pattern, 1e-9 relative), per-source column densities of
sampled sources (bit for bit), the full rate field of every other schedule
(plain, early exit), every box of the 64-box ensemble traced in one launch,
and the adjoint at 250^3 with 1e5 sources on sampled sources and cells."""
import os

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2311_01492_gb300 import synth as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2311_01492_gb300 import build
    build.build()


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda").to(dtype).contiguous()


def rel_ok(a, b, rtol):
    assert np.array_equal(a != 0, b != 0)
    nz = b != 0
    if nz.any():
        r = np.abs(a[nz] - b[nz]) / np.abs(b[nz])
        assert r.max() <= rtol, r.max()


CORES = max(1, len(os.sched_getaffinity(0)))


def check_workload(w, n_cd=6, autotune=True, plain=True):
    from paper_2311_01492_gb300 import api
    n, cell = w["n"], w["cell_cm"]
    tab = O.make_table("bb", 5e4)
    g = api.Grid(n, cell)
    g.set_tables("knots", g=tab.g, h=tab.h)
    g.set_density(dev(w["nH"].reshape(-1)))
    g.set_xHI(dev(w["xHI"].reshape(-1)))
    g.set_sources(dev(w["pos"], torch.int32), dev(w["ndot"]), dev(w["radius"]))
    if autotune:
        g.autotune()
    full = g.raytrace(schedule="batched").cpu().numpy()
    g.stats()
    if plain:
        rel_ok(g.raytrace(schedule="plain").cpu().numpy(), full, 1e-12)
    rel_ok(g.raytrace(schedule="early_exit").cpu().numpy(), full, 1e-12)
    # per-source column densities: the largest, the smallest and random sources
    rng = np.random.default_rng(5)
    R = w["radius"]
    picks = [int(np.argmax(R)), int(np.argmin(R))] + list(rng.choice(len(R), n_cd - 2, replace=False))
    for s in picks:
        cd = g.source_coldens(int(s)).cpu().numpy()
        ro = O.raytrace(n, cell, w["nH"], w["xHI"], w["pos"][s:s + 1], w["ndot"][s:s + 1],
                        R[s:s + 1], tab, gamma=False, coldens_src=0)["coldens"]
        assert np.array_equal(cd, ro), "source %d" % s
    # the complete rate field against the oracle (every source, every cell)
    go = O.raytrace(n, cell, w["nH"], w["xHI"], w["pos"], w["ndot"], R, tab,
                    nthreads=CORES)["gamma"]
    rel_ok(full, go, 1e-9)
    g.stats()
    g.close()


def test_box128_1e4_sources():
    check_workload(S.box128_1e4())


def test_box250_1e6_sources_bench_configuration():
    check_workload(S.box250_1e6(), n_cd=6)


def test_ensemble_of_64_boxes_every_box():
    from paper_2311_01492_gb300 import api
    boxes = S.ensemble(64)
    sizes = [b["n"] for b in boxes]
    assert set(sizes) == {32, 48, 64, 96, 128}
    cell = boxes[0]["cell_cm"]
    tab = O.make_table("bb", 5e4)
    g = api.Grid.ensemble(sizes, cell)
    g.set_tables("knots", g=tab.g, h=tab.h)
    g.set_density(dev(np.concatenate([b["nH"].reshape(-1) for b in boxes])))
    g.set_xHI(dev(np.concatenate([b["xHI"].reshape(-1) for b in boxes])))
    g.set_sources(dev(np.concatenate([b["pos"] for b in boxes]), torch.int32),
                  dev(np.concatenate([b["ndot"] for b in boxes])),
                  dev(np.concatenate([b["radius"] for b in boxes])),
                  dev(np.concatenate([np.full(len(b["pos"]), i) for i, b in enumerate(boxes)]),
                      torch.int32))
    g.autotune()
    gam = g.raytrace(schedule="batched").cpu().numpy()
    g.stats()
    offs = np.concatenate([[0], np.cumsum([n ** 3 for n in sizes])])
    for b, bx in enumerate(boxes):  # every box, traced by the oracle in full
        ref = O.raytrace(bx["n"], cell, bx["nH"], bx["xHI"], bx["pos"], bx["ndot"], bx["radius"],
                         tab, nthreads=CORES)["gamma"]
        rel_ok(gam[offs[b]:offs[b + 1]], ref, 1e-9)
    g.close()


def test_adjoint_box250_1e5_sources_sampled():
    """The gradient-throughput workload of the benchmark (250^3, 1e5 sources of the
    1e6 catalogue, blackbody chords, weights ~ N(0,1)): dL/dlog Ndot of 32 sampled
    sources against the linearity closed form sum_p w_p Gamma_sp of the oracle's
    single-source fields, and dL/dlog n_HI of 8 cells next to sources against the
    oracle's complex-step derivative (only sources whose traced region holds the
    cell contribute)."""
    from paper_2311_01492_gb300 import api
    w = S.box250_1e6()
    n, cell = w["n"], w["cell_cm"]
    rng = np.random.default_rng(11)
    sel = np.sort(rng.choice(len(w["ndot"]), size=100_000, replace=False))
    pos, ndot, R = w["pos"][sel], w["ndot"][sel], w["radius"][sel]
    wl = S.loss_weights(n ** 3)
    tab = O.make_table("bb", 5e4)
    g = api.Grid(n, cell)
    g.set_tables("knots", g=tab.g, h=tab.h)
    g.set_density(dev(w["nH"].reshape(-1)))
    g.set_xHI(dev(w["xHI"].reshape(-1)))
    g.set_sources(dev(pos, torch.int32), dev(ndot), dev(R))
    g.autotune()
    dn, dq = g.backward(dev(wl))
    dn, dq = dn.cpu().numpy(), dq.cpu().numpy()
    g.stats()
    g.close()
    # dL/dlog Ndot_s = sum_p w_p Gamma_sp (Gamma is linear in Ndot_s)
    picks = rng.choice(len(ndot), size=32, replace=False)
    for s in picks:
        gs = O.raytrace(n, cell, w["nH"], w["xHI"], pos[s:s + 1], ndot[s:s + 1], R[s:s + 1], tab,
                        nthreads=CORES)["gamma"]
        want = float(np.dot(wl, gs))
        scale = float(np.dot(np.abs(wl), gs))
        assert scale > 0
        assert abs(dq[s] - want) <= 1e-12 * scale, (s, dq[s], want, scale)
    # dL/dlog n_HI next to sampled sources (the gradient vanishes far from them)
    near = []
    for s, off in zip(rng.choice(len(ndot), size=8, replace=False),
                      [(1, 0, 0), (0, -1, 0), (0, 0, 2), (1, 1, 0), (-1, 0, 1), (2, -1, 0),
                       (0, 1, 1), (-1, -1, -1)]):
        c = [(int(pos[s][k]) + off[k]) % n for k in range(3)]
        near.append((c[0] * n + c[1]) * n + c[2])
    cells = np.array(near, dtype=np.int64)
    dn_o, _ = O.loss_grad_cs(n, cell, w["nH"], w["xHI"], pos, ndot, R, tab, wl, cells,
                             np.zeros(0, dtype=np.int32), nthreads=CORES)
    scale = np.abs(dn_o).max()
    assert scale > 0
    np.testing.assert_allclose(dn[cells], dn_o, rtol=1e-9, atol=1e-12 * scale)
