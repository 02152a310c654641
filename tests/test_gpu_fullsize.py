"""Parity at the benchmark workloads' full sizes, on outputs the oracle can
compute one by one: per-source column densities of sampled sources (bit for
bit) and the rates of random subsets of the sources (1e-9), in the launch
configuration the benchmark times (autotuned batched schedule).  The full
rate field is also compared between schedules (batched, plain, early exit)."""
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


def check_workload(w, n_cd=6, n_sub=150, autotune=True, plain=True):
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
    # rates of a random subset of the sources, same grid
    sub = np.sort(rng.choice(len(R), min(n_sub, len(R)), replace=False))
    g.set_sources(dev(w["pos"][sub], torch.int32), dev(w["ndot"][sub]), dev(R[sub]))
    gs = g.raytrace(schedule="batched").cpu().numpy()
    go = O.raytrace(n, cell, w["nH"], w["xHI"], w["pos"][sub], w["ndot"][sub], R[sub], tab,
                    nthreads=16)["gamma"]
    rel_ok(gs, go, 1e-9)
    g.stats()
    g.close()


def test_box128_1e4_sources():
    check_workload(S.box128_1e4())


def test_box250_1e6_sources_bench_configuration():
    check_workload(S.box250_1e6(), n_cd=6, n_sub=120)


def test_ensemble_of_64_boxes_sampled():
    from paper_2311_01492_gb300 import api
    boxes = S.ensemble(64)
    sizes = [b["n"] for b in boxes]
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
    # the three boxes with the fewest sources, traced by the oracle in full
    for b in np.argsort([len(bx["pos"]) for bx in boxes])[:3]:
        bx = boxes[b]
        ref = O.raytrace(bx["n"], cell, bx["nH"], bx["xHI"], bx["pos"], bx["ndot"], bx["radius"],
                         tab, nthreads=16)["gamma"]
        rel_ok(gam[offs[b]:offs[b + 1]], ref, 1e-9)
    g.close()
