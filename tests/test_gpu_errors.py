"""Failure reporting through the C ABI, triggered from the host (no GPU fault):
device-side check bits latched in the grid (injected) come back as
RT_ERR_BOUNDS from rt_check, rt_get_stats and the synchronising calls; a
process-wide device-memory cap makes the library's allocations fail with
RT_ERR_OOM and leaves the grid usable; call-order violations give
RT_ERR_STATE."""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2311_01492_gb300 import synth as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    from paper_2311_01492_gb300 import build
    build.build()
    from paper_2311_01492_gb300 import api as A
    return A


def _sources(n=24, nsrc=5):
    rng = np.random.default_rng(3)
    pos = torch.tensor(rng.integers(0, n, (nsrc, 3)), dtype=torch.int32, device="cuda")
    return (pos, torch.full((nsrc,), 1e50, dtype=torch.float64, device="cuda"),
            torch.full((nsrc,), 6.0, dtype=torch.float64, device="cuda"))


def _grid(api, n=24, nsrc=5):
    g = api.Grid(n, S.KPC_CM)
    g.set_tables("grey_exact")
    g.set_density(torch.full((n ** 3,), 1e-3, dtype=torch.float64, device="cuda"))
    g.set_xHI(torch.full((n ** 3,), 1e-4, dtype=torch.float64, device="cuda"))
    g.set_sources(*_sources(n, nsrc))
    return g


def test_latched_device_checks_are_reported(api):
    from paper_2311_01492_gb300 import _lib as L
    g = _grid(api)
    lib = L.lib()
    ref = g.raytrace().cpu().numpy()
    g.check()  # nothing latched
    for bits in (1, 2, 8, 1 | 8):
        assert lib.rt_inject_device_error(g._h, bits) == L.RT_OK
        st = lib.rt_check(g._h)
        assert st == L.RT_ERR_BOUNDS
        assert b"incomplete" in lib.rt_last_error()
        assert lib.rt_check(g._h) == L.RT_OK  # reported once, then cleared
    # the same through rt_get_stats and a synchronising call
    lib.rt_inject_device_error(g._h, 2)
    with pytest.raises(api.RtError, match="RT_ERR_BOUNDS"):
        g.stats()
    lib.rt_inject_device_error(g._h, 1)
    out = torch.empty(24 ** 3, dtype=torch.float64, device="cuda")
    assert lib.rt_raytrace_source_coldens(g._h, 0, C.c_void_p(out.data_ptr()), 2) == L.RT_ERR_BOUNDS
    # bad injection values are rejected; the grid still traces the same rates
    assert lib.rt_inject_device_error(g._h, 0) == L.RT_ERR_INVALID
    assert lib.rt_inject_device_error(g._h, 16) == L.RT_ERR_INVALID
    assert np.array_equal(g.raytrace().cpu().numpy(), ref)
    g.check()
    g.close()


def test_device_memory_cap_gives_out_of_memory(api):
    from paper_2311_01492_gb300 import _lib as L
    lib = L.lib()
    base = api.device_memory_in_use()
    g = _grid(api)
    held = api.device_memory_in_use()
    assert held > base
    ref = g.raytrace().cpu().numpy()
    try:
        api.set_device_memory_limit(held + 4096)
        # a new 64^3 grid needs several MB of fields: refused before cudaMalloc
        h = C.c_void_p()
        st = lib.rt_grid_create(C.byref(h), 64, S.KPC_CM, None, None)
        assert st == L.RT_ERR_OOM and not h.value
        assert api.device_memory_in_use() == held
        # more sources than the ingest buffers hold: refused; the grid then holds no
        # sources (zero rates) and takes a catalogue that fits again
        n = 24
        big = 200_000
        rng = np.random.default_rng(4)
        with pytest.raises(api.RtError, match="RT_ERR_OOM"):
            g.set_sources(torch.tensor(rng.integers(0, n, (big, 3)), dtype=torch.int32,
                                       device="cuda"),
                          torch.full((big,), 1e50, dtype=torch.float64, device="cuda"),
                          torch.full((big,), 3.0, dtype=torch.float64, device="cuda"))
        assert torch.count_nonzero(g.raytrace()).item() == 0
        g.set_sources(*_sources())
        assert np.array_equal(g.raytrace().cpu().numpy(), ref)
        g.check()
    finally:
        api.set_device_memory_limit(0)
    g2 = api.Grid(64, S.KPC_CM)  # no cap: fine
    g2.close()
    g.close()
    assert api.device_memory_in_use() == base


def test_call_order_violations(api):
    n = 8
    g = api.Grid(n, S.KPC_CM)
    with pytest.raises(api.RtError, match="RT_ERR_STATE"):
        g.raytrace()
    g.set_tables("grey_exact")
    with pytest.raises(api.RtError, match="RT_ERR_STATE"):
        g.raytrace()
    g.close()
