"""The allocation-free column-density entry point (rt_coldens_single_noalloc).

Some callers cannot allocate device memory at the moment they call the
library -- while someone else captures a CUDA graph, inside frameworks that
reserve all device memory at start-up, or in loops that cannot take an
allocation's implicit synchronisation.  This entry point serves them with a
fixed scratch array, and must give the same column densities, bit for bit, as
the allocating entry point rt_raytrace_source_coldens and as the CPU oracle,
also when called several times in a row (the scratch array keeps the previous
call's contents).  The cases cover an even and an odd box, a radius beyond the
periodic window (clipped traversal with wrap-around) and the largest accepted
traced half-extent (40 cells).  Collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2311_01492_gb300 import synth as S

pytestmark = pytest.mark.gpu

CELL = 0.78125 * S.MPC_CM


def _lib():
    from paper_2311_01492_gb300 import build
    build.build()
    from paper_2311_01492_gb300 import _lib
    return _lib


def _fields(n, seed):
    nH = S.lognormal_field(n, 2e-4, seed=seed)
    xHI = S.uniform_xhi(n, seed=seed + 1)
    return nH, xHI


def _noalloc(L, n, nH_d, xHI_d, src, R, out):
    from paper_2311_01492_gb300 import api
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = L.lib().rt_coldens_single_noalloc(n, CELL, api.SIGMA0, C.c_void_p(nH_d.data_ptr()),
                                           C.c_void_p(xHI_d.data_ptr()), src[0], src[1], src[2], R,
                                           C.c_void_p(out.data_ptr()), stream)
    L.check(st, "rt_coldens_single_noalloc")
    return out.cpu().numpy()


# (n, [(source cell, radius), ...]): an even box (two calls, the second smaller), an odd
# box, radii beyond the window (traversal clipped at the window and wrapped), and the
# largest traced half-extent the scratch holds (min(floor(R), n/2) = 40)
CASES = [(40, [((5, 33, 12), 17.5), ((20, 20, 39), 9.0)]),
         (37, [((0, 36, 18), 12.3), ((36, 0, 1), 18.0)]),
         (30, [((3, 27, 14), 25.0), ((29, 29, 29), 40.0)]),
         (80, [((7, 70, 41), 45.0)]),
         (81, [((80, 1, 40), 52.5)])]


@pytest.mark.parametrize("n,srcs", CASES)
def test_noalloc_column_density_matches_allocating_entry_point_and_oracle(n, srcs):
    L = _lib()
    from paper_2311_01492_gb300 import api
    nH, xHI = _fields(n, 77 + n)
    dev = dict(device="cuda", dtype=torch.float64)
    nH_d = torch.tensor(nH.reshape(-1), **dev)
    xHI_d = torch.tensor(xHI.reshape(-1), **dev)
    g = api.Grid(n, CELL)
    g.set_tables("grey_exact")
    g.set_density(nH_d)
    g.set_xHI(xHI_d)
    g.set_sources(torch.tensor([p for p, _ in srcs], device="cuda", dtype=torch.int32),
                  torch.full((len(srcs),), 1e52, **dev),
                  torch.tensor([r for _, r in srcs], **dev))
    ref = [g.source_coldens(s).cpu().numpy() for s in range(len(srcs))]
    g.close()
    tab = O.make_table("grey_exact")
    out = torch.full((n ** 3,), -1.0, **dev)
    for rep in range(2):  # twice in a row: the shared scratch keeps the last call's contents
        for (p, R), want in zip(srcs, ref):
            got = _noalloc(L, n, nH_d, xHI_d, p, R, out)
            assert np.count_nonzero(got) > 0
            assert np.array_equal(got, want), "differs from rt_raytrace_source_coldens"
            if rep == 0:
                ro = O.raytrace(n, CELL, nH, xHI, [p], [1e52], [R], tab, gamma=False,
                                coldens_src=0)["coldens"]
                assert np.array_equal(got, ro), "differs from the oracle"


def test_noalloc_call_takes_no_device_memory():
    """After the first call on a device (which looks up the scratch array's address),
    a call leaves the device's free memory unchanged."""
    L = _lib()
    n = 40
    nH, xHI = _fields(n, 91)
    dev = dict(device="cuda", dtype=torch.float64)
    nH_d = torch.tensor(nH.reshape(-1), **dev)
    xHI_d = torch.tensor(xHI.reshape(-1), **dev)
    out = torch.empty(n ** 3, **dev)
    first = _noalloc(L, n, nH_d, xHI_d, (1, 2, 3), 30.0, out)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    used0 = L.lib().rt_device_memory_in_use()
    again = _noalloc(L, n, nH_d, xHI_d, (1, 2, 3), 30.0, out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert L.lib().rt_device_memory_in_use() == used0
    assert np.array_equal(first, again)


def test_noalloc_rejects_cubes_beyond_its_fixed_scratch():
    L = _lib()
    n = 128
    x = torch.zeros(n ** 3, device="cuda", dtype=torch.float64)
    st = L.lib().rt_coldens_single_noalloc(n, 1e24, 6.3e-18, C.c_void_p(x.data_ptr()),
                                           C.c_void_p(x.data_ptr()), 1, 2, 3, 60.0,
                                           C.c_void_p(x.data_ptr()), None)
    assert st == L.RT_ERR_INVALID
    assert b"exceeds the fixed scratch limit" in L.lib().rt_last_error()
    # half-extent 41 from the window (n = 82, R = 60): also refused, nothing launched
    n = 82
    x = torch.zeros(n ** 3, device="cuda", dtype=torch.float64)
    st = L.lib().rt_coldens_single_noalloc(n, 1e24, 6.3e-18, C.c_void_p(x.data_ptr()),
                                           C.c_void_p(x.data_ptr()), 1, 2, 3, 60.0,
                                           C.c_void_p(x.data_ptr()), None)
    assert st == L.RT_ERR_INVALID
    assert torch.count_nonzero(x).item() == 0
