"""The allocation-free column-density entry point (rt_coldens_single_noalloc).

It exists for callers that cannot allocate device memory at call time; it
must give the same column densities, bit for bit, as the allocating entry
point rt_raytrace_source_coldens, also when called twice in a row (the fixed
scratch array keeps the previous call's contents).  Collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2311_01492_gb300 import synth as S

pytestmark = pytest.mark.gpu


def _lib():
    from paper_2311_01492_gb300 import build
    build.build()
    from paper_2311_01492_gb300 import _lib
    return _lib


def test_noalloc_column_density_matches_allocating_entry_point():
    L = _lib()
    from paper_2311_01492_gb300 import api
    n = 40
    cell = 0.78125 * S.MPC_CM
    nH = torch.tensor(S.lognormal_field(n, 2e-4, seed=77).reshape(-1), device="cuda",
                      dtype=torch.float64)
    xHI = torch.tensor(S.uniform_xhi(n, seed=78).reshape(-1), device="cuda", dtype=torch.float64)
    srcs = [((5, 33, 12), 17.5), ((20, 20, 39), 9.0)]  # the second call traces a smaller cube
    g = api.Grid(n, cell)
    g.set_tables("grey_exact")
    g.set_density(nH)
    g.set_xHI(xHI)
    g.set_sources(torch.tensor([p for p, _ in srcs], device="cuda", dtype=torch.int32),
                  torch.tensor([1e52, 1e51], device="cuda", dtype=torch.float64),
                  torch.tensor([r for _, r in srcs], device="cuda", dtype=torch.float64))
    ref = [g.source_coldens(s).cpu().numpy() for s in range(len(srcs))]
    out = torch.full((n ** 3,), -1.0, device="cuda", dtype=torch.float64)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for (p, R), want in zip(srcs, ref):
        st = L.lib().rt_coldens_single_noalloc(n, cell, api.SIGMA0, C.c_void_p(nH.data_ptr()),
                                               C.c_void_p(xHI.data_ptr()), p[0], p[1], p[2], R,
                                               C.c_void_p(out.data_ptr()), stream)
        L.check(st, "rt_coldens_single_noalloc")
        got = out.cpu().numpy()
        assert np.count_nonzero(got) > 0
        assert np.array_equal(got, want), "column density differs from rt_raytrace_source_coldens"
    g.close()


def test_noalloc_rejects_cubes_beyond_its_fixed_scratch():
    L = _lib()
    n = 128
    x = torch.zeros(n ** 3, device="cuda", dtype=torch.float64)
    st = L.lib().rt_coldens_single_noalloc(n, 1e24, 6.3e-18, C.c_void_p(x.data_ptr()),
                                           C.c_void_p(x.data_ptr()), 1, 2, 3, 60.0,
                                           C.c_void_p(x.data_ptr()), None)
    assert st == L.RT_ERR_INVALID
    assert b"exceeds the fixed scratch limit" in L.lib().rt_last_error()
