"""CPU-side checks of libasora: it loads, exports every declared symbol, and
its host-side pieces (shell enumeration, table quadrature, argument checks)
behave -- no GPU needed."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2311_01492_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    from paper_2311_01492_gb300 import _lib
    return _lib.lib()


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "asora.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rt_[a-z_0-9]+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    names = declared_symbols()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n


def test_shell_enumeration_is_a_bijection_onto_the_octahedral_shell(lib):
    from paper_2311_01492_gb300.api import shell_enumerate
    for q in range(0, 31):
        got = shell_enumerate(q)
        brute = {(a, b, c) for a in range(-q, q + 1) for b in range(-q, q + 1)
                 for c in range(-q, q + 1) if abs(a) + abs(b) + abs(c) == q}
        assert len(got) == len(brute) == (1 if q == 0 else 4 * q * q + 2)
        assert {tuple(x) for x in got} == brute
        top = 2 * q * (q + 1) + 1
        assert np.all(got[:top, 2] >= 0) and np.all(got[top:, 2] < 0)


def test_library_tables_match_oracle_quadrature(lib):
    from oracle import oracle as O
    from paper_2311_01492_gb300.api import table_blackbody
    for T in (5e3, 5e4, 1e5):
        g, h = table_blackbody(T)
        go, ho = O.table_knots("bb", T)
        np.testing.assert_allclose(g, go, rtol=1e-12, atol=0)
        np.testing.assert_allclose(h, ho, rtol=1e-12, atol=0)


def test_argument_errors_without_a_gpu(lib):
    from paper_2311_01492_gb300 import _lib as L
    h = C.c_void_p()
    p = L.rt_params()
    lib.rt_params_default(C.byref(p))
    assert p.sigma0_cm2 == 6.3e-18 and p.tau_lim == 1e-7
    assert lib.rt_grid_create(C.byref(h), 0, 1.0, C.byref(p), None) == L.RT_ERR_INVALID
    assert b"box size" in lib.rt_last_error()
    assert lib.rt_grid_create(C.byref(h), 16, -1.0, C.byref(p), None) == L.RT_ERR_INVALID
    assert lib.rt_raytrace(None, None, 0) == L.RT_ERR_INVALID
    assert lib.rt_table_nknots(30, 14, 6) == 44 * 64 + 2
    assert lib.rt_table_nknots(0, 14, 6) == -1
    assert lib.rt_shell_enumerate(-1, None) == -1


def test_device_memory_limit_argument_checks_need_no_gpu(lib):
    from paper_2311_01492_gb300 import _lib
    assert lib.rt_set_device_memory_limit(-1) == _lib.RT_ERR_INVALID
    assert b"negative" in lib.rt_last_error()
    assert lib.rt_device_memory_in_use() == 0  # nothing allocated without a GPU
    assert lib.rt_set_device_memory_limit(0) == _lib.RT_OK
