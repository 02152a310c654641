"""ctypes front end of the CPU oracle (``asora_oracle.cpp``).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` import this module.  The library under test
never imports it.

Every function takes and returns NumPy FP64 arrays in C order, index
``(i*n + j)*n + k``; see the C file header for the definitions followed
(arXiv 2311.01492 Sec. 2.1, 2.2, 3.1, 3.3 and App. A).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None

# The paper's physical constants and the table layout the tests use.
SIGMA0 = 6.30e-18          # cm^2, H I cross section at threshold (Sec. 4.1.3)
BETA = 2.8                 # sigma_nu = sigma0 (nu/nu_th)^-beta (Sec. 4.1.3)
TAU_LIM = 1e-7             # thin/thick switch on dtau*ds
TABLE_E0, TABLE_E1, TABLE_BITS = 30, 14, 6

_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_lp = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        L.or_table_nknots.restype = C.c_int
        L.or_table_nknots.argtypes = [C.c_int] * 3
        L.or_table_knot_taus.restype = None
        L.or_table_knot_taus.argtypes = [C.c_int, C.c_int, C.c_int, _dp]
        L.or_table_knots.restype = C.c_int
        L.or_table_knots.argtypes = [C.c_int, C.c_double, C.c_double, C.c_int, C.c_int, C.c_int,
                                     _dp, _dp]
        L.or_table_eval.restype = C.c_int
        L.or_table_eval.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p,
                                    C.c_int, C.c_int, _dp, _dp]
        L.or_shell_list.restype = C.c_int
        L.or_shell_list.argtypes = [C.c_int, C.c_void_p]
        L.or_raytrace2.restype = C.c_int
        L.or_raytrace2.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double,
                                   C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p,
                                   _dp, _dp, C.c_int, _ip, _dp, _dp,
                                   C.c_void_p, C.c_int, C.c_void_p, C.c_void_p,
                                   C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_double]
        L.or_raytrace.restype = C.c_int
        L.or_raytrace.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double,
                                  C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p,
                                  _dp, _dp, C.c_int, _ip, _dp, _dp,
                                  C.c_void_p, C.c_int, C.c_void_p, C.c_void_p,
                                  C.c_void_p, C.c_void_p, C.c_int, C.c_int]
        L.or_loss_grad_cs.restype = C.c_int
        L.or_loss_grad_cs.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double,
                                      C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p,
                                      _dp, _dp, C.c_int, _ip, _dp, _dp, _dp,
                                      C.c_int, _lp, _dp, C.c_int, _ip, _dp, C.c_double, C.c_int]
        L.or_lc_tau.restype = C.c_int
        L.or_lc_tau.argtypes = [C.c_int, C.c_double, C.c_double, _dp, _dp, C.c_int, C.c_int,
                                C.c_int, C.c_double, _dp]
        L.or_chemistry.restype = C.c_int
        L.or_chemistry.argtypes = [C.c_int64, _dp, _dp, _dp, _dp, C.c_double, C.c_double,
                                   C.c_double, C.c_double, C.c_int, C.c_double, _dp, _dp,
                                   C.POINTER(C.c_int64)]
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class Table:
    """Rate-table description: kind 0 = chords through knot values, 1 = analytic grey."""

    def __init__(self, kind, g=None, h=None, E0=TABLE_E0, E1=TABLE_E1, bits=TABLE_BITS):
        self.kind, self.E0, self.E1, self.bits = kind, E0, E1, bits
        self.g = None if g is None else _f64(g)
        self.h = None if h is None else _f64(h)

    def args(self):
        return (self.kind, self.E0, self.E1, self.bits, _ptr(self.g), _ptr(self.h))


def n_knots(E0=TABLE_E0, E1=TABLE_E1, bits=TABLE_BITS):
    return lib().or_table_nknots(E0, E1, bits)


def knot_taus(E0=TABLE_E0, E1=TABLE_E1, bits=TABLE_BITS):
    out = np.zeros(n_knots(E0, E1, bits))
    lib().or_table_knot_taus(E0, E1, bits, out)
    return out


def table_knots(spectrum="bb", T_bb=5e4, beta=BETA, E0=TABLE_E0, E1=TABLE_E1, bits=TABLE_BITS):
    """Knot values (g, h) of Eq. tables for a grey ('grey') or blackbody ('bb') source."""
    K = n_knots(E0, E1, bits)
    g = np.zeros(K)
    h = np.zeros(K)
    kind = 0 if spectrum == "grey" else 1
    rc = lib().or_table_knots(kind, float(T_bb), float(beta), E0, E1, bits, g, h)
    if rc != 0:
        raise ValueError("or_table_knots failed")
    return g, h


def make_table(spectrum="bb", T_bb=5e4, E0=TABLE_E0, E1=TABLE_E1, bits=TABLE_BITS):
    if spectrum == "grey_exact":
        return Table(1, None, None, E0, E1, bits)
    g, h = table_knots(spectrum, T_bb, BETA, E0, E1, bits)
    return Table(0, g, h, E0, E1, bits)


def table_eval(tab: Table, tau, which="g"):
    tau = _f64(np.atleast_1d(tau))
    out = np.zeros_like(tau)
    rc = lib().or_table_eval(*tab.args(), 0 if which == "g" else 1, tau.size, tau, out)
    if rc != 0:
        raise ValueError("bad table")
    return out


def shell_list(q):
    n = lib().or_shell_list(q, None)
    out = np.zeros((n, 3), dtype=np.int32)
    lib().or_shell_list(q, out.ctypes.data_as(C.c_void_p))
    return out


def raytrace(n, cell_cm, nH, xHI, pos, ndot, radius, table: Table, sigma0=SIGMA0,
             tau_lim=TAU_LIM, gamma=True, coldens_src=-1, wloss=None, nthreads=1,
             debug=False, interp=0, tau_w0=0.6):
    """Ray trace all sources (octahedral-shell SC).  Returns dict with
    'gamma' (n^3 or None), 'coldens'/'tau_in' (for coldens_src), 'loss'.
    interp: 0 the paper's geometric weights, 1 optical-depth-modulated weights
    with floor tau_w0 (see the C file header)."""
    nH = _f64(nH).reshape(-1)
    xHI = _f64(xHI).reshape(-1)
    pos = np.ascontiguousarray(pos, dtype=np.int32).reshape(-1, 3)
    ndot = _f64(ndot).reshape(-1)
    radius = _f64(np.broadcast_to(radius, ndot.shape)).copy()
    nc = n ** 3
    g = np.zeros(nc) if gamma else None
    cd = ti = None
    if coldens_src >= 0:
        cd = np.zeros(nc)
        ti = np.zeros(nc)
    loss = None
    if wloss is not None:
        wloss = _f64(wloss).reshape(-1)
        loss = np.zeros(1)
    rc = lib().or_raytrace2(n, cell_cm, sigma0, tau_lim, *table.args(), nH, xHI,
                            ndot.size, pos.reshape(-1), ndot, radius, _ptr(g), coldens_src,
                            _ptr(cd), _ptr(ti), _ptr(wloss), _ptr(loss), nthreads, int(debug),
                            int(interp), float(tau_w0))
    if rc == 2:
        raise RuntimeError("oracle: acausal read (an interpolant was not computed yet)")
    if rc != 0:
        raise ValueError("oracle: invalid arguments")
    return {"gamma": g, "coldens": cd, "tau_in": ti,
            "loss": None if loss is None else float(loss[0])}


def loss_grad_cs(n, cell_cm, nH, xHI, pos, ndot, radius, table: Table, wloss, cells, srcs,
                 sigma0=SIGMA0, tau_lim=TAU_LIM, h=1e-30, nthreads=1):
    """Complex-step dL/dlog n_HI at `cells` and dL/dlog Ndot at `srcs`, L = sum w Gamma."""
    pos = np.ascontiguousarray(pos, dtype=np.int32).reshape(-1, 3)
    ndot = _f64(ndot).reshape(-1)
    radius = _f64(np.broadcast_to(radius, ndot.shape)).copy()
    cells = np.ascontiguousarray(cells, dtype=np.int64).reshape(-1)
    srcs = np.ascontiguousarray(srcs, dtype=np.int32).reshape(-1)
    dn = np.zeros(cells.size)
    dq = np.zeros(srcs.size)
    rc = lib().or_loss_grad_cs(n, cell_cm, sigma0, tau_lim, *table.args(), _f64(nH).reshape(-1),
                               _f64(xHI).reshape(-1), ndot.size, pos.reshape(-1), ndot, radius,
                               _f64(wloss).reshape(-1), cells.size, cells, dn, srcs.size, srcs,
                               dq, h, nthreads)
    if rc != 0:
        raise ValueError("oracle: invalid arguments")
    return dn, dq


def lc_tau(n, cell_cm, nH, xHI, src, radius, sigma0=SIGMA0):
    """Long-characteristics optical depth out of every traced cell of one source."""
    out = np.full(n ** 3, np.nan)
    lib().or_lc_tau(n, cell_cm, sigma0, _f64(nH).reshape(-1), _f64(xHI).reshape(-1),
                    int(src[0]), int(src[1]), int(src[2]), float(radius), out)
    return out


def chemistry(nH, x0, xavg_in, gamma, dt, alpha_H=2.59e-13, C_H=0.0, tol=1e-10, maxit=50,
              conv_tol=1e-3):
    """Time-averaged chemistry step (Eq. time_avrg_sol); returns (<x_HII>, x_HII(t+dt), n_unconv)."""
    nH = _f64(nH).reshape(-1)
    xa = np.zeros_like(nH)
    xn = np.zeros_like(nH)
    cnt = C.c_int64(0)
    lib().or_chemistry(nH.size, nH, _f64(x0).reshape(-1), _f64(xavg_in).reshape(-1),
                       _f64(gamma).reshape(-1), dt, alpha_H, C_H, tol, maxit, conv_tol, xa, xn,
                       C.byref(cnt))
    return xa, xn, int(cnt.value)
