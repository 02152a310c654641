"""Python front end of libasora: the same calls as include/asora.h.

PyTorch provides device memory and streams; every step of the ray tracing,
rate accumulation and chemistry runs in the library's CUDA kernels.  There is
no CPU path: a missing library or GPU raises.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib as L
from ._lib import RtError  # noqa: F401  (re-export)

SIGMA0 = 6.30e-18
TAU_LIM = 1e-7
TABLE_E0, TABLE_E1, TABLE_BITS = 30, 14, 6
ALPHA_B_1E4K = 2.59e-13  # case-B recombination coefficient at 1e4 K (Sec. 4.1.1)

_SCHED = {"auto": L.RT_SCHED_AUTO, "plain": L.RT_SCHED_PLAIN, "batched": L.RT_SCHED_BATCHED,
          "early_exit": L.RT_SCHED_BATCHED_EXIT}


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _dev_f64(t, n=None, name="array"):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if t.dtype != torch.float64 or not t.is_contiguous():
        raise TypeError("%s must be a contiguous float64 tensor" % name)
    if n is not None and t.numel() != n:
        raise ValueError("%s must have %d elements" % (name, n))
    return t


def table_nknots(E0=TABLE_E0, E1=TABLE_E1, bits=TABLE_BITS):
    return L.lib().rt_table_nknots(E0, E1, bits)


def table_blackbody(T_bb=5e4, beta=2.8, E0=TABLE_E0, E1=TABLE_E1, bits=TABLE_BITS):
    """Knot values (g, h) of the blackbody transmission tables (host quadrature)."""
    K = table_nknots(E0, E1, bits)
    g = np.zeros(K)
    h = np.zeros(K)
    L.check(L.lib().rt_table_blackbody(T_bb, beta, E0, E1, bits, g.ctypes.data_as(C.c_void_p),
                                       h.ctypes.data_as(C.c_void_p)), "rt_table_blackbody")
    return g, h


def set_device_memory_limit(nbytes):
    """Process-wide cap on the device memory the library holds (0: none)."""
    L.check(L.lib().rt_set_device_memory_limit(int(nbytes)), "rt_set_device_memory_limit")


def device_memory_in_use():
    return int(L.lib().rt_device_memory_in_use())


def shell_enumerate(q):
    n = L.lib().rt_shell_enumerate(q, None)
    if n < 0:
        raise ValueError("q must be >= 0")
    out = np.zeros((n, 3), dtype=np.int32)
    L.lib().rt_shell_enumerate(q, out.ctypes.data_as(C.c_void_p))
    return out


class Grid:
    """A periodic box (or an ensemble of boxes) with its sources and tables."""

    def __init__(self, n, cell_cm, sigma0=SIGMA0, tau_lim=TAU_LIM, stream=None, _ns=None,
                 _cells=None):
        if not torch.cuda.is_available():
            raise RuntimeError("libasora needs a CUDA device")
        self._lib = L.lib()
        p = L.rt_params()
        self._lib.rt_params_default(C.byref(p))
        p.sigma0_cm2 = sigma0
        p.tau_lim = tau_lim
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = C.c_void_p()
        sp = C.c_void_p(self.stream.cuda_stream)
        if _ns is None:
            L.check(self._lib.rt_grid_create(C.byref(h), int(n), float(cell_cm), C.byref(p), sp),
                    "rt_grid_create")
            self.sizes = [int(n)]
        else:
            ns = np.ascontiguousarray(_ns, dtype=np.int32)
            cs = np.ascontiguousarray(_cells, dtype=np.float64)
            L.check(self._lib.rt_ensemble_create(C.byref(h), ns.size, ns.ctypes.data_as(C.c_void_p),
                                                 cs.ctypes.data_as(C.c_void_p), C.byref(p), sp),
                    "rt_ensemble_create")
            self.sizes = [int(x) for x in ns]
        self._h = h
        self.ncell = int(sum(x ** 3 for x in self.sizes))
        self.sigma0 = sigma0
        self._keep = {}

    @classmethod
    def ensemble(cls, sizes, cell_cm, **kw):
        sizes = list(sizes)
        cells = np.broadcast_to(np.asarray(cell_cm, dtype=np.float64), (len(sizes),))
        return cls(None, None, _ns=sizes, _cells=cells, **kw)

    # ----------------------------------------------------------- set-up
    def set_tables(self, spectrum="bb", T_bb=5e4, beta=2.8, g=None, h=None, E0=TABLE_E0,
                   E1=TABLE_E1, bits=TABLE_BITS):
        """spectrum: 'bb' (library quadrature), 'grey_exact' (exp evaluated in the
        kernels) or 'knots' (knot values g, h given by the caller)."""
        if spectrum == "grey_exact":
            L.check(self._lib.rt_set_tables(self._h, L.RT_TABLE_GREY_EXACT, E0, E1, bits, None,
                                            None), "rt_set_tables")
            return
        if spectrum == "bb":
            g, h = table_blackbody(T_bb, beta, E0, E1, bits)
        elif spectrum != "knots":
            raise ValueError("unknown spectrum %r" % spectrum)
        g = np.ascontiguousarray(g, dtype=np.float64)
        h = np.ascontiguousarray(h, dtype=np.float64)
        L.check(self._lib.rt_set_tables(self._h, L.RT_TABLE_CHORDS, E0, E1, bits,
                                        g.ctypes.data_as(C.c_void_p),
                                        h.ctypes.data_as(C.c_void_p)), "rt_set_tables")

    def set_density(self, nH):
        nH = _dev_f64(nH, self.ncell, "nH")
        L.check(self._lib.rt_set_density(self._h, _ptr(nH)), "rt_set_density")
        self._keep["nH"] = nH

    def set_xHI(self, xHI):
        xHI = _dev_f64(xHI, self.ncell, "xHI")
        L.check(self._lib.rt_set_xHI(self._h, _ptr(xHI)), "rt_set_xHI")
        self._keep["xHI"] = xHI

    def set_scale_factor(self, a):
        """Expanding background: proper cell = cell * a, proper n_H = n_H * a^-3."""
        L.check(self._lib.rt_set_scale_factor(self._h, float(a)), "rt_set_scale_factor")

    def set_sources(self, pos, ndot, radius, box=None):
        pos = pos.to(dtype=torch.int32).contiguous()
        if not pos.is_cuda or pos.dim() != 2 or pos.shape[1] != 3:
            raise ValueError("pos must be a CUDA (nsrc, 3) tensor")
        nsrc = pos.shape[0]
        ndot = _dev_f64(ndot.contiguous(), nsrc, "ndot")
        radius = _dev_f64(radius.contiguous(), nsrc, "radius")
        boxp = None
        if box is not None:
            box = box.to(dtype=torch.int32).contiguous()
            boxp = _ptr(box)
        L.check(self._lib.rt_set_sources(self._h, nsrc, _ptr(pos), boxp, _ptr(ndot), _ptr(radius)),
                "rt_set_sources")
        self.nsrc = nsrc

    # ------------------------------------------------------------ work
    def raytrace(self, gamma=None, schedule="batched"):
        if gamma is None:
            gamma = torch.empty(self.ncell, dtype=torch.float64, device="cuda")
        _dev_f64(gamma, self.ncell, "gamma")
        L.check(self._lib.rt_raytrace(self._h, _ptr(gamma), _SCHED[schedule]), "rt_raytrace")
        return gamma

    def source_coldens(self, src, out=None, schedule="batched"):
        if out is None:
            out = torch.empty(self.ncell, dtype=torch.float64, device="cuda")
        _dev_f64(out, self.ncell, "out")
        L.check(self._lib.rt_raytrace_source_coldens(self._h, int(src), _ptr(out),
                                                     _SCHED[schedule]),
                "rt_raytrace_source_coldens")
        return out

    def chemistry_step(self, gamma, x0, xavg_in, dt, alpha_H=ALPHA_B_1E4K, C_H=0.0, conv_tol=1e-3):
        xa = torch.empty_like(x0)
        xn = torch.empty_like(x0)
        cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
        for t, nm in ((gamma, "gamma"), (x0, "x0"), (xavg_in, "xavg_in")):
            _dev_f64(t, self.ncell, nm)
        L.check(self._lib.rt_chemistry_step(self._h, _ptr(gamma), _ptr(x0), _ptr(xavg_in), dt,
                                            alpha_H, C_H, conv_tol, _ptr(xa), _ptr(xn), _ptr(cnt)),
                "rt_chemistry_step")
        return xa, xn, cnt

    def iterate(self, x, dt, alpha_H=ALPHA_B_1E4K, C_H=0.0, max_iter=10, conv_tol=1e-3,
                conv_frac=1e-4, use_graph=True, gamma=None):
        """One RT <-> chemistry time step; x (x_HII, CUDA float64) is updated in place."""
        _dev_f64(x, self.ncell, "x")
        if gamma is None:
            gamma = torch.empty(self.ncell, dtype=torch.float64, device="cuda")
        it = C.c_int(0)
        L.check(self._lib.rt_iterate(self._h, _ptr(x), dt, alpha_H, C_H, max_iter, conv_tol,
                                     conv_frac, int(bool(use_graph)), _ptr(gamma), C.byref(it)),
                "rt_iterate")
        self._keep.pop("xHI", None)
        return gamma, it.value

    def backward(self, w, dlogn=None, dlogndot=None):
        """Adjoint of raytrace for L = sum(w * Gamma): (dL/dlog n_HI, dL/dlog Ndot)."""
        _dev_f64(w, self.ncell, "w")
        if dlogn is None:
            dlogn = torch.empty(self.ncell, dtype=torch.float64, device="cuda")
        if dlogndot is None:
            dlogndot = torch.empty(max(self.nsrc, 1), dtype=torch.float64, device="cuda")
        L.check(self._lib.rt_raytrace_backward(self._h, _ptr(w), _ptr(dlogn), _ptr(dlogndot)),
                "rt_raytrace_backward")
        return dlogn, dlogndot[:self.nsrc]

    def set_interpolation(self, mode="geometric", tau_weight_min=0.6):
        """Interpolation weights: "geometric" (the paper's) or "optical_depth"."""
        m = {"geometric": L.RT_INTERP_GEOMETRIC, "optical_depth": L.RT_INTERP_OPTICAL_DEPTH}[mode]
        L.check(self._lib.rt_set_interpolation(self._h, m, float(tau_weight_min)),
                "rt_set_interpolation")

    def set_adjoint_mode(self, stop_at_opaque=True):
        L.check(self._lib.rt_set_adjoint_mode(self._h, int(bool(stop_at_opaque))),
                "rt_set_adjoint_mode")

    def set_schedule(self, block_big=128, hsmall=19, hface=13):
        """Batched schedule: CTA size, warp-mode threshold, whole-face-warp threshold."""
        L.check(self._lib.rt_set_schedule(self._h, int(block_big), int(hsmall), int(hface)),
                "rt_set_schedule")

    def autotune(self, cache_path=None):
        """Pick the batched schedule by timing; returns (block_big, hsmall, hface)."""
        b, hs, hf = C.c_int(0), C.c_int(0), C.c_int(0)
        L.check(self._lib.rt_autotune(self._h, None if cache_path is None else
                                      str(cache_path).encode(), C.byref(b), C.byref(hs),
                                      C.byref(hf)),
                "rt_autotune")
        return b.value, hs.value, hf.value

    def stats(self):
        s = L.rt_stats()
        L.check(self._lib.rt_get_stats(self._h, C.byref(s)), "rt_get_stats")
        return {k: getattr(s, k) for k, _ in s._fields_}

    def check(self):
        """Synchronise and raise RtError(RT_ERR_BOUNDS) if a device-side check failed."""
        L.check(self._lib.rt_check(self._h), "rt_check")

    def close(self):
        if getattr(self, "_h", None):
            self._lib.rt_grid_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class RayTraceFn(torch.autograd.Function):
    """Gamma as a differentiable function of log n_HI (per cell) and log Ndot (per
    source); the backward pass is the library's adjoint kernel.  The grid's
    sources are re-registered with rates exp(log_ndot) and its density with
    n_H = exp(log_nhi), x_HI = 1 on every call."""

    @staticmethod
    def forward(ctx, log_nhi, log_ndot, grid, pos, radius, schedule="batched"):
        nhi = torch.exp(log_nhi).contiguous()
        ndot = torch.exp(log_ndot).contiguous()
        ones = torch.ones_like(nhi)
        grid.set_density(nhi)
        grid.set_xHI(ones)
        grid.set_sources(pos, ndot, radius)
        gamma = grid.raytrace(schedule=schedule)
        ctx.grid = grid
        ctx.save_for_backward(nhi, ones, pos, ndot, radius)
        return gamma

    @staticmethod
    def backward(ctx, gout):
        grid = ctx.grid
        nhi, ones, pos, ndot, radius = ctx.saved_tensors
        grid.set_density(nhi)
        grid.set_xHI(ones)
        grid.set_sources(pos, ndot, radius)
        dn, dq = grid.backward(gout.contiguous())
        return dn, dq, None, None, None, None


def raytrace_autograd(grid, log_nhi, log_ndot, pos, radius, schedule="batched"):
    return RayTraceFn.apply(log_nhi, log_ndot, grid, pos, radius, schedule)
