"""ctypes declarations of libasora (include/asora.h).  Argument marshalling only."""
import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libasora.so")

RT_OK, RT_ERR_INVALID, RT_ERR_OOM, RT_ERR_CUDA, RT_ERR_TIMEOUT, RT_ERR_STATE, RT_ERR_BOUNDS = range(7)
RT_SCHED_AUTO, RT_SCHED_PLAIN, RT_SCHED_BATCHED, RT_SCHED_BATCHED_EXIT = 0, 1, 2, 3
RT_TABLE_CHORDS, RT_TABLE_GREY_EXACT = 0, 1
RT_INTERP_GEOMETRIC, RT_INTERP_OPTICAL_DEPTH = 0, 1
STATUS_NAMES = {0: "RT_OK", 1: "RT_ERR_INVALID", 2: "RT_ERR_OOM", 3: "RT_ERR_CUDA",
                4: "RT_ERR_TIMEOUT", 5: "RT_ERR_STATE", 6: "RT_ERR_BOUNDS"}


class RtError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


class rt_params(C.Structure):
    _fields_ = [("sigma0_cm2", C.c_double), ("tau_lim", C.c_double)]


class rt_stats(C.Structure):
    _fields_ = [("trace_ms", C.c_double), ("prep_ms", C.c_double),
                ("source_voxels", C.c_int64), ("items", C.c_int64), ("rate_cells", C.c_int64),
                ("kernel_launches", C.c_int64), ("launches", C.c_int),
                ("schedule", C.c_int), ("block", C.c_int), ("grid", C.c_int),
                ("row_table_bytes", C.c_int64)]


_L = None

_P = C.c_void_p
_D = C.c_double
_I = C.c_int

SIGNATURES = {
    "rt_params_default": (None, [C.POINTER(rt_params)]),
    "rt_last_error": (C.c_char_p, []),
    "rt_grid_create": (_I, [C.POINTER(_P), _I, _D, C.POINTER(rt_params), _P]),
    "rt_ensemble_create": (_I, [C.POINTER(_P), _I, _P, _P, C.POINTER(rt_params), _P]),
    "rt_set_stream": (_I, [_P, _P]),
    "rt_table_nknots": (_I, [_I, _I, _I]),
    "rt_table_blackbody": (_I, [_D, _D, _I, _I, _I, _P, _P]),
    "rt_set_tables": (_I, [_P, _I, _I, _I, _I, _P, _P]),
    "rt_set_density": (_I, [_P, _P]),
    "rt_set_xHI": (_I, [_P, _P]),
    "rt_set_scale_factor": (_I, [_P, _D]),
    "rt_set_sources": (_I, [_P, _I, _P, _P, _P, _P]),
    "rt_raytrace": (_I, [_P, _P, _I]),
    "rt_raytrace_source_coldens": (_I, [_P, _I, _P, _I]),
    "rt_chemistry_step": (_I, [_P, _P, _P, _P, _D, _D, _D, _D, _P, _P, _P]),
    "rt_iterate": (_I, [_P, _P, _D, _D, _D, _I, _D, _D, _I, _P, C.POINTER(_I)]),
    "rt_get_stats": (_I, [_P, C.POINTER(rt_stats)]),
    "rt_check": (_I, [_P]),
    "rt_inject_device_error": (_I, [_P, _I]),
    "rt_set_device_memory_limit": (_I, [C.c_int64]),
    "rt_device_memory_in_use": (C.c_int64, []),
    "rt_set_schedule": (_I, [_P, _I, _I, _I]),
    "rt_raytrace_backward": (_I, [_P, _P, _P, _P]),
    "rt_set_adjoint_mode": (_I, [_P, _I]),
    "rt_set_interpolation": (_I, [_P, _I, _D]),
    "rt_autotune": (_I, [_P, C.c_char_p, C.POINTER(_I), C.POINTER(_I), C.POINTER(_I)]),
    "rt_grid_destroy": (None, [_P]),
    "rt_shell_enumerate": (_I, [_I, _P]),
    "rt_kernel_launch_count": (C.c_longlong, []),
    "rt_coldens_single_noalloc": (_I, [_I, _D, _D, _P, _P, _I, _I, _I, _D, _P, _P]),
}


def lib():
    """Load libasora.so.  Raises if it has not been built: there is no fallback."""
    global _L
    if _L is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libasora.so is not built (run python -m paper_2311_01492_gb300.build"
                              " or __graft_entry__.build())")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _L = L
    return _L


def check(status, what=""):
    if status != RT_OK:
        msg = lib().rt_last_error()
        raise RtError(status, (what + ": " if what else "") + (msg.decode() if msg else ""))
