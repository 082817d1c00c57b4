"""ctypes loader for libvpm.so (declarations mirror include/vpm.h).

The library is built in-tree by ``paper_2511_11430_gb300.build``.  Loading fails
loudly when it is missing: there is no CPU fallback anywhere in this package.
"""
from __future__ import annotations

import ctypes
import os
import threading

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libvpm.so")

VPM_OK = 0
VPM_ERR_INVALID_ARG = -1
VPM_ERR_CUDA = -2
VPM_ERR_NONFINITE = -3
VPM_ERR_NOT_CONVERGED = -4
VPM_ERR_WORKSPACE = -5
VPM_ERR_LIMIT = -6

VPM_COMPENSATED = 0x1
VPM_STRETCH_CLASSIC = 0x2
VPM_CHECK_FINITE = 0x4

VPM_OP_INDUCE = 1
VPM_OP_SEGMENTS = 2
VPM_OP_RHS = 3
VPM_OP_STEP = 4
VPM_OP_AIC_SOLVE = 5
VPM_OP_BACKWARD = 6
VPM_OP_WAKE_CONVERT = 7
VPM_OP_WAKE_ROW = 8
VPM_OP_LOADS = 9
VPM_OP_TREE = 10
VPM_OP_RHS_TREE = 11
VPM_OP_STEP_TREE = 12
VPM_OP_STAGE = 13

VPM_TRACE_ALL = 0
VPM_TRACE_SWEEP = 1
VPM_TRACE_ADJOINT = 2
VPM_TRACE_PSE = 3
VPM_TRACE_SWEEP_VEL = 4
VPM_TRACE_SEGMENTS = 5

VPM_MAX_ITEMS = 1 << 30
VPM_MAX_AIC = 8192
VPM_NOALLOC_SCRATCH_BYTES = 64 << 20

STATUS_NAMES = {
    0: "VPM_OK", -1: "VPM_ERR_INVALID_ARG", -2: "VPM_ERR_CUDA", -3: "VPM_ERR_NONFINITE",
    -4: "VPM_ERR_NOT_CONVERGED", -5: "VPM_ERR_WORKSPACE", -6: "VPM_ERR_LIMIT",
}


class VpmParams(ctypes.Structure):
    _fields_ = [
        ("sigma", ctypes.c_float),
        ("nu", ctypes.c_float),
        ("c_v", ctypes.c_float),
        ("seg_core", ctypes.c_float),
        ("u_inf", ctypes.c_float * 3),
        ("vatistas_n", ctypes.c_int),
        ("flags", ctypes.c_int),
    ]


class VpmError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_F = ctypes.c_float
_D = ctypes.c_double
_INT = ctypes.c_int
_SZ = ctypes.c_size_t

SIGNATURES = {
    "vpm_last_error": (ctypes.c_char_p, []),
    "vpm_version": (_INT, []),
    "vpm_device_error": (_INT, [ctypes.POINTER(_INT)]),
    "vpm_workspace_size": (_INT, [_INT, _I64, _I64, _I64, _INT, ctypes.POINTER(_SZ)]),
    "vpm_induce": (_INT, [_P, _P, _I64, _P, _I64, _F, _INT, _P, _P, _P, _SZ, _P]),
    "vpm_segments_induce": (_INT, [_P, _P, _I64, _P, _I64, _F, _INT, _INT, _P, _P, _P, _SZ, _P]),
    "vpm_tree_induce": (_INT, [_P, _P, _I64, _F, _F, _INT, _P, _P, _P, _SZ, _P]),
    "vpm_rhs": (_INT, [_P, _P, _I64, _P, _P, _I64, ctypes.POINTER(VpmParams), _P, _P, _P, _P, _SZ, _P]),
    "vpm_pack_state": (_INT, [_P, _P, _P, _I64, _P, _P, _P]),
    "vpm_step": (_INT, [_P, _P, _P, _I64, _P, _P, _I64, ctypes.POINTER(VpmParams), _D, _P, _SZ, _P]),
    "vpm_rk3_stage": (_INT, [_INT, _P, _P, _P, _P, _I64, _P, _P, _I64, ctypes.POINTER(VpmParams), _D, _P, _SZ,
                              _P]),
    "vpm_rhs_tree": (_INT, [_P, _P, _I64, _P, _P, _I64, ctypes.POINTER(VpmParams), _F, _INT, _P, _P, _P, _P, _SZ,
                            _P]),
    "vpm_step_tree": (_INT, [_P, _P, _P, _I64, _P, _P, _I64, ctypes.POINTER(VpmParams), _F, _INT, _D, _P, _SZ, _P]),
    "aic_build": (_INT, [_P, _P, _P, _INT, _F, _INT, _P, _P, _P, _P, _P]),
    "aic_solve": (_INT, [_P, _P, _P, _INT, _D, _INT, ctypes.POINTER(_INT), ctypes.POINTER(_D), _P, _SZ, _P]),
    "vpm_induce_backward": (_INT, [_P, _P, _I64, _P, _I64, _F, _INT, _P, _P, _P, _P, _SZ, _P]),
    "vpm_induce_noalloc": (_INT, [_P, _P, _I64, _P, _I64, _F, _INT, _P, _P, _P]),
    "vpm_selftest_wait": (_INT, [_D, _P, _P]),
    "vpm_wake_segments": (_INT, [_P, _P, _I64, _I64, _I64, _P, _P, _P]),
    "vpm_points_pack": (_INT, [_P, _I64, _P, _P]),
    "vpm_ring_segments": (_INT, [_P, _P, _I64, _P, _P, _P]),
    "vpm_segment_midpoints": (_INT, [_P, _P, _I64, _P, _P]),
    "vpm_blade_loads": (_INT, [_P, _P, _I64, _P, _P, _P, _P, _P, _P, _P, _P, _I64, _D, _D, _P, _P, _SZ, _P]),
    "vpm_points_advect": (_INT, [_P, _P, _I64, _D, _P, _P]),
    "vpm_wake_convert": (_INT, [_P, _P, _P, _P, _P, _P, _I64, _D, _INT, _INT, _P, _P, _I64, _P, _P, _SZ, _P]),
    "vpm_wake_convert_row": (_INT, [_P, _P, _P, _I64, _D, _INT, _INT, _P, _P, _I64, _P, _P, _SZ, _P]),
    "vpm_trace_enable": (_INT, [_INT]),
    "vpm_trace_reset": (_INT, []),
    "vpm_trace_read": (_INT, [_INT, ctypes.POINTER(_I64), ctypes.POINTER(_D)]),
}

_lock = threading.Lock()
_lib = None


def load(path: str | None = None):
    """Load libvpm.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(
                f"libvpm.so not found at {p}: build it with `python -c 'import __graft_entry__ as g; g.build()'` "
                "(there is no CPU fallback)")
        lib = ctypes.CDLL(p)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def check(status: int) -> None:
    if status != VPM_OK:
        msg = load().vpm_last_error()
        raise VpmError(status, msg.decode() if msg else "")
