"""ctypes loader for libsrt.so (the C ABI in include/srt.h).

The library is built in-tree by ``paper_2402_15641_gb300.build``.  There is no
fallback: if the library is missing or fails to load, every call raises.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsrt.so")

SRT_OK, SRT_ERR_ARG, SRT_ERR_GEOMETRY, SRT_ERR_OOM, SRT_ERR_CUDA = 0, 1, 2, 3, 4
SRT_ERR_WORKSPACE, SRT_ERR_TIMEOUT, SRT_ERR_NOT_READY = 5, 6, 7
SRT_FP32, SRT_BF16 = 0, 1
SRT_KEEP_F64 = 1
SRT_CSR_ONLY = 2
SRT_A1_ROTATION = 8
SRT_RHO_LINEAR = 16
SRT_ROWWISE = 32
SRT_A1_FULL = 64
SRT_FUSE_RESHAPES = 128
SRT_VOXEL_LINEAR = 256
SRT_NOALLOC_WORKSPACE_BYTES = 32 << 20


class SrtGeometry(ctypes.Structure):
    _fields_ = [
        ("ms", ctypes.c_int32), ("mz", ctypes.c_int32),
        ("dxy", ctypes.c_double), ("dz", ctypes.c_double), ("radius", ctypes.c_double),
        ("n_phi", ctypes.c_int32), ("phi0", ctypes.c_double),
        ("n_zs", ctypes.c_int32), ("zs_lo", ctypes.c_double), ("zs_hi", ctypes.c_double),
        ("n_ell", ctypes.c_int32), ("ell_lo", ctypes.c_double), ("ell_hi", ctypes.c_double),
        ("weight_dtype", ctypes.c_int32), ("flags", ctypes.c_int32),
        ("n_phi_total", ctypes.c_int32), ("phi_first", ctypes.c_int32),
    ]


class SrtPlanInfo(ctypes.Structure):
    _fields_ = [
        ("rows1", ctypes.c_int64), ("cols1", ctypes.c_int64), ("nnz1", ctypes.c_int64),
        ("rows2", ctypes.c_int64), ("cols2", ctypes.c_int64), ("nnz2", ctypes.c_int64),
        ("dropped1", ctypes.c_int64), ("dropped2", ctypes.c_int64),
        ("device_bytes", ctypes.c_int64), ("weight_dtype", ctypes.c_int32),
        ("a2_taps", ctypes.c_int32), ("n_taps", ctypes.c_int64),
        ("a1_rot", ctypes.c_int32), ("tile_order", ctypes.c_int32),
        ("tile_records", ctypes.c_int64 * 3),
    ]


# name -> (restype, argtypes)
_VP, _I32, _I64, _SZ = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
_GP = ctypes.POINTER(SrtGeometry)
SIGNATURES = {
    "srt_geometry_default": (ctypes.c_int, [_GP, _I32, _I32, ctypes.c_double, ctypes.c_double,
                                            ctypes.c_double, _I32, _I32, _I32]),
    "srt_plan": (ctypes.c_int, [_GP, _VP, ctypes.POINTER(_VP)]),
    "srt_plan_info": (ctypes.c_int, [_VP, ctypes.POINTER(SrtPlanInfo)]),
    "srt_workspace_bytes": (ctypes.c_int, [_VP, _I32, ctypes.POINTER(_SZ)]),
    "srt_forward": (ctypes.c_int, [_VP, _VP, _VP, _I32, _VP, _SZ, _VP]),
    "srt_adjoint": (ctypes.c_int, [_VP, _VP, _VP, _I32, _VP, _SZ, _VP]),
    "srt_host_workspace_bytes": (ctypes.c_int, [_VP, _I32, ctypes.POINTER(_SZ)]),
    "srt_forward_host": (ctypes.c_int, [_VP, _VP, _VP, _I32, _VP, _SZ, _VP]),
    "srt_forward_noalloc": (ctypes.c_int, [_VP, _VP, _VP, _I32, _VP]),
    "srt_adjoint_noalloc": (ctypes.c_int, [_VP, _VP, _VP, _I32, _VP]),
    "srt_adjoint_host": (ctypes.c_int, [_VP, _VP, _VP, _I32, _VP, _SZ, _VP]),
    "srt_dot_workspace_bytes": (_SZ, []),
    "srt_dot_f64": (ctypes.c_int, [_VP, _VP, _I64, _VP, _VP, _SZ, _VP]),
    "srt_plan_export": (ctypes.c_int, [_VP, _I32, _VP, _VP, _VP, _VP]),
    "srt_plan_set_timing": (ctypes.c_int, [_VP, _I32]),
    "srt_stage_times": (ctypes.c_int, [_VP, _I32, ctypes.POINTER(ctypes.c_float), _I32]),
    "srt_launches_per_call": (ctypes.c_int, [_VP, _I32, _I32]),
    "srt_fp32_fma_peak": (ctypes.c_int, [_I32, ctypes.POINTER(ctypes.c_double), _VP]),
    "srt_pipe_create": (ctypes.c_int, [_VP, _I32, _I32, ctypes.POINTER(_VP)]),
    "srt_pipe_submit": (ctypes.c_int, [_VP, _I32, _VP, _VP, ctypes.POINTER(_I64)]),
    "srt_pipe_wait": (ctypes.c_int, [_VP, _I64, ctypes.c_double]),
    "srt_pipe_stage_times": (ctypes.c_int, [_VP, _I64, ctypes.POINTER(ctypes.c_float)]),
    "srt_pipe_destroy": (ctypes.c_int, [_VP]),
    "srt_plan_destroy": (ctypes.c_int, [_VP]),
    "srt_error_string": (ctypes.c_char_p, [ctypes.c_int]),
    "srt_checks_read": (ctypes.c_int, [ctypes.POINTER(ctypes.c_int64)]),
    "srt_checks_cap": (ctypes.c_int, [_I32]),
}


class SrtError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        msg = lib().srt_error_string(code).decode() if _lib is not None else str(code)
        super().__init__(f"{where}: {msg} (status {code})")


_lib = None


def load(path: str):
    """A libsrt build at `path` with every ABI signature declared."""
    if not os.path.exists(path):
        raise RuntimeError(
            f"{os.path.basename(path)} not found at {path}: build it with "
            "`python -m paper_2402_15641_gb300.build` (there is no CPU fallback)")
    L = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    return L


def lib():
    """Load libsrt.so once; raises if it has not been built."""
    global _lib
    if _lib is None:
        _lib = load(LIB_PATH)
    return _lib


def check(code: int, where: str) -> None:
    if code != SRT_OK:
        raise SrtError(code, where)
