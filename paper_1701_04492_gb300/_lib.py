"""ctypes loader of the in-tree libnufft.so (the C ABI of include/nufft.h).

Argument marshalling only.  The library must have been built (``build()`` in
``paper_1701_04492_gb300.build``); a missing library is an error, never a fallback.
"""

from __future__ import annotations

import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
# NUFFT_LIB selects another build of the same ABI, e.g. the checked libnufft_check.so
LIB_PATH = os.environ.get("NUFFT_LIB") or os.path.join(_PKG, "libnufft.so")

NUFFT_F32, NUFFT_F64 = 0, 1
NUFFT_PLAN_UNFUSED = 1
NUFFT_PLAN_TIMING = 2
NUFFT_PLAN_AUTOTUNE = 4
NUFFT_BATCH_GRAPH = 8
NUFFT_PLAN_LONG_COLUMNS = 16
NUFFT_BATCH_PER_PROBLEM = 32
NUFFT_PLAN_HALF_TILE = 64
NUFFT_BATCH_PERSISTENT = 128
NUFFT_RESERVE_STEP_HOST = 1
STATUS = {0: "NUFFT_OK", -1: "NUFFT_EINVAL", -2: "NUFFT_ENOMEM", -3: "NUFFT_ECUDA",
          -4: "NUFFT_EUNSUPPORTED", -5: "NUFFT_ESTATE", -6: "NUFFT_ETIMEOUT",
          -7: "NUFFT_ECHECK"}

# name -> (restype, argtypes), mirroring include/nufft.h
_vp, _i64, _i32, _dbl, _u32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_uint
SIGNATURES = {
    "nufft2_plan": (_i32, [ctypes.POINTER(_vp), _i64, _i64, _vp, _dbl, _i32, _i64, _u32, _vp]),
    "nufft2_plan_info": (_i32, [_vp, ctypes.POINTER(_i32), ctypes.POINTER(_dbl), ctypes.POINTER(_i64),
                                ctypes.POINTER(_i64)]),
    "nufft2_plan_export": (_i32, [_vp, _vp, _vp, ctypes.POINTER(_dbl), _vp]),
    "nufft_destroy": (_i32, [_vp]),
    "nufft2_exec": (_i32, [_vp, _vp, _vp, _vp]),
    "nufft1_exec": (_i32, [_vp, _vp, _vp, _vp]),
    "nufft2_exec_dx": (_i32, [_vp, _vp, _vp, _vp, _i32, _vp]),
    "nufft2_exec_deriv": (_i32, [_vp, _vp, _vp, _vp, _vp]),
    "nufft2_grad_x": (_i32, [_vp, _vp, _vp, _vp, _i32, _vp]),
    "nufft_rank": (_i32, [_dbl, _dbl, ctypes.POINTER(_i32)]),
    "nufft_lowrank_coeffs": (_i32, [_i32, _dbl, ctypes.POINTER(_dbl)]),
    "nufft_tune_save": (_i32, [ctypes.c_char_p, ctypes.POINTER(_i64)]),
    "nufft_tune_load": (_i32, [ctypes.c_char_p, ctypes.POINTER(_i64)]),
    "nufft_tune_clear": (_i32, [ctypes.POINTER(_i64)]),
    "nufft2_exec_batch": (_i32, [_vp, _i64, _vp, _i64, _vp, _i64, _vp]),
    "nufft1_exec_batch": (_i32, [_vp, _i64, _vp, _i64, _vp, _i64, _vp]),
    "nufft2_exec_deriv_batch": (_i32, [_vp, _i64, _vp, _i64, _vp, _vp, _i64, _vp]),
    "nufft2_grad_x_batch": (_i32, [_vp, _i64, _vp, _vp, _i64, _vp, _i32, _vp]),
    "nufft2_exec_host": (_i32, [_vp, _vp, _vp, _vp]),
    "nufft2_plan_reserve": (_i32, [_vp, _i64, _u32, _vp]),
    "nufft2_plan_reserved": (_i32, [_vp, ctypes.POINTER(_i64), ctypes.POINTER(_i32)]),
    "nufft2_step_host": (_i32, [_vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "nufft2_exec_unfused": (_i32, [_vp, _vp, _vp, _vp]),
    "nufft_kernel_times": (_i32, [_vp, ctypes.POINTER(ctypes.c_float), _i32, ctypes.POINTER(_i32)]),
    "nufft2_check": (_i32, [_vp, _vp]),
    "nufft2_exec_noalloc": (_i32, [_i64, _i64, _vp, _dbl, _vp, _vp, _vp]),
    "nufft_strerror": (ctypes.c_char_p, [_i32]),
    "nufft_fp32_fma_peak": (_i32, [_i64, _i32, _vp, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(_dbl)]),
    "nufft_test_fail_alloc": (_i32, [_i32]),
    "nufft_test_wait_timeout": (_i32, [_vp]),
    "nufft2_inverse": (_i32, [_vp, _vp, _vp, _dbl, _i32, ctypes.POINTER(_i32), ctypes.POINTER(_dbl), _vp]),
    "nufft2d_plan": (_i32, [ctypes.POINTER(_vp), _i64, _i64, _i64, _vp, _vp, _dbl, _i32, _u32, _vp]),
    "nufft2d_plan_info": (_i32, [_vp, ctypes.POINTER(_i32), ctypes.POINTER(_i32), ctypes.POINTER(_dbl),
                                 ctypes.POINTER(_dbl), ctypes.POINTER(_i64), ctypes.POINTER(_i64)]),
    "nufft2_plan_many": (_i32, [ctypes.POINTER(_vp), _i64, _vp, _vp, _vp, _vp, _vp, _i32, _u32, _vp]),
    "nufft_batch_info": (_i32, [_vp, ctypes.POINTER(_i64), ctypes.POINTER(_i64), ctypes.POINTER(_i64), _vp, _vp]),
    "nufft2_exec_many": (_i32, [_vp, _vp, _vp, _vp]),
    "nufft1_exec_many": (_i32, [_vp, _vp, _vp, _vp]),
    "nufft2_exec_each": (_i32, [_vp, _vp, _vp, _i32, _vp]),
    "nufft_batch_check": (_i32, [_vp, _vp]),
    "nufft_batch_launches": (_i32, [_vp, ctypes.POINTER(_i64)]),
    "nufft_batch_destroy": (_i32, [_vp]),
}

_lib = None


class NufftError(RuntimeError):
    def __init__(self, code, what=""):
        self.code = code
        name = STATUS.get(code, str(code))
        msg = _lib.nufft_strerror(code).decode() if _lib is not None else name
        super().__init__("%s failed: %s (%s)" % (what, name, msg))


def load():
    """Load libnufft.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("%s is not built (run paper_1701_04492_gb300.build.build()); "
                               "there is no CPU fallback" % LIB_PATH)
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def check(code, what):
    if code != 0:
        raise NufftError(code, what)
