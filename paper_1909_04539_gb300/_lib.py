"""ctypes binding of libbsolve.so: symbol signatures only.  The library must
have been built (``paper_1909_04539_gb300.build.build()``); there is no
fallback implementation."""
from __future__ import annotations

import ctypes
import os

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "lib", "libbsolve.so")

_LIB = None

i32, i64, vp, dp = ctypes.c_int, ctypes.c_int64, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)

# name -> (restype, argtypes); kept in the order of include/*.h
SIGNATURES = {
    "bs_factor": (i32, [dp, i32, i64, ctypes.POINTER(vp)]),
    "bs_factor_periodic": (i32, [dp, i64, ctypes.POINTER(vp)]),
    "bs_destroy": (i32, [vp]),
    "bs_handle_info": (i32, [vp, ctypes.POINTER(i32), ctypes.POINTER(i64), ctypes.POINTER(ctypes.c_size_t)]),
    "bs_lhs_bytes": (i64, [i32, i64, i32]),
    "bs_solve": (i32, [vp, vp, i32, i32, i64, vp]),
    "bs_solve_bf16": (i32, [vp, vp, vp, i32, i64, vp]),
    "bs_solve_refine": (i32, [vp, vp, i32, vp, i32, i64, i32, i32, vp]),
    "bs_solve_adjoint": (i32, [vp, vp, i32, i32, i64, vp, vp, vp]),
    "bs_adi_halfstep": (i32, [vp, vp, vp, i32, i64, i64, ctypes.c_double, i32, i32, vp]),
    "bs_cn_steps": (i32, [vp, vp, i32, i32, i64, i32, vp]),
    "bs_band_grad": (i32, [vp, vp, vp, i32, i32, i64, vp, vp]),
    "bs_band_grad_noalloc": (i32, [vp, vp, vp, i32, i32, i64, vp, vp]),
    "bs_server_create": (i32, [ctypes.c_size_t, i32, ctypes.POINTER(vp)]),
    "bs_server_destroy": (i32, [vp]),
    "bs_server_submit": (i32, [vp, vp, vp, vp, i32, i64, ctypes.POINTER(i64)]),
    "bs_server_poll": (i32, [vp, i64, ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_double)]),
    "bs_server_wait": (i32, [vp, i64, ctypes.c_double, ctypes.POINTER(i32)]),
    "bs_server_cancel": (i32, [vp, i64]),
    "bs_server_release": (i32, [vp, i64]),
    "bs_server_pause": (i32, [vp, i32]),
    "bs_server_fail_on_admit": (i32, [vp, i64]),
    "bs_server_stats": (i32, [vp, ctypes.POINTER(i64), i32]),
    "bs_set_option": (i32, [i32, i64]),
    "bs_device_status": (i32, [ctypes.POINTER(i32), i32]),
    "bs_measure_fp64_rate": (i32, [dp, vp]),
    "bs_last_error": (ctypes.c_char_p, []),
    "bs_strerror": (ctypes.c_char_p, [i32]),
}


class BsolveError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(msg)
        self.status = status


def lib() -> ctypes.CDLL:
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"libbsolve.so is not built ({LIB_PATH} missing); run "
                "paper_1909_04539_gb300.build.build() -- there is no CPU fallback")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = L
    return _LIB


def check(status: int, fn: str) -> None:
    if status != 0:
        L = lib()
        raise BsolveError(status, f"{fn}: {L.bs_strerror(status).decode()}: {L.bs_last_error().decode()}")
