"""ctypes loader for the in-tree CUDA library ``_build/libtdgemm.so``.

Argument marshalling only; every step of the computation runs in the library's
kernels.  There is no fallback: if the library is missing or fails to load the
import raises.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libtdgemm.so")

TDG_F32, TDG_F64 = 0, 1
FORMS = {"plain": 0, "sym": 1, "asym": 2, "tc_int": 3, "tc_fp8": 4}
DTYPES = {"f32": TDG_F32, "f64": TDG_F64}
TDG_ALLOW_FALLBACK = 0x1
TDG_KEEP_PACKED = 0x2
TDG_NOISE_RMS = 0x4
TDG_PAIR_EXACT = 0x8
TDG_NOISE_UNIFORM = 0x10
STATUS = {0: "TDG_OK", 1: "TDG_EINVAL", 2: "TDG_ENOMEM", 3: "TDG_ECUDA", 4: "TDG_EUNSUPPORTED",
          5: "TDG_EUNREACHABLE", 6: "TDG_ETIMEOUT", 7: "TDG_ENONFINITE", 8: "TDG_ESTATE"}

# every symbol include/tdgemm.h declares
EXPORTS = ["tdgemm_plan", "tdgemm_set_rep_noise", "tdgemm_set_manual",
           "tdgemm_set_kernel_control", "tdgemm_kernel_mask", "tdgemm_quantize_pack",
           "tdgemm_quantize_pack_a",
           "tdgemm_gemm", "tdgemm_run", "tdgemm_run_host", "tdgemm_run_host_async", "tdgemm_unpack",
           "tdgemm_plan_info",
           "tdgemm_plan_destroy", "tdgemm_snr", "tdgemm_run_static", "tdgemm_set_wait_test",
           "tdgemm_set_speedup",
           "tdgemm_fma_probe", "tdgemm_last_error", "tdgemm_version"]


class Info(ctypes.Structure):
    _fields_ = [("W_used", ctypes.c_int32), ("q", ctypes.c_int32), ("gamma_a", ctypes.c_int32),
                ("gamma_b", ctypes.c_int32), ("r_max", ctypes.c_int64), ("w_ef", ctypes.c_int32),
                ("level", ctypes.c_int32), ("pred_snr_db", ctypes.c_double),
                ("workspace_bytes", ctypes.c_int64), ("device_status", ctypes.c_int32),
                ("carrier", ctypes.c_int32)]


class TDGemmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"tdgemm CUDA library not built ({path}); run "
                          "`python -m paper_1110_5765_gb300.build`")
    L = ctypes.CDLL(path)
    vp, i64, i32, dbl, u32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_uint32
    L.tdgemm_plan.argtypes = [ctypes.POINTER(vp), ctypes.c_char, ctypes.c_char, i64, i64, i64,
                              i64, i64, i64, i32, i32, i32, i32, dbl, i32, u32]
    L.tdgemm_set_rep_noise.argtypes = [vp, i32, ctypes.POINTER(dbl), i32, i32]
    L.tdgemm_set_manual.argtypes = [vp, i32, dbl, dbl]
    L.tdgemm_set_kernel_control.argtypes = [vp, i32, dbl]
    L.tdgemm_kernel_mask.argtypes = [vp, vp, i64]
    L.tdgemm_quantize_pack.argtypes = [vp, vp, vp, vp]
    L.tdgemm_quantize_pack_a.argtypes = [vp, vp, vp]
    L.tdgemm_gemm.argtypes = [vp, vp, dbl, dbl, vp]
    L.tdgemm_run.argtypes = [vp, vp, vp, vp, dbl, dbl, vp]
    L.tdgemm_run_host.argtypes = [vp, vp, vp, vp, dbl, dbl, vp]
    L.tdgemm_run_host_async.argtypes = [vp, vp, vp, vp, dbl, dbl, vp]
    L.tdgemm_unpack.argtypes = [vp, vp, vp, vp]
    L.tdgemm_plan_info.argtypes = [vp, ctypes.POINTER(Info)]
    L.tdgemm_plan_destroy.argtypes = [vp]
    L.tdgemm_snr.argtypes = [vp, i64, i32, vp, i64, i64, i64, vp, vp]
    L.tdgemm_run_static.argtypes = [ctypes.c_char, ctypes.c_char, i64, i64, i64, i64, i64, i64,
                                    i32, i32, i32, i32, i32, vp, vp, vp, dbl, dbl, vp]
    L.tdgemm_set_wait_test.argtypes = [vp, i64]
    L.tdgemm_set_speedup.argtypes = [vp, i32, dbl]
    L.tdgemm_fma_probe.argtypes = [i32, i64, ctypes.POINTER(dbl), vp]
    L.tdgemm_last_error.restype = ctypes.c_char_p
    L.tdgemm_version.restype = ctypes.c_char_p
    for name in EXPORTS:
        if name not in ("tdgemm_last_error", "tdgemm_version"):
            getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def check(status: int):
    if status != 0:
        msg = _lib.tdgemm_last_error().decode(errors="replace") if _lib else ""
        raise TDGemmError(status, msg)
