"""ctypes view of libsho.so (the C ABI of include/sho.h).  Argument marshalling only."""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libsho.so")

SHO_OK = 0
SHO_ERR_CUDA = -7
STATUS_NAMES = {
    0: "SHO_OK", -1: "SHO_ERR_ARG", -2: "SHO_ERR_NUMAX", -3: "SHO_ERR_CUBE", -4: "SHO_ERR_SPACING",
    -5: "SHO_ERR_DTYPE", -6: "SHO_ERR_OOM", -7: "SHO_ERR_CUDA", -8: "SHO_ERR_TIMEOUT", -9: "SHO_ERR_DEVICE",
    -10: "SHO_ERR_CAPACITY", -11: "SHO_ERR_STATE", -12: "SHO_ERR_CANCELLED",
}
DTYPES = {"f64": 0, "f32": 1, "bf16": 2}
PRECS = {"fp64": 0, "fp32": 1, "tf32": 2, "3xtf32": 3, "bf16": 4, "split_fp16": 5, "ff64": 6}


class ShoError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        msg = lib().sho_strerror(status).decode() if _lib is not None else ""
        super().__init__(f"{what}: {STATUS_NAMES.get(status, status)} ({msg})")


class sho_grid(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int * 3), ("h", ctypes.c_double), ("periodic", ctypes.c_int)]


class sho_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64), ("failed", ctypes.c_uint64),
                ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double), ("mean_ms", ctypes.c_double),
                ("max_ms", ctypes.c_double), ("busy_seconds", ctypes.c_double),
                ("algorithmic_bytes", ctypes.c_double), ("gbs", ctypes.c_double),
                ("resident_bytes", ctypes.c_size_t), ("workspace_bytes", ctypes.c_size_t),
                ("peak_bytes", ctypes.c_size_t), ("max_inflight", ctypes.c_int)]


_lib = None
_lock = threading.Lock()

_VP = ctypes.c_void_p
_DP = ctypes.POINTER(ctypes.c_double)
_IP = ctypes.POINTER(ctypes.c_int)
_I = ctypes.c_int
_GP = ctypes.POINTER(sho_grid)

# name -> (restype, argtypes); every symbol declared in include/*.h
SIGNATURES = {
    "sho_version": (_I, []),
    "sho_nstates": (_I, [_I]),
    "sho_max_spacing": (ctypes.c_double, [ctypes.c_double, _I]),
    "sho_strerror": (ctypes.c_char_p, [_I]),
    "sho_create": (_I, [ctypes.POINTER(_VP), _I]),
    "sho_destroy": (_I, [_VP]),
    "sho_set_strict": (_I, [_VP, _I]),
    "sho_set_support_radius": (_I, [_VP, ctypes.c_double]),
    "sho_set_expand_kernel": (_I, [_VP, _I]),
    "sho_set_project_kernel": (_I, [_VP, _I]),
    "sho_set_device_checks": (_I, [_VP, _I]),
    # include/sho_selftest.h
    "sho_selftest_umma": (_I, [_I, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float),
                               ctypes.POINTER(ctypes.c_float)]),
    "sho_selftest_ozaki": (_I, [ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float),
                                ctypes.POINTER(ctypes.c_float)]),
    "sho_sync": (_I, [_VP]),
    "sho_last_cuda_error": (ctypes.c_char_p, [_VP]),
    "sho_project_path": (_I, [_GP, _VP, _I, _I, _I, _I, _I, _I]),
    "sho_plane_plan_check": (_I, [_GP, _I, _DP, _DP, _I, _IP, _IP]),
    "sho_project_bloch": (_I, [_VP, _GP, _DP, _VP, _I, _I, _DP, _DP, _I, _I, _I, _VP, _VP]),
    "sho_add_bloch": (_I, [_VP, _GP, _DP, _VP, _I, _I, _DP, _DP, _I, _I, _I, _VP, _VP]),
    "sho_radial_labels": (_I, [_I, _IP, _IP, _IP]),
    "sho_radial_matrix": (_I, [_I, _DP]),
    "sho_radial_transform": (_I, [_VP, _I, _I, _I, _VP, _VP, _I, _I, _VP]),
    "sho_project": (_I, [_VP, _GP, _VP, _I, _I, _I, _DP, _DP, _I, _I, _I, _VP, _I, _VP]),
    "sho_add": (_I, [_VP, _GP, _VP, _I, _I, _I, _DP, _DP, _I, _I, _I, _VP, _I, _VP]),
    "sho_add_scaled": (_I, [_VP, _GP, ctypes.c_double, _I, _VP, _I, _I, _I, _DP, _DP, _I, _I, _I, _VP, _I, _VP]),
    "sho_forces": (_I, [_VP, _GP, _VP, _I, _I, _I, _DP, _DP, _I, _I, _I, _VP, _I, _DP, _VP]),
    "sho_forces_noalloc": (_I, [_GP, _VP, _I, _I, _I, _DP, _DP, _I, _I, _I, _VP, _I, _DP, _VP]),
    "sho_apply_nonlocal": (_I, [_VP, _GP, _VP, _I, _I, _I, _DP, _DP, _I, _I, _I, _VP, _VP, _VP]),
    "sho_usu_build": (_I, [_VP, _GP, _I, _DP, _DP, _I, _I, _I, _I, _VP, _VP]),
    "sho_usu_project": (_I, [_VP, _GP, _VP, _I, _I, _DP, _DP, _I, _I, _I, _VP, _VP, _VP]),
    "sho_usu_add": (_I, [_VP, _GP, _VP, _I, _I, _DP, _DP, _I, _I, _I, _VP, _VP, _VP]),
    "sho_server_create": (_I, [ctypes.POINTER(_VP), _I, ctypes.c_size_t, _I]),
    "sho_server_destroy": (_I, [_VP]),
    "sho_system_register": (_I, [_VP, _GP, _I, _I, _DP, _DP, _I, _I, _I, _VP, ctypes.POINTER(_I)]),
    "sho_system_unregister": (_I, [_VP, _I]),
    "sho_system_read": (_I, [_VP, _I, _VP, _VP]),
    "sho_system_write_coeff": (_I, [_VP, _I, _VP]),
    "sho_submit": (_I, [_VP, _I, _I, _I, ctypes.POINTER(ctypes.c_uint64)]),
    "sho_wait": (_I, [_VP, ctypes.c_uint64, _I]),
    "sho_cancel": (_I, [_VP, ctypes.c_uint64]),
    "sho_wait_status": (_I, [_VP, ctypes.c_uint64, _I, _IP, _DP]),
    "sho_server_get_stats": (_I, [_VP, ctypes.POINTER(sho_server_stats)]),
    "sho_server_reset_stats": (_I, [_VP]),
    # include/sho_fault.h
    "sho_fault_wait_limit": (_I, [_VP, ctypes.c_longlong]),
    "sho_fault_stop_rows": (_I, [_VP, _I]),
    "sho_fault_check_extent": (_I, [_VP, ctypes.c_longlong]),
    "sho_fault_hold": (_I, [_VP, _I, _I]),
    "sho_fault_server_pipeline": (_I, [_VP, ctypes.c_longlong, _I]),
}


def lib():
    """Load libsho.so; raises if it has not been built (there is no fallback path)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    f"{LIB_PATH} is missing: build the CUDA library first "
                    "(python -m paper_1905_00480_gb300.build); there is no CPU fallback")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def check(status: int, what: str):
    if status != SHO_OK:
        raise ShoError(status, what)
