"""ctypes binding of libdiagmg.so (include/diagmg.h): argument marshalling only.

Every function here has the name and argument order of its C counterpart.
The library must have been built (``paper_math_9907190_gb300.build.build()``);
there is no fallback: loading fails loudly without it."""

from __future__ import annotations

import ctypes
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdiagmg.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "diagmg.h")

MG_OK, MG_EINVAL, MG_ENOMEM, MG_ECUDA, MG_ENOCONV, MG_EDIVERGED, MG_ETIMEOUT = 0, -1, -2, -3, -4, -5, -6
MG_DIAG, MG_USUAL = 0, 1
MG_FP64, MG_MIXED = 0, 1


class mg_desc(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int), ("pitch", ctypes.c_int),
                ("hierarchy", ctypes.c_int), ("order", ctypes.c_int), ("precision", ctypes.c_int),
                ("coarsest", ctypes.c_int), ("omega", ctypes.c_double * 4)]


_i, _d, _vp = ctypes.c_int, ctypes.c_double, ctypes.c_void_p
_ip, _dp = ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)

SIGNATURES = {
    "mg_create": (_i, [ctypes.POINTER(_vp), ctypes.POINTER(mg_desc)]),
    "mg_destroy": (_i, [_vp]),
    "mg_num_levels": (_i, [_vp, _ip]),
    "mg_level_info": (_i, [_vp, _i, _ip, _ip]),
    "mg_residual": (_i, [_vp, _vp, _vp, _d, _i, _vp, _dp, _vp]),
    "mg_restrict_diag": (_i, [_vp, _i, _vp]),
    "mg_coarse_solve": (_i, [_vp, _vp]),
    "mg_jacobi_prolong": (_i, [_vp, _i, _dp, _vp]),
    "mg_level_get": (_i, [_vp, _i, _i, _vp, _vp]),
    "mg_level_set": (_i, [_vp, _i, _i, _vp, _vp]),
    "mg_vcycle": (_i, [_vp, _vp, _vp, _vp]),
    "mg_solve": (_i, [_vp, _vp, _vp, _d, _i, _ip, _dp, _dp, _vp]),
    "mg_solve_zero": (_i, [_vp, _vp, _vp, _d, _i, _ip, _dp, _dp, _vp]),
    "mg_solve_host": (_i, [_vp, _vp, _vp, _vp, _d, _i, _ip, _dp, _vp]),
    "mg_solve_host_many": (_i, [_vp, _i, _vp, _vp, _d, _i, _ip, _dp, _vp]),
    "mg_fp64_rate": (_i, [_vp, _dp, _vp]),
    "mg_launch_count": (_i, [_vp, ctypes.POINTER(ctypes.c_longlong)]),
    "mg_probe_set": (_i, [_vp, _i]),
    "mg_probe_read": (_i, [_vp, ctypes.POINTER(ctypes.c_longlong), _dp, _vp]),
    "mg_residual_noalloc": (_i, [_i, _i, _i, _d, _i, _vp, _vp, _vp, _vp, _vp]),
    "mg_batch_create": (_i, [ctypes.POINTER(_vp), _i, _i, _ip, _i, _i, _i, _i, _dp]),
    "mg_batch_destroy": (_i, [_vp]),
    "mg_solve_batched": (_i, [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp), _d, _i, _ip, _dp, _vp]),
    "mg_batch_launch_count": (_i, [_vp, ctypes.POINTER(ctypes.c_longlong)]),
    "mg_batch_status": (_i, [_vp, _ip]),
    "mg_tune": (_i, [_vp, _vp, _vp, ctypes.c_char_p, _ip, _vp]),
    "mg_set_omega": (_i, [_vp, _dp]),
    "mg_set_sweeps": (_i, [_vp, _i]),
    "mg_set_gamma": (_i, [_vp, _i]),
    "mg_rho": (_i, [_vp, _vp, _vp, _i, _i, _dp, _vp]),
    "mg_solve_two_stage": (_i, [_vp, _vp, _vp, _dp, _d, _d, _i, _ip, _ip, _dp, _vp]),
    "mg_tune_info": (_i, [_vp, _ip, _ip, _ip, _ip]),
    "mg_batch_tune": (_i, [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.c_char_p, _vp]),
    "mg_strerror": (ctypes.c_char_p, [_i]),
    "mg_last_error": (ctypes.c_char_p, []),
}

_lib = None


def header_functions() -> list[str]:
    """Names of the functions declared in include/diagmg.h."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mg_[a-z0-9_]+)\s*\(", text)))


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built: run paper_math_9907190_gb300.build.build() "
                               "(there is no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype, fn.argtypes = res, args
        _lib = L
    return _lib


class MGError(RuntimeError):
    def __init__(self, status: int, where: str):
        L = lib()
        msg = L.mg_strerror(status).decode()
        detail = L.mg_last_error().decode()
        super().__init__(f"{where}: {msg} ({status}){' — ' + detail if detail and status == MG_ECUDA else ''}")
        self.status = status


def check(status: int, where: str) -> int:
    if status != MG_OK:
        raise MGError(status, where)
    return status


def __getattr__(name):
    if name in SIGNATURES:
        return getattr(lib(), name)
    raise AttributeError(name)
