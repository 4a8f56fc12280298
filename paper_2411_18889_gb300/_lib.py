"""ctypes declarations of libnbody's C ABI (include/nbody.h).

Loading fails loudly when the shared library has not been built: there is no
fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
import re

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libnbody.so")
HEADER = os.path.join(os.path.dirname(PKG), "include", "nbody.h")

NBODY_OK = 0
NBODY_EINVAL = -1
NBODY_ENOMEM = -2
NBODY_ECUDA = -3
NBODY_ETIMEOUT = -4
NBODY_ENOTSUP = -5
NBODY_EBOUNDS = -6
NBODY_PREC_MIXED = 0
NBODY_PREC_PLAIN = 1
NBODY_PREC_MIXED_UNSORTED = 2
NBODY_ACC_COMPENSATED = 0
NBODY_ACC_FP32 = 1
NBODY_ACC_KAHAN_PAIR = 2


class NbodyOpts(ctypes.Structure):
    _fields_ = [("stream", ctypes.c_void_p), ("precision", ctypes.c_int), ("accumulate", ctypes.c_int),
                ("config", ctypes.c_int), ("reserved", ctypes.c_int)]


class NbodyError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {strerror(code)} ({code})")


_lib = None

_i64, _int, _dbl, _flt, _vp = ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_float, ctypes.c_void_p
_OPTS = ctypes.POINTER(NbodyOpts)
SIGNATURES = {
    "nbody_opts_default": (None, [_OPTS]),
    "nbody_accel": (_int, [_i64, _vp, _vp, _dbl, _vp, _vp, _OPTS]),
    "nbody_accel_f32": (_int, [_i64, _vp, _vp, _flt, _vp, _vp, _OPTS]),
    "nbody_leapfrog": (_int, [_i64, _vp, _vp, _vp, _dbl, _dbl, _i64, _OPTS]),
    "nbody_leapfrog_f32": (_int, [_i64, _vp, _vp, _vp, _flt, _flt, _i64, _OPTS]),
    "nbody_energy": (_int, [_i64, _vp, _vp, _vp, _dbl, _vp, _OPTS]),
    "nbody_energy_f32": (_int, [_i64, _vp, _vp, _vp, _flt, _vp, _OPTS]),
    "nbody_accel_batched": (_int, [_i64, _vp, _vp, _vp, _vp, _vp, _vp, _OPTS]),
    "nbody_leapfrog_batched": (_int, [_i64, _vp, _vp, _vp, _vp, _vp, _dbl, _i64, _OPTS]),
    "nbody_accel_ij": (_int, [_i64, _vp, _i64, _vp, _vp, _dbl, _vp, _vp, _OPTS]),
    "nbody_accel_ij_f32": (_int, [_i64, _vp, _i64, _vp, _vp, _flt, _vp, _vp, _OPTS]),
    "nbody_accel_vjp": (_int, [_i64, _vp, _vp, _dbl, _vp, _vp, _vp, _vp, _OPTS]),
    "nbody_tape_bytes": (_i64, [_i64, _i64, _i64]),
    "nbody_leapfrog_record": (_int, [_i64, _vp, _vp, _vp, _dbl, _dbl, _i64, _i64, _vp, _OPTS]),
    "nbody_leapfrog_vjp_tape": (_int, [_i64, _vp, _dbl, _dbl, _i64, _i64, _vp, _vp, _vp, _vp, _vp, _vp, _OPTS]),
    "nbody_leapfrog_vjp": (_int, [_i64, _vp, _vp, _vp, _dbl, _dbl, _i64, _i64, _vp, _vp, _vp, _vp, _vp, _OPTS]),
    "nbody_tune_load": (_int, [ctypes.c_char_p]),
    "nbody_tuned_shape": (_int, [_int, _i64, _int]),
    "nbody_num_configs": (_int, []),
    "nbody_num_batched_configs": (_int, []),
    "nbody_config_block": (_int, [_int]),
    "nbody_last_device_error": (_int, []),
    "nbody_last_cuda_error": (_int, []),
    "nbody_strerror": (ctypes.c_char_p, [_int]),
    "nbody_selftest_wait": (_int, [_dbl, _OPTS]),
    "nbody_accel_noalloc": (_int, [_i64, _vp, _vp, _dbl, _vp, _vp, _vp, _vp]),
    "nbody_profile_enable": (None, [_int]),
    "nbody_profile_read": (_int, [ctypes.POINTER(_dbl), ctypes.POINTER(_i64), ctypes.POINTER(_i64)]),
    "nbody_profile_read_kind": (_int, [_int, ctypes.POINTER(_dbl), ctypes.POINTER(_i64)]),
    "nbody_finalize": (None, []),
    "nbody_version": (_int, []),
}


def header_functions(path: str = HEADER):
    """Names of the functions include/nbody.h declares."""
    src = open(path).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:NBODY_API\s+)?(?:const\s+)?\w+\s*\*?\s*(nbody_\w+)\s*\(", src,
                                 flags=re.M)))


def open_library(path: str):
    """ctypes handle of a build of the library at `path`, signatures set."""
    if not os.path.exists(path):
        raise ImportError(f"libnbody.so is not built ({path}); run paper_2411_18889_gb300.build.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


def load():
    """Load libnbody.so (build it first: paper_2411_18889_gb300.build)."""
    global _lib
    if _lib is None:
        _lib = open_library(LIB_PATH)
    return _lib


def strerror(code: int) -> str:
    try:
        return load().nbody_strerror(int(code)).decode()
    except ImportError:
        return f"code {code}"


def check(code: int, what: str) -> None:
    if code != NBODY_OK:
        raise NbodyError(code, what)
