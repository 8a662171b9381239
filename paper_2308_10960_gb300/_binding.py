"""ctypes binding of the C ABI declared in ``include/hlr.h`` (argument marshalling only).

Every computation runs in ``libhlr_gb300.so``; this module converts Python/numpy/torch
arguments to plain pointers and sizes and raises :class:`HlrError` on a negative status.
The library must have been built (``__graft_entry__.build()``); importing this module fails
loudly when it is missing.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhlr_gb300.so")

HLR_OK = 0
HLR_ERR_INVALID = -1
HLR_ERR_OOM = -2
HLR_ERR_CUDA = -3
HLR_ERR_TIMEOUT = -4
HLR_ERR_NOCONV = -5
HLR_ERR_UNSUPPORTED = -6
HLR_DENSE = 0
HLR_LOWRANK = 1
HLR_FMT_AFL_APLR = 1
HLR_FMT_FP64 = 2
HLR_FMT_AFLP = 3
HLR_FMT_BFL = 4
HLR_FMT_DFL = 5
HLR_FMT_MP = 6
HLR_ACC_FP64 = 0
HLR_ACC_FP32 = 1
HLR_PROFILE = 0x100
HLR_MULTI = 0x200
HLR_DECODE_MAP = 1 << 16
HLR_ENCODE_DEVICE = 1 << 17
HLR_KERNEL_EXP = 1
HLR_KERNEL_LAPLACE = 2
HLR_KERNEL_MATERN15 = 3

_ERRNAMES = {
    HLR_ERR_INVALID: "HLR_ERR_INVALID", HLR_ERR_OOM: "HLR_ERR_OOM", HLR_ERR_CUDA: "HLR_ERR_CUDA",
    HLR_ERR_TIMEOUT: "HLR_ERR_TIMEOUT", HLR_ERR_NOCONV: "HLR_ERR_NOCONV",
    HLR_ERR_UNSUPPORTED: "HLR_ERR_UNSUPPORTED",
}

_dp = C.POINTER(C.c_double)
_i64p = C.POINTER(C.c_int64)


class BlockDesc(C.Structure):
    _fields_ = [("row0", C.c_int64), ("nrows", C.c_int64), ("col0", C.c_int64), ("ncols", C.c_int64),
                ("kind", C.c_int32), ("rank", C.c_int32), ("D", _dp), ("W", _dp), ("sigma", _dp), ("X", _dp)]


class HMatrixDesc(C.Structure):
    _fields_ = [("n", C.c_int64), ("perm", _i64p), ("nblocks", C.c_int64), ("blocks", C.POINTER(BlockDesc)),
                ("eps", C.c_double), ("format", C.c_int32), ("tuning", C.c_int32)]


class Info(C.Structure):
    _fields_ = [("n", C.c_int64), ("nblocks", C.c_int64), ("ndense", C.c_int64), ("nlowrank", C.c_int64),
                ("nunits", C.c_int64), ("nleaves", C.c_int64), ("nitems", C.c_int64), ("rank_sum", C.c_int64),
                ("values", C.c_int64), ("fp64_bytes", C.c_uint64), ("stream_bytes", C.c_uint64),
                ("header_bytes", C.c_uint64), ("algorithmic_bytes", C.c_uint64), ("device_bytes", C.c_uint64),
                ("flops", C.c_double), ("phase1_bytes", C.c_uint64), ("phase2_bytes", C.c_uint64),
                ("launches", C.c_int64)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class KernelProblem(C.Structure):
    _fields_ = [("kernel", C.c_int32), ("dim", C.c_int32), ("n", C.c_int64), ("points", _dp),
                ("scale", C.c_double), ("diag", C.c_double), ("eps", C.c_double), ("eta", C.c_double),
                ("leaf_size", C.c_int32), ("threads", C.c_int32)]


# (name, restype, argtypes): every symbol that include/hlr.h declares
SIGNATURES = [
    ("hlr_upload", C.c_int, [C.POINTER(HMatrixDesc), C.c_void_p, C.POINTER(C.c_uint64), C.POINTER(C.c_size_t)]),
    ("hlr_matvec", C.c_int, [C.c_uint64, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    ("hlr_matvec_host", C.c_int, [C.c_uint64, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    ("hlr_matvec_batched", C.c_int, [C.c_int, C.POINTER(C.c_uint64), C.POINTER(C.c_int32), C.POINTER(C.c_void_p),
                                     C.POINTER(C.c_int64), C.POINTER(C.c_void_p), C.POINTER(C.c_int64), C.c_int,
                                     C.c_void_p]),
    ("hlr_solve_cg", C.c_int, [C.c_uint64, C.c_void_p, C.c_void_p, C.c_double, C.c_int, C.c_int, C.c_void_p,
                               C.POINTER(C.c_int), C.POINTER(C.c_double)]),
    ("hlr_check", C.c_int, [C.c_uint64, C.c_void_p]),
    ("hlr_selftest_wait", C.c_int, [C.c_uint64, C.c_int64, C.c_void_p]),
    ("hlr_free", C.c_int, [C.c_uint64]),
    ("hlr_last_error", C.c_char_p, []),
    ("hlr_get_info", C.c_int, [C.c_uint64, C.POINTER(Info)]),
    ("hlr_profile_read", C.c_int, [C.c_uint64, C.POINTER(C.c_double), C.POINTER(C.c_int)]),
    ("hlr_afl_encode", C.c_int, [_dp, C.c_int64, C.c_double, _dp, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                 C.c_void_p, C.c_size_t, C.POINTER(C.c_size_t)]),
    ("hlr_encode", C.c_int, [C.c_int32, _dp, C.c_int64, C.c_double, _dp, C.POINTER(C.c_int32),
                             C.POINTER(C.c_int32), C.c_void_p, C.c_size_t, C.POINTER(C.c_size_t)]),
    ("hlr_encode_device", C.c_int, [C.c_int32, C.c_int64, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p,
                                    C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p]),
    ("hlr_afl_decode_device", C.c_int, [C.c_void_p, C.c_int64, C.c_double, C.c_int32, C.c_int32, C.c_void_p,
                                        C.c_void_p]),
    ("hlr_decode_units", C.c_int, [C.c_uint64, C.c_void_p, C.c_int64, C.c_void_p]),
    ("hlr_decode_units_static", C.c_int, [C.c_uint64, C.c_void_p, C.c_int64, C.c_void_p]),
    ("hlr_unit_list", C.c_int, [C.POINTER(HMatrixDesc), C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_int64,
                                C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    ("hlr_build", C.c_int, [C.POINTER(KernelProblem), C.POINTER(C.c_void_p)]),
    ("hlr_host_describe", C.c_int, [C.c_void_p, C.POINTER(HMatrixDesc)]),
    ("hlr_host_free", None, [C.c_void_p]),
    ("hlr_host_save", C.c_int, [C.c_void_p, C.c_char_p]),
    ("hlr_host_load", C.c_int, [C.c_char_p, C.POINTER(C.c_void_p)]),
]


class HlrError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_ERRNAMES.get(code, code)}: {msg}")
        self.code = code


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`")
    lib = C.CDLL(LIB_PATH)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = _load()


def check(code: int) -> int:
    if code < 0:
        raise HlrError(code, lib.hlr_last_error().decode())
    return code


def f64ptr(a: np.ndarray):
    return a.ctypes.data_as(_dp)
