"""ctypes face of ``cmatvec.c``: the plain C / OpenMP CPU baseline of the compressed H-matrix-vector
product (TEST INFRASTRUCTURE ONLY: used by the tests and by the benchmark's CPU-baseline and
reference legs; the product library never loads it).

The library is built by ``build()`` (gcc, OpenMP, no FP contraction) next to this file. Inputs
are plain numpy arrays: the FP64 blocks of an H-matrix in cluster order and its permutation.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "cmatvec.c")
LIB = os.path.join(HERE, "liboracle_cmatvec.so")

_lib = None


def build(force: bool = False) -> str:
    """Compile cmatvec.c (when it is newer than the library) and return the library path."""
    if force or not os.path.exists(LIB) or os.path.getmtime(SRC) > os.path.getmtime(LIB):
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", SRC, "-o", LIB, "-lm"]
        r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
        if r.returncode != 0:
            raise RuntimeError("oracle C build failed:\n" + " ".join(cmd) + "\n" + r.stdout)
    return LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(LIB)
        vp = C.c_void_p
        L.hlro_build.restype = vp
        L.hlro_build.argtypes = [C.c_int64, vp, C.c_int64, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, C.c_double]
        L.hlro_matvec.restype = C.c_int
        L.hlro_matvec.argtypes = [vp, vp, vp, C.c_int, C.c_int]
        L.hlro_free.argtypes = [vp]
        L.hlro_bytes.restype = C.c_double
        L.hlro_bytes.argtypes = [vp, C.c_int]
        L.hlro_units.restype = C.c_int64
        L.hlro_units.argtypes = [vp]
        L.hlro_unit_info.argtypes = [vp, C.c_int64, vp, vp, vp, vp]
        L.hlro_unit_decode.argtypes = [vp, C.c_int64, vp]
        L.hlro_mantissa_bits.restype = C.c_int
        L.hlro_mantissa_bits.argtypes = [C.c_double]
        _lib = L
    return _lib


class CMatrix:
    """A matrix compressed by the C baseline (AFL dense leaves at eps, AFL-APLR lowrank columns).

    blocks: sequence of dicts with row0, nrows, col0, ncols, kind (0 dense, 1 lowrank) and D
    (nrows x ncols) or W (nrows x k), S (k), X (ncols x k) as FP64 arrays; the arrays are kept
    alive here (the plain product reads them)."""

    def __init__(self, n: int, perm: np.ndarray, blocks, eps: float):
        L = lib()
        nb = len(blocks)
        self.n = int(n)
        self._keep = []
        f = lambda k: np.zeros(nb, dtype=np.int64)
        r0, nr, c0, nc = f(0), f(0), f(0), f(0)
        kind = np.zeros(nb, dtype=np.int32)
        rank = np.zeros(nb, dtype=np.int32)
        ptr = {k: np.zeros(nb, dtype=np.uint64) for k in "DWSX"}
        for i, b in enumerate(blocks):
            r0[i], nr[i], c0[i], nc[i] = b["row0"], b["nrows"], b["col0"], b["ncols"]
            kind[i] = 0 if int(b["kind"]) == 0 else 1
            if kind[i] == 0:
                D = np.asfortranarray(b["D"], dtype=np.float64)
                self._keep.append(D)
                ptr["D"][i] = D.ctypes.data
            else:
                S = np.ascontiguousarray(b["S"], dtype=np.float64)
                rank[i] = S.size
                if S.size:
                    W = np.asfortranarray(b["W"], dtype=np.float64)
                    X = np.asfortranarray(b["X"], dtype=np.float64)
                    self._keep += [S, W, X]
                    ptr["S"][i], ptr["W"][i], ptr["X"][i] = S.ctypes.data, W.ctypes.data, X.ctypes.data
        self._keep += [r0, nr, c0, nc, kind, rank, ptr]
        perm = np.ascontiguousarray(perm, dtype=np.int64)
        self.h = L.hlro_build(self.n, perm.ctypes.data, nb, r0.ctypes.data, nr.ctypes.data, c0.ctypes.data,
                              nc.ctypes.data, kind.ctypes.data, rank.ctypes.data, ptr["D"].ctypes.data,
                              ptr["W"].ctypes.data, ptr["S"].ctypes.data, ptr["X"].ctypes.data, float(eps))
        if not self.h:
            raise RuntimeError("hlro_build failed (non-finite data or out of memory)")

    def matvec(self, x: np.ndarray, y: np.ndarray, plain: bool = False, threads: int = 0) -> np.ndarray:
        """y += A~ x (original order) on `threads` threads (0: all); plain=True uses the FP64
        factors themselves (the uncompressed H-matrix-vector product)."""
        x = np.ascontiguousarray(x, dtype=np.float64)
        if not (isinstance(y, np.ndarray) and y.dtype == np.float64 and y.flags.c_contiguous):
            raise ValueError("y must be a contiguous float64 array")
        if lib().hlro_matvec(self.h, x.ctypes.data, y.ctypes.data, int(plain), int(threads)) != 0:
            raise MemoryError("hlro_matvec: scratch allocation failed")
        return y

    def algorithmic_bytes(self, plain: bool = False) -> float:
        return float(lib().hlro_bytes(self.h, int(plain)))

    def units(self) -> int:
        return int(lib().hlro_units(self.h))

    def unit(self, u: int):
        """(m_min, e, m, decoded values) of unit u (upload order)."""
        n = C.c_int64(0)
        mm = C.c_double(0)
        e = C.c_int32(0)
        m = C.c_int32(0)
        lib().hlro_unit_info(self.h, int(u), C.byref(n), C.byref(mm), C.byref(e), C.byref(m))
        out = np.zeros(n.value, dtype=np.float64)
        lib().hlro_unit_decode(self.h, int(u), out.ctypes.data)
        return mm.value, e.value, m.value, out

    def free(self):
        if self.h:
            lib().hlro_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass
