"""GB300-native compressed H-matrix-vector product (Kriemann, "Hierarchical Lowrank Arithmetic
with Binary Compression", arXiv 2308.10960).

Python face of the C ABI in ``include/hlr.h``. An H-matrix (Def. 2.3) is uploaded once; its
dense leaves are stored in the AFL binary format and its lowrank leaves W Sigma X^T column by
column at adaptive precision (AFL-APLR, Sections 3.2-3.3). ``DeviceHMatrix.matvec`` computes
y += A~ x (Section 5.4) in hand-written sm_103a kernels that decode the bit streams on the fly.
PyTorch provides device memory and streams only.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import _binding as B
from ._binding import (HLR_ACC_FP32, HLR_ACC_FP64, HLR_DENSE, HLR_ENCODE_DEVICE, HLR_ERR_INVALID, HLR_ERR_NOCONV,
                       HLR_FMT_AFL_APLR, HLR_FMT_FP64, HLR_KERNEL_EXP, HLR_KERNEL_LAPLACE, HLR_KERNEL_MATERN15,
                       HLR_LOWRANK, HlrError)

__all__ = [
    "HlrError", "DeviceHMatrix", "HostHMatrix", "upload", "build_kernel_hmatrix", "afl_encode",
    "afl_decode_device", "matvec_batched", "HLR_ACC_FP32", "HLR_ACC_FP64", "HLR_FMT_AFL_APLR", "HLR_FMT_FP64",
    "HLR_DENSE", "HLR_LOWRANK", "HLR_ENCODE_DEVICE", "lib_path", "tuning_code", "encode", "encode_device", "unit_arrays",
    "load_host_hmatrix",
]

_ACC = {"fp32": HLR_ACC_FP32, "fp64": HLR_ACC_FP64, HLR_ACC_FP32: HLR_ACC_FP32, HLR_ACC_FP64: HLR_ACC_FP64}
_FMT = {"afl": HLR_FMT_AFL_APLR, "fp64": HLR_FMT_FP64, "aflp": B.HLR_FMT_AFLP, "bfl": B.HLR_FMT_BFL,
        "dfl": B.HLR_FMT_DFL, "mp": B.HLR_FMT_MP, HLR_FMT_AFL_APLR: HLR_FMT_AFL_APLR, HLR_FMT_FP64: HLR_FMT_FP64,
        B.HLR_FMT_AFLP: B.HLR_FMT_AFLP, B.HLR_FMT_BFL: B.HLR_FMT_BFL, B.HLR_FMT_DFL: B.HLR_FMT_DFL,
        B.HLR_FMT_MP: B.HLR_FMT_MP}
_KERNEL = {"exp2d": HLR_KERNEL_EXP, "exp": HLR_KERNEL_EXP, "laplace": HLR_KERNEL_LAPLACE,
           "matern15": HLR_KERNEL_MATERN15}


def lib_path() -> str:
    return B.LIB_PATH


def _stream_ptr(stream) -> int | None:
    if stream is None:
        import torch
        if not torch.cuda.is_available():
            return None          # legacy default stream; host-only calls fail before using it
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _dev_ptr(t, n: int | None = None, dtype=None) -> int:
    import torch
    dtype = torch.float64 if dtype is None else dtype
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != dtype or not t.is_contiguous():
        raise HlrError(HLR_ERR_INVALID, f"expected a contiguous {dtype} CUDA tensor")
    if n is not None and t.numel() < n:
        raise HlrError(HLR_ERR_INVALID, f"tensor has {t.numel()} elements, need {n}")
    return t.data_ptr()


def _host_ptr(a, n: int) -> int:
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags.c_contiguous or a.size < n:
            raise HlrError(HLR_ERR_INVALID, "expected a contiguous float64 host array")
        return a.ctypes.data
    import torch
    if not isinstance(a, torch.Tensor) or a.is_cuda or a.dtype != torch.float64 or not a.is_contiguous() \
            or a.numel() < n:
        raise HlrError(HLR_ERR_INVALID, "expected a contiguous float64 host tensor")
    return a.data_ptr()


class _DescBuilder:
    """Holds the ctypes descriptor and keeps every referenced numpy array alive."""

    def __init__(self, n: int, perm, blocks, eps: float, fmt: int):
        self.keep = []
        self.n = int(n)
        self.perm = None if perm is None else np.ascontiguousarray(perm, dtype=np.int64)
        arr = (B.BlockDesc * len(blocks))()
        for i, b in enumerate(blocks):
            d = arr[i]
            d.row0, d.nrows, d.col0, d.ncols = int(b["row0"]), int(b["nrows"]), int(b["col0"]), int(b["ncols"])
            d.kind = int(b["kind"])
            if d.kind == HLR_DENSE:
                D = np.asfortranarray(b["D"], dtype=np.float64)
                self.keep.append(D)
                d.D = B.f64ptr(D)
                d.rank = 0
            else:
                S = np.ascontiguousarray(b["S"], dtype=np.float64)
                d.rank = int(S.size)
                if S.size:
                    W = np.asfortranarray(b["W"], dtype=np.float64)
                    X = np.asfortranarray(b["X"], dtype=np.float64)
                    self.keep += [W, X, S]
                    d.W, d.X, d.sigma = B.f64ptr(W), B.f64ptr(X), B.f64ptr(S)
        self.arr = arr
        self.desc = B.HMatrixDesc()
        self.desc.n = self.n
        self.desc.perm = None if self.perm is None else self.perm.ctypes.data_as(B._i64p)
        self.desc.nblocks = len(blocks)
        self.desc.blocks = C.cast(arr, C.POINTER(B.BlockDesc))
        self.desc.eps = float(eps)
        self.desc.format = fmt
        self.desc.tuning = 0


class DeviceHMatrix:
    """An uploaded compressed H-matrix (owns a library handle)."""

    def __init__(self, handle: int):
        self.handle = int(handle)
        inf = B.Info()
        B.check(B.lib.hlr_get_info(C.c_uint64(self.handle), C.byref(inf)))
        self.info = inf.as_dict()
        self.n = int(self.info["n"])

    def matvec(self, x, y, acc="fp32", stream=None, profile=False, sm_share: int = 0):
        """y += A~ x (both contiguous float64 CUDA tensors of length n, original order).
        sm_share: 1..7 eighths of the persistent kernels' CTA slots (HLR_SM_SHARE; 0 = all)."""
        flags = _ACC[acc] | (B.HLR_PROFILE if profile else 0) | (int(sm_share) << 16)
        B.check(B.lib.hlr_matvec(C.c_uint64(self.handle), _dev_ptr(x, self.n), _dev_ptr(y, self.n),
                                 flags, _stream_ptr(stream)))
        return y

    def profile_read(self):
        """(per-kernel milliseconds [permute, phase1, phase2, scatter] summed, number of products)
        of the products launched with profile=True since the previous read."""
        ms = (C.c_double * 4)()
        calls = C.c_int(0)
        B.check(B.lib.hlr_profile_read(C.c_uint64(self.handle), ms, C.byref(calls)))
        return list(ms), calls.value

    def matvec_host(self, x, y, acc="fp32", stream=None):
        """y += A~ x with HOST buffers (numpy arrays or CPU tensors, pinned for async copies):
        copies in, computes on the GPU, copies y back and waits (hlr_matvec_host)."""
        xp = _host_ptr(x, self.n)
        yp = _host_ptr(y, self.n)
        B.check(B.lib.hlr_matvec_host(C.c_uint64(self.handle), xp, yp, _ACC[acc], _stream_ptr(stream)))
        return y

    def solve_cg(self, b, x, rtol=1e-8, maxit=1000, acc="fp64", stream=None, raise_noconv=True, sm_share: int = 0):
        """Solve A~ x = b by CG (x holds the initial guess). Returns (iterations, true rel. residual).
        sm_share: 1..7 eighths of the product kernels' CTA slots (HLR_SM_SHARE; 0 = all)."""
        it = C.c_int(0)
        rel = C.c_double(0.0)
        rc = B.lib.hlr_solve_cg(C.c_uint64(self.handle), _dev_ptr(b, self.n), _dev_ptr(x, self.n), float(rtol),
                                int(maxit), _ACC[acc] | (int(sm_share) << 16), _stream_ptr(stream), C.byref(it),
                                C.byref(rel))
        if rc == HLR_ERR_NOCONV and not raise_noconv:
            return it.value, rel.value
        B.check(rc)
        return it.value, rel.value

    def decode_units(self, out):
        """Decode every stored unit to FP64 on the GPU (bit-exact path), concatenated in unit order."""
        B.check(B.lib.hlr_decode_units(C.c_uint64(self.handle), _dev_ptr(out), out.numel(), _stream_ptr(None)))
        return out

    def decode_units_static(self, out, stream=None):
        """decode_units for callers that cannot allocate device memory: the slice map goes to a
        fixed 4 MiB array of the library (no allocation, no synchronisation; calls that overlap
        on the GPU race)."""
        B.check(B.lib.hlr_decode_units_static(C.c_uint64(self.handle), _dev_ptr(out), out.numel(),
                                              _stream_ptr(stream)))
        return out

    def check(self, stream=None):
        """Wait for the stream; raise HlrError(HLR_ERR_TIMEOUT) if a kernel gave up a bounded wait."""
        B.check(B.lib.hlr_check(C.c_uint64(self.handle), _stream_ptr(stream)))

    def selftest_wait(self, cycles: int = 2_000_000, stream=None):
        """Launch the failure-detection self-test (hlr_selftest_wait): a bounded device wait
        that cannot succeed and gives up after `cycles` clock cycles; the next check() raises
        HlrError(HLR_ERR_TIMEOUT)."""
        B.check(B.lib.hlr_selftest_wait(C.c_uint64(self.handle), int(cycles), _stream_ptr(stream)))

    def free(self):
        if self.handle:
            B.check(B.lib.hlr_free(C.c_uint64(self.handle)))
            self.handle = 0

    def __del__(self):
        try:
            if self.handle:
                B.lib.hlr_free(C.c_uint64(self.handle))
        except Exception:
            pass


def tuning_code(sub_rows: int = 64, leaf_rows: int = 64, piece_kb: int = 16, ctas_per_sm: int = 0) -> int:
    """HLR_TUNING | HLR_CTAS_PER_SM of include/hlr.h: rows per lane of an X column (32/64/128),
    rows of a phase-2 task (32/64), piece size in KiB (4..16), CTAs per SM the work lists are
    made for (0 = as many as are resident, 1..8); the defaults give 0."""
    if sub_rows not in (32, 64, 128) or leaf_rows not in (32, 64) or not 4 <= piece_kb <= 16 \
            or not 0 <= ctas_per_sm <= 8:
        raise HlrError(HLR_ERR_INVALID, "bad tuning")
    shape = int(ctas_per_sm) << 20
    if (sub_rows, leaf_rows, piece_kb) == (64, 64, 16):
        return shape
    return (sub_rows.bit_length() - 1) | ((leaf_rows.bit_length() - 1) << 4) | (piece_kb << 8) | shape


def upload(n: int, perm, blocks, eps: float, fmt="afl", stream=None, tuning: int = 0) -> DeviceHMatrix:
    """Upload an H-matrix given as a list of block dicts (row0, nrows, col0, ncols, kind and D
    or W, S, X as numpy arrays, cluster order) with perm[p] = original index of position p."""
    db = _DescBuilder(n, perm, blocks, eps, _FMT[fmt])
    db.desc.tuning = int(tuning)
    h = C.c_uint64(0)
    nbytes = C.c_size_t(0)
    B.check(B.lib.hlr_upload(C.byref(db.desc), _stream_ptr(stream), C.byref(h), C.byref(nbytes)))
    return DeviceHMatrix(h.value)


def matvec_batched(mats, Xs, Ys, acc="fp32", stream=None, multi=False, sm_share: int = 0):
    """Y_q += A~_q X_q for every request q (X_q, Y_q: n_q x r_q column-major float64 CUDA tensors,
    i.e. tensors of shape (r_q, n_q) in row-major memory, or 1-D of length n_q). multi=True
    (HLR_MULTI) runs every column as a product of its own on its own scratch, so that a column's
    result is bit for bit that of ``matvec`` for it, whatever it is batched with, and the call
    may overlap with ``matvec`` / ``solve_cg`` on the same matrix on another stream."""
    q = len(mats)
    hs = (C.c_uint64 * q)(*[m.handle for m in mats])
    nr = (C.c_int32 * q)()
    xp = (C.c_void_p * q)()
    yp = (C.c_void_p * q)()
    lx = (C.c_int64 * q)()
    ly = (C.c_int64 * q)()
    for i, (m, X, Y) in enumerate(zip(mats, Xs, Ys)):
        r = 1 if X.dim() == 1 else X.shape[0]
        nr[i] = r
        xp[i] = _dev_ptr(X, m.n * r)
        yp[i] = _dev_ptr(Y, m.n * r)
        lx[i] = m.n
        ly[i] = m.n
    flags = _ACC[acc] | (B.HLR_MULTI if multi else 0) | (int(sm_share) << 16)
    B.check(B.lib.hlr_matvec_batched(q, hs, nr, xp, lx, yp, ly, flags, _stream_ptr(stream)))


class HostHMatrix:
    """An FP64 H-matrix built on the host by the library (owns a host object)."""

    def __init__(self, ptr: int, points: np.ndarray):
        self.ptr = ptr
        self._points = points
        self.desc = B.HMatrixDesc()
        B.check(B.lib.hlr_host_describe(C.c_void_p(self.ptr), C.byref(self.desc)))
        self.n = int(self.desc.n)
        self.eps = float(self.desc.eps)

    @property
    def perm(self) -> np.ndarray:
        return np.ctypeslib.as_array(self.desc.perm, shape=(self.n,)).copy()

    def structure(self) -> np.ndarray:
        """(nblocks, 6) int64 array: row0, nrows, col0, ncols, kind, rank."""
        out = np.zeros((self.desc.nblocks, 6), dtype=np.int64)
        for i in range(self.desc.nblocks):
            d = self.desc.blocks[i]
            out[i] = (d.row0, d.nrows, d.col0, d.ncols, d.kind, d.rank)
        return out

    def block(self, i: int) -> dict:
        """Copy of block i as numpy arrays (D, or W, S, X)."""
        d = self.desc.blocks[i]
        b = {"row0": d.row0, "nrows": d.nrows, "col0": d.col0, "ncols": d.ncols, "kind": d.kind}
        if d.kind == HLR_DENSE:
            b["D"] = np.ctypeslib.as_array(d.D, shape=(d.nrows * d.ncols,)).reshape(d.nrows, d.ncols, order="F").copy()
        else:
            k = d.rank
            b["S"] = np.ctypeslib.as_array(d.sigma, shape=(k,)).copy() if k else np.zeros(0)
            b["W"] = np.ctypeslib.as_array(d.W, shape=(d.nrows * k,)).reshape(d.nrows, k, order="F").copy() \
                if k else np.zeros((d.nrows, 0))
            b["X"] = np.ctypeslib.as_array(d.X, shape=(d.ncols * k,)).reshape(d.ncols, k, order="F").copy() \
                if k else np.zeros((d.ncols, 0))
        return b

    def block_views(self):
        """Every block as a dict like ``block(i)`` but with numpy views of the library's own
        arrays (no copies; valid until free())."""
        out = []
        for i in range(self.desc.nblocks):
            d = self.desc.blocks[i]
            b = {"row0": d.row0, "nrows": d.nrows, "col0": d.col0, "ncols": d.ncols, "kind": d.kind}
            if d.kind == HLR_DENSE:
                b["D"] = np.ctypeslib.as_array(d.D, shape=(d.nrows * d.ncols,)).reshape(d.nrows, d.ncols, order="F")
            else:
                k = d.rank
                if k:
                    b["S"] = np.ctypeslib.as_array(d.sigma, shape=(k,))
                    b["W"] = np.ctypeslib.as_array(d.W, shape=(d.nrows * k,)).reshape(d.nrows, k, order="F")
                    b["X"] = np.ctypeslib.as_array(d.X, shape=(d.ncols * k,)).reshape(d.ncols, k, order="F")
                else:
                    b["S"] = np.zeros(0)
            out.append(b)
        return out

    def save(self, path: str):
        """Checkpoint the matrix to `path` (hlr_host_save); read it back with load_host_hmatrix."""
        B.check(B.lib.hlr_host_save(C.c_void_p(self.ptr), os.fsencode(path)))

    def unit_arrays(self, fmt: str = "afl", eps: float | None = None):
        """The matrix's units in upload order as (values, offsets, precisions): see
        ``unit_arrays`` (hlr_unit_list over the library's own blocks)."""
        self.desc.format = _FMT[fmt]
        self.desc.eps = self.eps if eps is None else float(eps)
        return _unit_list(self.desc)

    def unit_offsets(self, fmt: str = "afl", eps: float | None = None):
        """(offsets, precisions) of the matrix's units in upload order (hlr_unit_list without the
        values): unit u holds the values offsets[u] .. offsets[u+1] of the unit order that
        DeviceHMatrix.decode_units writes."""
        self.desc.format = _FMT[fmt]
        self.desc.eps = self.eps if eps is None else float(eps)
        nu = C.c_int64(0)
        nv = C.c_int64(0)
        B.check(B.lib.hlr_unit_list(C.byref(self.desc), None, None, None, 0, 0, C.byref(nu), C.byref(nv)))
        off = np.zeros(nu.value + 1, dtype=np.int64)
        prec = np.zeros(nu.value, dtype=np.float64)
        B.check(B.lib.hlr_unit_list(C.byref(self.desc), off.ctypes.data, prec.ctypes.data, None, nu.value + 1, 0,
                                    C.byref(nu), C.byref(nv)))
        return off, prec

    def upload(self, fmt="afl", eps: float | None = None, stream=None, tuning: int = 0,
               decode_map: bool = False, encode_device: bool = False) -> DeviceHMatrix:
        """Compress (fmt="afl") or copy (fmt="fp64") and upload to the current GPU. tuning:
        work layout of the AFL kernels (``tuning_code``; 0 = default); decode_map: keep the map
        of decode_units whatever the size (HLR_DECODE_MAP); encode_device: compress on the GPU
        during the upload (HLR_ENCODE_DEVICE; the same bytes as the host encoder)."""
        self.desc.format = _FMT[fmt]
        self.desc.eps = self.eps if eps is None else float(eps)
        self.desc.tuning = (int(tuning) | (B.HLR_DECODE_MAP if decode_map else 0)
                            | (B.HLR_ENCODE_DEVICE if encode_device else 0))
        h = C.c_uint64(0)
        nbytes = C.c_size_t(0)
        B.check(B.lib.hlr_upload(C.byref(self.desc), _stream_ptr(stream), C.byref(h), C.byref(nbytes)))
        return DeviceHMatrix(h.value)

    def free(self):
        if self.ptr:
            B.lib.hlr_host_free(C.c_void_p(self.ptr))
            self.ptr = 0

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def build_kernel_hmatrix(points: np.ndarray, kernel: str, eps: float, scale: float = 1.0, diag: float = 0.0,
                         eta: float = 2.0, leaf_size: int = 64, threads: int = 0) -> HostHMatrix:
    """Build the FP64 H-matrix of a kernel matrix on the host (cluster tree, block tree, ACA +
    SVD recompression), multithreaded in native code."""
    P = np.ascontiguousarray(points, dtype=np.float64)
    prob = B.KernelProblem()
    prob.kernel = _KERNEL[kernel]
    prob.dim = P.shape[1]
    prob.n = P.shape[0]
    prob.points = B.f64ptr(P)
    prob.scale = float(scale)
    prob.diag = float(diag)
    prob.eps = float(eps)
    prob.eta = float(eta)
    prob.leaf_size = int(leaf_size)
    prob.threads = int(threads)
    out = C.c_void_p(0)
    B.check(B.lib.hlr_build(C.byref(prob), C.byref(out)))
    return HostHMatrix(out.value, P)


def load_host_hmatrix(path: str) -> HostHMatrix:
    """A matrix saved by HostHMatrix.save (hlr_host_load: checked against its version and hash)."""
    out = C.c_void_p(0)
    B.check(B.lib.hlr_host_load(os.fsencode(path), C.byref(out)))
    return HostHMatrix(out.value, None)


def encode(a: np.ndarray, u: float, fmt: str = "afl"):
    """Host encoder of the library for any compressed format (afl, aflp, bfl, dfl, mp): returns
    (m_min, e, m, stream bytes padded to 16)."""
    a = np.ascontiguousarray(a, dtype=np.float64).ravel()
    m_min = C.c_double(0)
    e = C.c_int32(0)
    m = C.c_int32(0)
    nbytes = C.c_size_t(0)
    cap = (a.size * 64 + 7) // 8 + 32
    buf = np.zeros(cap, dtype=np.uint8)
    f = _FMT[fmt] if fmt in _FMT else int(fmt)
    B.check(B.lib.hlr_encode(f, B.f64ptr(a), a.size, float(u), C.byref(m_min), C.byref(e), C.byref(m),
                             buf.ctypes.data, cap, C.byref(nbytes)))
    return m_min.value, e.value, m.value, buf[: nbytes.value].tobytes()


def encode_device(values, offsets, precisions, fmt: str = "afl", stream=None):
    """GPU encoder of the library (hlr_encode_device): units values[offsets[u]:offsets[u+1]]
    (FP64 / int64 CUDA tensors) at precisions[u], encoded on the device in one asynchronous
    call. Returns (m_min, e, m, out_off, out) as CUDA tensors; unit u's stream, byte for byte
    what encode() writes, is out[out_off[u]:out_off[u+1]]; e[u] = -1 marks a rejected unit."""
    import torch
    nunits = precisions.numel()
    total = values.numel()
    dev = values.device
    m_min = torch.empty(nunits, dtype=torch.float64, device=dev)
    e = torch.empty(nunits, dtype=torch.int32, device=dev)
    m = torch.empty(nunits, dtype=torch.int32, device=dev)
    out_off = torch.empty(nunits + 1, dtype=torch.int64, device=dev)
    cap = 8 * total + 16 * nunits + 16
    out = torch.empty(cap, dtype=torch.uint8, device=dev)
    f = _FMT[fmt] if fmt in _FMT else int(fmt)
    if offsets.numel() != nunits + 1:
        raise HlrError(HLR_ERR_INVALID, "offsets must hold nunits + 1 entries")
    B.check(B.lib.hlr_encode_device(f, nunits, _dev_ptr(offsets, dtype=torch.int64), total, _dev_ptr(values),
                                    _dev_ptr(precisions), _dev_ptr(m_min), _dev_ptr(e, dtype=torch.int32),
                                    _dev_ptr(m, dtype=torch.int32), _dev_ptr(out_off, dtype=torch.int64),
                                    _dev_ptr(out, dtype=torch.uint8), cap, _stream_ptr(stream)))
    return m_min, e, m, out_off, out


def _unit_list(desc):
    nu = C.c_int64(0)
    nv = C.c_int64(0)
    B.check(B.lib.hlr_unit_list(C.byref(desc), None, None, None, 0, 0, C.byref(nu), C.byref(nv)))
    off = np.zeros(nu.value + 1, dtype=np.int64)
    prec = np.zeros(nu.value, dtype=np.float64)
    vals = np.zeros(nv.value, dtype=np.float64)
    B.check(B.lib.hlr_unit_list(C.byref(desc), off.ctypes.data, prec.ctypes.data, vals.ctypes.data, nu.value + 1,
                                nv.value, C.byref(nu), C.byref(nv)))
    return vals, off, prec


def unit_arrays(blocks, eps: float, fmt: str = "afl"):
    """The units of a block list (dicts as for ``upload``) in upload order as (values, offsets,
    precisions) numpy arrays: dense leaf -> its column-major values, lowrank block -> W
    columns, then X columns; each unit's precision is the one upload gives it (hlr_unit_list:
    dense eps, lowrank column i eps sigma_0 / sigma_i, MP dense leaves FP64)."""
    blocks = list(blocks)
    n = 0
    for b in blocks:
        n = max(n, int(b["row0"]) + int(b["nrows"]), int(b["col0"]) + int(b["ncols"]))
    db = _DescBuilder(n, None, blocks, eps, _FMT[fmt])
    return _unit_list(db.desc)


def afl_encode(a: np.ndarray, u: float):
    """Host AFL encoder of the library: returns (m_min, e, m, stream bytes padded to 16)."""
    a = np.ascontiguousarray(a, dtype=np.float64).ravel()
    m_min = C.c_double(0)
    e = C.c_int32(0)
    m = C.c_int32(0)
    nbytes = C.c_size_t(0)
    cap = (a.size * 64 + 7) // 8 + 32
    buf = np.zeros(cap, dtype=np.uint8)
    B.check(B.lib.hlr_afl_encode(B.f64ptr(a), a.size, float(u), C.byref(m_min), C.byref(e), C.byref(m),
                                 buf.ctypes.data_as(C.c_void_p), cap, C.byref(nbytes)))
    return m_min.value, e.value, m.value, buf[: nbytes.value].tobytes()


def afl_decode_device(stream_dev, n: int, m_min: float, e: int, m: int, out, stream=None):
    """Decode one AFL stream (uint8 CUDA tensor, 16-byte aligned) into out (float64 CUDA tensor)."""
    B.check(B.lib.hlr_afl_decode_device(stream_dev.data_ptr(), int(n), float(m_min), int(e), int(m),
                                        _dev_ptr(out, n), _stream_ptr(stream)))
    return out
