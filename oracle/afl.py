"""AFL binary compression of one data unit and the APLR precision rule (oracle; test
infrastructure only).

Section 3.2 defines AFL: a data block is stored in a 1-e_r-m_eps format whose exponent width
e_r follows from the block's dynamic range and whose mantissa width m_eps follows from the
requested accuracy; before conversion every value is scaled by 1/m_min and shifted by +1 (the
remark in Section 3.2), so all stored values are >= 2 and only the low exponent bits need to
be kept. The bits are not byte aligned.

Section 3.3 (APLR) stores column i of the orthogonal lowrank factors W and X with its own
precision u~_i chosen such that sigma_i ~ delta / u~_i, delta = eps * ||M||.

Readings taken where the text is silent or garbled (each is listed with its reason in the
design notes of the repository):

* magnitudes: m_min is the smallest NONZERO |a_j|; zeros map to v = 1 and decode to 0.
* mantissa width for precision u: m = ceil(-log2 u), clamped to [0, 52], evaluated exactly
  from the binary exponent of u (u = f 2^E, f in [1/2, 1) gives ceil(-log2 u) = 1 - E).
* rounding to m mantissa bits: round half up on the FP64 bit pattern of v (add 2^(51-m),
  clear the low 52-m bits); a carry runs into the exponent.
* exponent field: field = (biased exponent of the rounded v) - 1023 >= 0, and e is the
  smallest width that holds the largest field: e = ceil(log2(E_max + 1)) (0 if E_max = 0).
  This replaces the garbled e_r = ceil(log2 log2 r) and is taken after rounding.
* code of value j: sign * 2^(e+m) | field * 2^m | top m mantissa bits; width w = 1 + e + m.
* packing: value j occupies stream bits [j w, (j+1) w), bits numbered LSB-first inside
  little-endian 64-bit words (equivalently LSB-first inside consecutive bytes); the stream
  is zero-padded to a multiple of 16 bytes.
* decoding: v = bits((field + 1023) << 52 | mant << (52 - m)), a = (v - 1) * m_min in IEEE
  FP64 round-to-nearest (no fused multiply-add), negated when the sign bit is set.
* APLR: delta = eps * sigma_0 (spectral norm), u~_i = (eps * sigma_0) / sigma_i.

Byte-aligned variants (Section 3.2, after AFL):

* AFLP: AFL with the mantissa width raised to the smallest m' >= m for which 1 + e + m' is a
  multiple of 8 (e taken after rounding at m', as for AFL); decoded exactly like AFL.
* BFL: 8 exponent bits, i.e. the FP32 layout: the value is cast to FP32 (round to nearest
  even), its bit pattern rounded half up to m' mantissa bits, m' the smallest of 7, 15, 23 with
  m' >= m (23 when m > 23), and the top 1 + 8 + m' bits stored; decoded by shifting the code
  back into an FP32 pattern.
* DFL: 11 exponent bits, the FP64 layout: the FP64 pattern rounded half up to m' mantissa
  bits, m' the smallest of 4, 12, ..., 52 with m' >= m, top 1 + 11 + m' bits stored.
  BFL and DFL store no m_min (it is 1) and e is the fixed exponent width.

Mixed precision comparison format MP-D-S-H (Section 3.3, after [AmeBoiBut:2022]): every column i
of a lowrank factor is stored in the cheapest of FP16, FP32, FP64 whose unit roundoff
(Table 1: 2^-11, 2^-24, 2^-53) is <= its APLR precision u~_i = delta / sigma_i; values are cast
to that format with round to nearest even; dense leaves stay FP64 (the comparison compresses
only lowrank factors). A unit is tagged mp16 / mp32 / mp64 and e is the format's exponent width.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

MANT_BITS = 52
MANT_MASK = (1 << 52) - 1
STREAM_ALIGN = 16


def mantissa_bits(u: float) -> int:
    """m = ceil(-log2 u) clamped to [0, 52], exact via u = f 2^E (f in [0.5,1)) -> 1 - E."""
    if not (u > 0.0) or not math.isfinite(u):
        raise ValueError(f"precision must be positive and finite, got {u!r}")
    _, E = math.frexp(u)
    return min(max(1 - E, 0), MANT_BITS)


def aplr_precisions(sigma: np.ndarray, eps: float) -> np.ndarray:
    """Per-column precisions u~_i = delta / sigma_i with delta = eps * sigma_0 (Section 3.3)."""
    sigma = np.asarray(sigma, dtype=np.float64)
    if sigma.size == 0:
        return sigma.copy()
    delta = eps * float(sigma[0])
    return np.array([delta / float(s) for s in sigma], dtype=np.float64)


FORMATS = ("afl", "aflp", "bfl", "dfl", "mp")
MP_ROUNDOFF = {"mp16": 2.0 ** -11, "mp32": 2.0 ** -24, "mp64": 2.0 ** -53}


@dataclass(frozen=True)
class AFLUnit:
    """One compressed data unit: ``n`` values of width w = 1 + e + m in ``data``, in format
    ``fmt`` (AFL, or its byte-aligned variants AFLP, BFL, DFL)."""
    n: int
    m_min: float
    e: int
    m: int
    data: bytes
    fmt: str = "afl"

    @property
    def w(self) -> int:
        return 1 + self.e + self.m

    @property
    def stream_bits(self) -> int:
        return self.n * self.w


def _round_to_mantissa(v: np.ndarray, m: int) -> np.ndarray:
    """Round FP64 values v >= 1 to m mantissa bits, half up on the bit pattern."""
    b = v.view(np.uint64).copy()
    if m < MANT_BITS:
        b += np.uint64(1 << (MANT_BITS - 1 - m))
        b &= ~np.uint64((1 << (MANT_BITS - m)) - 1)
    return b


def codes_of(a: np.ndarray, u: float) -> tuple[np.ndarray, float, int, int]:
    """Integer codes of the values a (storage order) at precision u: (codes, m_min, e, m)."""
    return codes_at(a, mantissa_bits(u))


def codes_at(a: np.ndarray, m: int) -> tuple[np.ndarray, float, int, int]:
    """AFL codes of the values a with m mantissa bits: (codes, m_min, e, m)."""
    a = np.ascontiguousarray(a, dtype=np.float64).ravel()
    if not np.all(np.isfinite(a)):
        raise ValueError("AFL input must be finite")
    mag = np.abs(a)
    nonzero = mag != 0.0
    if not np.any(nonzero):
        return np.zeros(a.size, dtype=np.uint64), 0.0, 0, m
    m_min = float(mag[nonzero].min())
    v = mag / m_min + 1.0                        # scaled by 1/m_min, shifted by +1
    b = _round_to_mantissa(v, m)
    field = (b >> np.uint64(52)).astype(np.int64) - 1023
    assert field.min() >= 0
    mant = (b & np.uint64(MANT_MASK)) >> np.uint64(MANT_BITS - m)
    e = int(field.max()).bit_length()            # = ceil(log2(E_max + 1))
    sign = (a < 0.0).astype(np.uint64)
    code = (sign << np.uint64(e + m)) | (field.astype(np.uint64) << np.uint64(m)) | mant
    return code, m_min, e, m


def pack(codes: np.ndarray, w: int) -> bytes:
    """Pack w-bit codes LSB-first, value j at bits [j w, (j+1) w); pad to 16 bytes."""
    n = codes.size
    if n == 0 or w == 0:
        return b""
    shifts = np.arange(w, dtype=np.uint64)
    bitmat = ((codes[:, None] >> shifts[None, :]) & np.uint64(1)).astype(np.uint8)
    raw = np.packbits(bitmat.ravel(), bitorder="little").tobytes()
    pad = (-len(raw)) % STREAM_ALIGN
    return raw + b"\0" * pad


def unpack(data: bytes, n: int, w: int) -> np.ndarray:
    """Inverse of :func:`pack`: the n w-bit codes as uint64."""
    if n == 0:
        return np.zeros(0, dtype=np.uint64)
    bits = np.unpackbits(np.frombuffer(data, dtype=np.uint8), bitorder="little")[: n * w]
    bitmat = bits.reshape(n, w).astype(np.uint64)
    return (bitmat << np.arange(w, dtype=np.uint64)[None, :]).sum(axis=1, dtype=np.uint64)


def encode(a: np.ndarray, u: float, fmt: str = "afl") -> AFLUnit:
    """Encode the values a (in storage order) at precision u in format fmt."""
    if fmt == "aflp":
        return encode_aflp(a, u)
    if fmt == "bfl":
        return encode_bfl(a, u)
    if fmt == "dfl":
        return encode_dfl(a, u)
    if fmt == "mp":
        return encode_mp(a, u)
    if fmt != "afl":
        raise ValueError(f"unknown format {fmt!r}")
    code, m_min, e, m = codes_of(a, u)
    return AFLUnit(n=code.size, m_min=m_min, e=e, m=m, data=pack(code, 1 + e + m))


def encode_aflp(a: np.ndarray, u: float) -> AFLUnit:
    """AFLP: AFL with the smallest m' >= m(u) that makes 1 + e + m' a multiple of 8."""
    m = mantissa_bits(u)
    while True:
        code, m_min, e, mm = codes_at(a, m)
        if (1 + e + m) % 8 == 0 or m == MANT_BITS:
            break
        m += 1
    return AFLUnit(n=code.size, m_min=m_min, e=e, m=m, data=pack(code, 1 + e + m), fmt="aflp")


def bfl_mantissa(u: float) -> int:
    """BFL mantissa width: the smallest of 7, 15, 23 that is >= m(u) (23 if none is)."""
    m = mantissa_bits(u)
    return next((mp for mp in (7, 15, 23) if mp >= m), 23)


def dfl_mantissa(u: float) -> int:
    """DFL mantissa width: the smallest of 4, 12, ..., 52 that is >= m(u)."""
    m = mantissa_bits(u)
    return next(mp for mp in range(4, 53, 8) if mp >= m)


def encode_bfl(a: np.ndarray, u: float) -> AFLUnit:
    """BFL: FP32 cast, mantissa rounded half up to m' bits, top 9 + m' bits of the pattern."""
    a = np.ascontiguousarray(a, dtype=np.float64).ravel()
    mp = bfl_mantissa(u)
    x = a.astype(np.float32)
    if not np.all(np.isfinite(x)):
        raise ValueError("BFL input must be finite in FP32")
    b = x.view(np.uint32).astype(np.uint64)
    if mp < 23:
        b = (b + np.uint64(1 << (22 - mp))) & ~np.uint64((1 << (23 - mp)) - 1)
    if np.any(((b >> np.uint64(23)) & np.uint64(0xFF)) == np.uint64(0xFF)):
        raise ValueError("BFL rounding overflows FP32")
    code = b >> np.uint64(23 - mp)
    return AFLUnit(n=code.size, m_min=1.0, e=8, m=mp, data=pack(code, 9 + mp), fmt="bfl")


def encode_dfl(a: np.ndarray, u: float) -> AFLUnit:
    """DFL: the FP64 pattern rounded half up to m' mantissa bits, top 12 + m' bits."""
    a = np.ascontiguousarray(a, dtype=np.float64).ravel()
    if not np.all(np.isfinite(a)):
        raise ValueError("DFL input must be finite")
    mp = dfl_mantissa(u)
    b = a.view(np.uint64).copy()
    if mp < MANT_BITS:
        b = (b + np.uint64(1 << (MANT_BITS - 1 - mp))) & ~np.uint64((1 << (MANT_BITS - mp)) - 1)
    if np.any(((b >> np.uint64(52)) & np.uint64(0x7FF)) == np.uint64(0x7FF)):
        raise ValueError("DFL rounding overflows FP64")
    code = b >> np.uint64(MANT_BITS - mp)
    return AFLUnit(n=code.size, m_min=1.0, e=11, m=mp, data=pack(code, 12 + mp), fmt="dfl")


def mp_format(u: float) -> str:
    """The cheapest IEEE format (mp16, mp32, mp64) whose unit roundoff is <= u."""
    for f in ("mp16", "mp32", "mp64"):
        if MP_ROUNDOFF[f] <= u:
            return f
    return "mp64"


def encode_mp(a: np.ndarray, u: float, fmt: str | None = None) -> AFLUnit:
    """MP-D-S-H unit: the values cast (round to nearest even) to the format chosen for u
    (or to fmt), stored as their IEEE bit patterns."""
    a = np.ascontiguousarray(a, dtype=np.float64).ravel()
    f = fmt or mp_format(u)
    dt, ut, e, m = {"mp16": (np.float16, np.uint16, 5, 10), "mp32": (np.float32, np.uint32, 8, 23),
                    "mp64": (np.float64, np.uint64, 11, 52)}[f]
    x = a.astype(dt)
    if not np.all(np.isfinite(x)):
        raise ValueError(f"value not finite in {f}")
    code = x.view(ut).astype(np.uint64)
    return AFLUnit(n=code.size, m_min=1.0, e=e, m=m, data=pack(code, 1 + e + m), fmt=f)


def decode(unit: AFLUnit) -> np.ndarray:
    """Decode a unit to FP64. AFL/AFLP: a = (v - 1) * m_min, negated for a set sign bit;
    BFL: the code shifted back into an FP32 pattern; DFL: into an FP64 pattern."""
    code = unpack(unit.data, unit.n, unit.w)
    if unit.fmt == "mp16":
        return code.astype(np.uint16).view(np.float16).astype(np.float64)
    if unit.fmt == "mp32":
        return code.astype(np.uint32).view(np.float32).astype(np.float64)
    if unit.fmt == "mp64":
        return code.view(np.float64).copy()
    if unit.fmt == "bfl":
        return (code << np.uint64(23 - unit.m)).astype(np.uint32).view(np.float32).astype(np.float64)
    if unit.fmt == "dfl":
        return (code << np.uint64(MANT_BITS - unit.m)).view(np.float64).copy()
    e, m = unit.e, unit.m
    mant = code & np.uint64((1 << m) - 1)
    field = (code >> np.uint64(m)) & np.uint64((1 << e) - 1)
    sign = (code >> np.uint64(e + m)) & np.uint64(1)
    vbits = ((field + np.uint64(1023)) << np.uint64(52)) | (mant << np.uint64(MANT_BITS - m))
    v = vbits.view(np.float64)
    a = (v - 1.0) * unit.m_min
    return np.where(sign == 1, -a, a)


def stream_bytes(unit: AFLUnit) -> int:
    """Unpadded stream size ceil(n w / 8) in bytes."""
    return (unit.stream_bits + 7) // 8
