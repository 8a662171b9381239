"""Arithmetic identities the GPU kernels rely on, checked on the CPU with IEEE FP32 / FP64 numpy
arithmetic (the same round-to-nearest operations the kernels issue).

* Mid-width decode (product kernels): for an AFL code of w <= 32 bits with e <= 4 (or m <= 23),
  v's top 23 mantissa bits give an FP32 v_hi with v_hi - 1 exact, and adding the remaining
  m - 23 bits, lo * 2^(field - m), rounds once: the result is RN32(v - 1), the value the FP64
  route float(v - 1) gives (Section 3.2 decoding, reading s19).
* Reciprocal quotient (GPU encoder): with r = RN(1 / m_min), the pattern of RN(RN(|a| r) + 1)
  rounds half up to m bits like v = RN(RN(|a| / m_min) + 1) whenever it lies more than 32 units
  away from the half-way point of the m-bit grid and m <= 45 (Section 3.2 encoding).
"""
import numpy as np
import pytest


def _f32(bits):
    return np.array([bits & 0xFFFFFFFF], dtype=np.uint32).view(np.float32)[0]


def _v_minus_1_fp64(code, e, m):
    em = e + m
    b = ((code & ((1 << em) - 1)) << (52 - m)) + (1023 << 52)
    v = np.array([b], dtype=np.uint64).view(np.float64)[0] - 1.0
    return -v if (code >> em) & 1 else v


def _mid32(code, e, m):
    mant = code & ((0xFFFFFFFF >> (32 - m)) if m else 0)
    field = (code >> m) & ((1 << e) - 1)
    k = m - 23 if m > 23 else 0
    hi = (mant >> k) if m > 23 else (mant << (23 - m))
    lo = np.float32(mant & ((1 << k) - 1)) * _f32((field + 127 - m) << 23)
    r = (_f32(((field + 127) << 23) | hi) - np.float32(1.0)) + lo
    return -r if (code >> (e + m)) & 1 else r


@pytest.mark.parametrize("e", [0, 1, 2, 3, 4, 5, 7])
def test_mid_width_decode_equals_fp64_route(e):
    g = np.random.default_rng(100 + e)
    for m in range(0, 32 - e):
        if e > 4 and m > 23:
            continue  # outside the mid-width condition
        w = 1 + e + m
        codes = list(g.integers(0, 1 << w, 200)) + [0, (1 << w) - 1, 1 << (e + m), (1 << (e + m)) - 1]
        for code in codes:
            code = int(code)
            a = np.float32(_v_minus_1_fp64(code, e, m))
            b = np.float32(_mid32(code, e, m))
            assert a.view(np.uint32) == b.view(np.uint32), (e, m, hex(code))


def _round_pattern(b, m):
    if m < 52:
        b = (b + (1 << (51 - m))) & ~((1 << (52 - m)) - 1)
    return b


def _bits(x):
    return int(np.array([x], dtype=np.float64).view(np.uint64)[0])


def test_reciprocal_quotient_rounds_like_the_division():
    g = np.random.default_rng(7)
    checked = fallback = 0
    for m in list(range(0, 46)):
        half = 1 << (51 - m) if m < 52 else 0
        mask = (1 << (52 - m)) - 1
        for m_min in (3.0, 0.7, 1.0 / 3.0, 5e-200, 7e150, float(g.uniform(0.5, 2.0))):
            r = 1.0 / m_min
            # magnitudes whose exact v sits at or near a half-way point, and random ones
            k = g.integers(0, 2 ** min(m, 40), 60).astype(np.float64)
            v = (1.0 + (2.0 * k + 1.0) * 2.0 ** -(m + 1)) * 2.0 ** g.integers(1, 12, k.size)
            v = v * (1.0 + g.integers(-6, 7, k.size) * 2.0 ** -52)
            av = np.concatenate([m_min * (v - 1.0), m_min * np.exp(g.uniform(0, 20, 60))])
            av = av[np.isfinite(av) & (av >= m_min)]
            for a in av:
                exact = _round_pattern(_bits(a / m_min + 1.0), m)
                b = _bits(a * r + 1.0)
                low = b & mask
                dist = abs(low - half)
                checked += 1
                if dist > 32 and m <= 45:
                    assert _round_pattern(b, m) == exact, (m, m_min, a)
                else:
                    fallback += 1
    assert checked > 10000 and fallback > 0
