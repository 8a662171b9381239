"""Pins of the oracle AFL codec and APLR rule (Sections 3.2 and 3.3).

* a hand-worked code (tests/golden/afl_hand_example.txt);
* the per-entry error bound |a~ - a| <= (2^-(m+1) + 2^-51) (|a| + m_min) for every m;
* exact special cases (0, +-m_min), exponent carries, minimal exponent width, idempotence;
* mantissa width m = ceil(-log2 u) checked against the real logarithm;
* APLR precisions u~_i = eps sigma_0 / sigma_i.
"""
import math
import os

import numpy as np
import pytest

from oracle import afl

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _hand():
    d = {}
    with open(os.path.join(GOLD, "afl_hand_example.txt")) as f:
        for ln in f:
            if ln.strip() and not ln.startswith("#"):
                k, *v = ln.split()
                d[k] = v
    return d


def test_hand_worked_example():
    d = _hand()
    a = np.array([float(v) for v in d["values"]])
    unit = afl.encode(a, float(d["u"][0]))
    assert unit.m_min == float(d["m_min"][0])
    assert unit.e == int(d["e"][0]) and unit.m == int(d["m"][0])
    codes, *_ = afl.codes_of(a, float(d["u"][0]))
    assert [int(c) for c in codes] == [int(v) for v in d["codes"]]
    assert unit.data.hex() == d["hex"][0]
    np.testing.assert_array_equal(afl.decode(unit), a)


def _cases():
    g = np.random.default_rng(11)
    yield g.standard_normal(777)
    yield g.standard_normal(64) * 1e-3
    yield np.exp(g.uniform(-40, 40, size=500)) * g.choice([-1.0, 1.0], size=500)
    z = g.standard_normal(300)
    z[::7] = 0.0
    yield z
    yield np.array([3.5, -3.5, 3.5])
    # values whose scaled mantissa is all ones: rounding carries into the exponent
    yield np.array([1.0, 2.0 - 2.0 ** -40, -(4.0 - 2.0 ** -30), 7.999999])


@pytest.mark.parametrize("m", list(range(0, 53)))
def test_per_entry_bound_every_mantissa_width(m):
    u = 1.0 if m == 0 else 2.0 ** -m
    assert afl.mantissa_bits(u) == m
    for a in _cases():
        unit = afl.encode(a, u)
        d = afl.decode(unit)
        bound = (2.0 ** (-m - 1) + 2.0 ** -51) * (np.abs(a) + unit.m_min)
        assert np.all(np.abs(d - a) <= bound), (m, np.max(np.abs(d - a) / bound))
        assert np.all(d[a == 0.0] == 0.0)
        assert np.all(np.sign(d[a != 0.0]) == np.sign(a[a != 0.0]))
        assert len(unit.data) % 16 == 0
        assert len(unit.data) >= (a.size * unit.w + 7) // 8
        assert len(unit.data) - (a.size * unit.w + 7) // 8 < 16


def test_exact_special_values():
    a = np.array([0.25, -0.25, 0.0, 1.75, -9.0])
    for m in (0, 3, 20, 52):
        d = afl.decode(afl.encode(a, 1.0 if m == 0 else 2.0 ** -m))
        assert d[0] == 0.25 and d[1] == -0.25 and d[2] == 0.0


def test_all_zero_unit():
    unit = afl.encode(np.zeros(10), 1e-6)
    assert unit.e == 0 and unit.m_min == 0.0
    np.testing.assert_array_equal(afl.decode(unit), np.zeros(10))


def test_exponent_width_is_minimal_and_covers_carry():
    g = np.random.default_rng(5)
    for _ in range(200):
        a = np.exp(g.uniform(-30, 30, size=50))
        m = int(g.integers(0, 53))
        codes, m_min, e, mm = afl.codes_of(a, 1.0 if m == 0 else 2.0 ** -m)
        field = (codes >> np.uint64(mm)) & np.uint64((1 << e) - 1)
        emax = int(field.max())
        assert emax < 2 ** e                    # fits
        assert e == 0 or emax >= 2 ** (e - 1)   # and no narrower width would
    # v = 2 - 2^-40 rounds up to 2.0 at m = 10: the field grows from 0 to 1
    codes, m_min, e, m = afl.codes_of(np.array([1.0, 1.0 - 2.0 ** -40]), 2.0 ** -10)
    assert m_min == 1.0 - 2.0 ** -40 and e == 1


@pytest.mark.parametrize("m", [1, 4, 13, 20, 27, 40, 48])
def test_idempotent_reencoding(m):
    g = np.random.default_rng(m)
    a = g.standard_normal(513)
    unit = afl.encode(a, 2.0 ** -m)
    again = afl.encode(afl.decode(unit), 2.0 ** -m)
    assert again.data == unit.data and again.m_min == unit.m_min


def test_mantissa_bits_matches_real_log():
    g = np.random.default_rng(3)
    for u in np.exp(g.uniform(math.log(1e-15), math.log(0.9), size=2000)):
        x = -math.log2(u)
        if abs(x - round(x)) > 1e-9:
            assert afl.mantissa_bits(u) == math.ceil(x)
    assert afl.mantissa_bits(1e-6) == 20
    assert afl.mantissa_bits(2.0 ** -20) == 20
    assert afl.mantissa_bits(1e-30) == 52
    assert afl.mantissa_bits(3.0) == 0


def test_aplr_precisions():
    s = np.array([10.0, 1.0, 0.1, 2e-5])
    u = afl.aplr_precisions(s, 1e-6)
    np.testing.assert_allclose(u, [1e-6, 1e-5, 1e-4, 0.5], rtol=1e-15)
    # the first column gets the block accuracy eps, later columns fewer bits
    ms = [afl.mantissa_bits(v) for v in u]
    assert ms == sorted(ms, reverse=True) and ms[0] == 20


def test_pack_unpack_roundtrip_widths():
    g = np.random.default_rng(9)
    for w in range(1, 64):
        codes = g.integers(0, 2 ** min(w, 62), size=101, dtype=np.uint64) & np.uint64((1 << w) - 1)
        data = afl.pack(codes, w)
        np.testing.assert_array_equal(afl.unpack(data, 101, w), codes)
        # bit j*w+b of the stream is bit b of code j (LSB-first bytes)
        bits = np.unpackbits(np.frombuffer(data, np.uint8), bitorder="little")
        j = 57
        for b in range(w):
            assert bits[j * w + b] == (int(codes[j]) >> b) & 1
