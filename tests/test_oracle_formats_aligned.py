"""Byte-aligned variants of AFL (Section 3.2): AFLP, BFL (FP32 layout) and DFL (FP64 layout),
pinned against what they must equal: the FP32 cast (BFL with 23 mantissa bits), bfloat16
round-to-nearest (BFL with 7 bits, away from ties), the identity (DFL with 52 bits), the
relative bound 2^-(m'+1) of rounding to m' bits, AFL's bound for AFLP, byte-aligned widths and
minimal mantissa widths, and encode(decode) idempotence."""
import numpy as np
import pytest

from oracle import afl
from oracle import hmatrix as ohm


def _vals(seed, n=2000):
    g = np.random.default_rng(seed)
    return g.standard_normal(n) * np.exp(g.uniform(-20, 20, n))


@pytest.mark.parametrize("u", [1e-2, 2.0 ** -9, 1e-4, 1e-6, 2.0 ** -23, 1e-9, 1e-14])
def test_widths_are_byte_aligned_and_minimal(u):
    a = _vals(1)
    m = afl.mantissa_bits(u)
    p = afl.encode(a, u, "aflp")
    assert p.w % 8 == 0 and p.m >= m
    for mm in range(m, p.m):          # no smaller width works
        _, _, e, _ = afl.codes_at(a, mm)
        assert (1 + e + mm) % 8 != 0
    b = afl.encode(a, u, "bfl")
    assert b.w in (16, 24, 32) and b.e == 8 and b.m == min([mp for mp in (7, 15, 23) if mp >= m] or [23])
    d = afl.encode(a, u, "dfl")
    assert d.w % 8 == 0 and d.e == 11 and d.m >= m and d.m - m < 8
    for unit in (p, b, d):
        assert len(unit.data) >= afl.stream_bytes(unit) == unit.n * unit.w // 8


def test_bfl23_is_the_fp32_cast_and_bfl7_is_bfloat16():
    a = _vals(2)
    assert np.array_equal(afl.decode(afl.encode(a, 2.0 ** -23, "bfl")), a.astype(np.float32).astype(np.float64))
    torch = pytest.importorskip("torch")
    x32 = a.astype(np.float32)
    low = x32.view(np.uint32) & np.uint32(0xFFFF)
    keep = low != 0x8000                   # away from ties, half up = round to nearest even
    ref = torch.from_numpy(x32[keep]).to(torch.bfloat16).to(torch.float64).numpy()
    got = afl.decode(afl.encode(a[keep], 2.0 ** -7, "bfl"))
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("u", [1e-3, 1e-6, 1e-10])
def test_relative_rounding_bounds(u):
    a = _vals(3)
    d = afl.decode(afl.encode(a, u, "dfl"))
    mp = afl.dfl_mantissa(u)
    assert np.all(np.abs(d - a) <= 2.0 ** -(mp + 1) * np.abs(a) * (1 + 2.0 ** -50))
    b = afl.decode(afl.encode(a.astype(np.float32).astype(np.float64), u, "bfl"))
    mp = afl.bfl_mantissa(u)
    x = a.astype(np.float32).astype(np.float64)
    assert np.all(np.abs(b - x) <= 2.0 ** -(mp + 1) * np.abs(x) * (1 + 2.0 ** -20))
    p = afl.encode(a, u, "aflp")
    r = afl.decode(p)
    bound = (2.0 ** (-p.m - 1) + 2.0 ** -51) * (np.abs(a) + p.m_min)
    assert np.all(np.abs(r - a) <= bound)


def test_dfl52_identity_and_special_values():
    a = np.array([0.0, -0.0, 1.0, -2.5, 1e-300, -1e300, 5e-324])
    assert np.array_equal(afl.decode(afl.encode(a, 2.0 ** -60, "dfl")).view(np.int64), a.view(np.int64))
    z = afl.decode(afl.encode(np.zeros(5), 1e-6, "bfl"))
    assert np.array_equal(z, np.zeros(5))


@pytest.mark.parametrize("fmt", ["aflp", "bfl", "dfl"])
def test_encode_decode_idempotent(fmt):
    a = _vals(4, 500)
    unit = afl.encode(a, 1e-6, fmt)
    again = afl.encode(afl.decode(unit), 1e-6, fmt)
    assert again.data == unit.data and (again.e, again.m) == (unit.e, unit.m)


@pytest.mark.parametrize("fmt", ["aflp", "bfl", "dfl"])
def test_compressed_matrix_error(fmt, exp2d_case):
    p, H, C = exp2d_case
    Cf = ohm.compress(H, fmt=fmt)
    A = ohm.to_dense(H, decoded=False)
    Af = ohm.to_dense(Cf)
    # byte-aligned formats keep at least the AFL precision of every unit
    assert np.linalg.norm(Af - A, 2) <= 2 * np.linalg.norm(ohm.to_dense(C) - A, 2) + 1e-12 * np.linalg.norm(A, 2)
    assert all(u.fmt == fmt for b in Cf.blocks for u in b.units)


def test_mp_units_are_ieee_casts_and_formats_follow_precision():
    """MP-D-S-H (Section 3.3): each column in the cheapest of FP16/FP32/FP64 whose unit roundoff
    (Table 1) is <= its precision; the stored values are the round-to-nearest casts."""
    a = _vals(8) * 1e-3
    for u, f, dt in ((1e-3, "mp16", np.float16), (2.0 ** -11, "mp16", np.float16), (1e-4, "mp32", np.float32),
                     (2.0 ** -24, "mp32", np.float32), (1e-8, "mp64", np.float64)):
        x = np.clip(a, -6e4, 6e4)
        unit = afl.encode(x, u, "mp")
        assert unit.fmt == f and unit.w == {"mp16": 16, "mp32": 32, "mp64": 64}[f]
        assert np.array_equal(afl.decode(unit), x.astype(dt).astype(np.float64))


def test_mp_block_error_bound(exp2d_case):
    """The bound of [AmeBoiBut:2022, Thm 2.1] as quoted in Section 3.3 with p = 3 formats:
    ||M - W Sigma X^T|| <= (2p - 1 + sum_i sqrt(r_i) u_i) delta per lowrank block; dense leaves exact."""
    p, H, C = exp2d_case
    Cm = ohm.compress(H, fmt="mp")
    for b, cb in zip(H.blocks, Cm.blocks):
        if b.kind == ohm.DENSE:
            assert np.array_equal(ohm.decode_block(cb), b.D)
            continue
        if not b.rank:
            continue
        W, S, X = ohm.decode_block(cb)
        M = (b.W * b.S) @ b.X.T
        err = np.linalg.norm(M - (W * S) @ X.T, 2)
        delta = H.eps * b.S[0]
        fm = [u.fmt for u in cb.units[:b.rank]]
        r = {f: fm.count(f) for f in ("mp16", "mp32", "mp64")}
        bound = (2 * 3 - 1 + sum(np.sqrt(r[f]) * afl.MP_ROUNDOFF[f] for f in r)) * delta
        assert err <= bound, (err, bound)
