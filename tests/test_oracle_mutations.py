"""Planted mistakes: each test plants a plausible bug in the ORACLE (on the CPU, through
monkeypatching) and checks that one of the pins used above fails. This shows that the pins
are able to tell a correct oracle from a wrong one.
"""
import numpy as np
import pytest

import synth
from oracle import afl
from oracle import hmatrix as hm
from oracle import matvec as mv


@pytest.fixture(scope="module")
def small():
    p = synth.exp2d_problem(1024, seed=0)
    H = hm.build_hmatrix(p, 1e-6, method="svd")
    A = p.entries(np.arange(p.n), np.arange(p.n))
    x = synth.rhs(p.n, 1)
    return p, H, A, x


def _dense_agreement(H, A, x):
    C = hm.compress(H)
    y = mv.matvec(C, x)
    return np.linalg.norm(y - A @ x) / np.linalg.norm(A @ x)


def _bound_ok(m=20):
    a = np.random.default_rng(1).standard_normal(300)
    unit = afl.encode(a, 2.0 ** -m)
    d = afl.decode(unit)
    return bool(np.all(np.abs(d - a) <= (2.0 ** (-m - 1) + 2.0 ** -51) * (np.abs(a) + unit.m_min)))


def test_correct_oracle_passes(small):
    p, H, A, x = small
    assert _bound_ok()
    assert _dense_agreement(H, A, x) <= 3e-6


def test_dropped_shift_in_decoder_fails(monkeypatch):
    orig = afl.decode

    def bad(unit):
        return orig(unit) + np.where(orig(unit) >= 0, 1, -1) * unit.m_min   # forgets the -1
    monkeypatch.setattr(afl, "decode", bad)
    assert not _bound_ok()


def test_wrong_rounding_direction_fails(monkeypatch):
    def trunc(v, m):    # drops the half-ulp (truncation instead of rounding): error up to 2^-m
        b = v.view(np.uint64).copy()
        if m < 52:
            b &= ~np.uint64((1 << (52 - m)) - 1)
        return b
    monkeypatch.setattr(afl, "_round_to_mantissa", trunc)
    assert not _bound_ok()


def test_unpermuted_x_fails(small, monkeypatch):
    p, H, A, x = small
    orig = mv.block_contributions

    def bad(C, xx):
        C2 = hm.CHMatrix(C.n, np.arange(C.n), C.blocks, C.eps)
        yield from orig(C2, xx)
    monkeypatch.setattr(mv, "block_contributions", bad)
    assert _dense_agreement(H, A, x) > 1e-3


def test_dropped_sigma_fails(small, monkeypatch):
    p, H, A, x = small
    orig = hm.decode_block

    def bad(cb):
        r = orig(cb)
        if cb.kind == hm.LOWRANK:
            W, S, X = r
            return W, np.ones_like(S), X
        return r
    monkeypatch.setattr(hm, "decode_block", bad)
    assert _dense_agreement(H, A, x) > 1e-3


def test_transposed_dense_block_fails(small, monkeypatch):
    p, H, A, x = small
    orig = hm.decode_block

    def bad(cb):
        if cb.kind == hm.DENSE:
            return afl.decode(cb.units[0]).reshape(cb.nrows, cb.ncols, order="C")
        return orig(cb)
    monkeypatch.setattr(hm, "decode_block", bad)
    assert _dense_agreement(H, A, x) > 1e-3


def test_inverted_aplr_rule_fails(small, monkeypatch):
    p, H, A, x = small

    def bad(sigma, eps):      # delta = ||M|| instead of eps ||M||: the eps is dropped
        sigma = np.asarray(sigma)
        return np.array([float(sigma[0]) / float(s) for s in sigma])
    monkeypatch.setattr(afl, "aplr_precisions", bad)
    assert _dense_agreement(H, A, x) > 1e-5


def test_off_by_one_truncation_rank_fails(small, monkeypatch):
    p, H, A, x = small
    orig = hm.truncation_rank
    monkeypatch.setattr(hm, "truncation_rank", lambda s, eps: max(orig(s, eps) - 1, 0))
    H2 = hm.build_hmatrix(p, 1e-6, method="svd")
    worst = 0.0
    for b in H2.blocks[:400]:
        if b.kind == hm.LOWRANK:
            M = p.entries(H2.perm[b.row0:b.row0 + b.nrows], H2.perm[b.col0:b.col0 + b.ncols])
            s0 = np.linalg.svd(M, compute_uv=False)[0]
            worst = max(worst, np.linalg.norm(M - (b.W * b.S) @ b.X.T, 2) / s0)
    assert worst > 1e-6      # Eq. (1) violated: the Eckart-Young pin fails
