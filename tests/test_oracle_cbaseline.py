"""Pins of the C CPU baseline (oracle/cmatvec.c, the compressed H-matrix-vector product of
Section 5.4 decoding on the fly on the host cores) against the Python oracle, which is itself
pinned to the paper (Tables 1-2, closed forms, brute force):

* every unit it encodes (Sections 3.2, 3.3) has the oracle's parameters and decodes to the
  oracle's values bit for bit;
* its product equals the oracle's exactly rounded product to FP64 summation accuracy, and its
  plain FP64 product equals the uncompressed H-matrix product;
* the same thread count gives the same bits.
"""
import numpy as np
import pytest

import synth
from oracle import afl
from oracle import cbaseline as cb
from oracle import hmatrix as ohm
from oracle import matvec as omv
from tests._util import oracle_blocks


def _cmatrix(H):
    return cb.CMatrix(H.n, H.perm, oracle_blocks(H), H.eps)


def test_mantissa_bits_matches_the_oracle():
    for u in [1.0, 0.75, 0.5, 0.3, 1e-6, 2.0 ** -20, 2.0 ** -20 * 1.5, 1e-8, 1e-17, 2.0 ** -60, 5e-324]:
        assert cb.lib().hlro_mantissa_bits(u) == afl.mantissa_bits(u), u


def test_units_bit_exact_with_the_oracle(exp2d_case):
    p, H, C = exp2d_case
    M = _cmatrix(H)
    units = [u for b in C.blocks for u in b.units]
    assert M.units() == len(units)
    for k, U in enumerate(units):
        m_min, e, m, vals = M.unit(k)
        assert (m_min, e, m) == (U.m_min, U.e, U.m), k
        assert np.array_equal(vals.view(np.int64), afl.decode(U).view(np.int64)), k
    M.free()


def test_product_and_plain_product(matern_small_case):
    p, H, C = matern_small_case
    M = _cmatrix(H)
    x = synth.rhs(p.n, 1)
    y0 = np.random.default_rng(3).standard_normal(p.n)
    ref = omv.matvec(C, x, y0)
    y = M.matvec(x, y0.copy(), threads=4)
    assert np.linalg.norm(y - ref) / np.linalg.norm(ref) <= 1e-13
    y1 = M.matvec(x, y0.copy(), threads=1)
    assert np.linalg.norm(y1 - ref) / np.linalg.norm(ref) <= 1e-13
    y2 = M.matvec(x, y0.copy(), threads=4)
    assert np.array_equal(y.view(np.int64), y2.view(np.int64))
    plain = M.matvec(x, y0.copy(), plain=True, threads=3)
    Ah = ohm.to_dense(H, decoded=False)
    pref = y0 + Ah @ x
    assert np.linalg.norm(plain - pref) / np.linalg.norm(pref) <= 1e-13
    # the stored (compressed) matrix is within the Eq. 1 accuracy of the plain one
    assert np.linalg.norm(y - plain) / np.linalg.norm(plain) <= 1e-5
    assert M.algorithmic_bytes() < M.algorithmic_bytes(plain=True)
    M.free()
