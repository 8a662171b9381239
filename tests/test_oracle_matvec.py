"""Pins of the oracle H-matrix-vector product (Section 5.4) and CG.

* against the dense kernel matrix A x by brute force (n = 4096): within C eps;
* against numpy's product with the decoded dense matrix A~: 1e-14 (a library routine);
* exact identity: at full precision (m = 52) the compressed product equals the uncompressed
  H-matrix product to ~1e-15;
* single rows and multiple right-hand sides agree with the full product;
* CG agrees with the direct solution of A~ x = b and with scipy's CG.
"""
import numpy as np
import pytest

import synth
from oracle import cg as ocg
from oracle import hmatrix as hm
from oracle import matvec as mv


def test_matvec_against_dense_kernel_and_decoded(exp2d_case):
    p, H, C = exp2d_case
    x = synth.rhs(p.n, 1)
    y0 = np.random.default_rng(2).standard_normal(p.n)
    y = mv.matvec(C, x, y0)
    A = p.entries(np.arange(p.n), np.arange(p.n))
    ref = y0 + A @ x
    assert np.linalg.norm(y - ref) / np.linalg.norm(ref) <= 3e-6
    At = hm.to_dense(C)
    ref2 = y0 + At @ x
    assert np.linalg.norm(y - ref2) / np.linalg.norm(ref2) <= 1e-14


def test_full_precision_equals_uncompressed(matern_small_case):
    p, H, C = matern_small_case
    Cfull = hm.compress(H, precision_override=2.0 ** -60)
    x = synth.rhs(p.n, 1)
    y = mv.matvec(Cfull, x)
    Ah = hm.to_dense(H, decoded=False)
    ref = Ah @ x
    assert np.linalg.norm(y - ref) / np.linalg.norm(ref) <= 1e-14


def test_rows_and_multi_rhs(exp2d_case):
    p, H, C = exp2d_case
    X = synth.rhs(p.n, 5, nrhs=2)
    Y = mv.matvec_multi(C, X)
    rows = np.array([0, 17, 4095, 2048])
    r0 = mv.rows_of(C, X[:, 0], rows)
    np.testing.assert_allclose(r0, Y[rows, 0], rtol=0, atol=1e-14 * np.abs(Y).max())
    d = mv.dense_rows(p, X[:, 1], rows)
    A = p.entries(rows, np.arange(p.n))
    np.testing.assert_allclose(d, A @ X[:, 1], rtol=1e-12)


def test_cg_matches_direct_solution():
    p = synth.matern_problem(600, seed=100)
    H = hm.build_hmatrix(p, 1e-6, method="svd")
    C = hm.compress(H)
    At = hm.to_dense(C)
    b = synth.rhs(p.n, 8)
    x, it, rel = ocg.cg(lambda v: At @ v, b, np.zeros(p.n), 1e-10, 2000)
    assert rel <= 1e-10
    xs = np.linalg.solve(At, b)
    kappa = np.linalg.cond(At)
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) <= kappa * 1e-10 * 10
    scipy_sparse = pytest.importorskip("scipy.sparse.linalg")
    xc, info = scipy_sparse.cg(At, b, rtol=1e-10, maxiter=2000)
    assert info == 0
    assert np.linalg.norm(x - xc) / np.linalg.norm(xc) <= kappa * 1e-10 * 10


def test_rows_exact_and_abs_rows_against_full_product(exp2d_case):
    """rows_exact gives the full product's entries bit for bit (the same exactly rounded sums),
    also from the sub-list of blocks that cover the rows; abs_rows equals |A~| |x| from the
    decoded dense matrix."""
    p, H, C = exp2d_case
    x = synth.rhs(p.n, 3)
    y0 = np.random.default_rng(4).standard_normal(p.n)
    full = mv.matvec(C, x, y0)
    rows = np.sort(np.random.default_rng(5).choice(p.n, size=96, replace=False))
    got = mv.rows_exact(C, x, rows, y0)
    assert np.array_equal(got.view(np.int64), full[rows].view(np.int64))
    inv = np.empty(p.n, dtype=np.int64)
    inv[C.perm] = np.arange(p.n)
    pos = inv[rows]
    sub = hm.CHMatrix(C.n, C.perm, [b for b in C.blocks if np.any((pos >= b.row0) & (pos < b.row0 + b.nrows))], C.eps)
    assert len(sub.blocks) < len(C.blocks)
    got2 = mv.rows_exact(sub, x, rows, y0)
    assert np.array_equal(got2.view(np.int64), got.view(np.int64))
    At = hm.to_dense(C)
    ref = np.abs(At[rows]) @ np.abs(x)
    np.testing.assert_allclose(mv.abs_rows(sub, x, rows), ref, rtol=1e-13)
