"""The H-LU oracle (Section 4.1: LU factorisation with standard and with accumulator arithmetic,
Algorithms 2 and 3, over optionally compressed storage) against what the mathematics fixes:

* with no admissible blocks the H-LU is the textbook LU without pivoting: the same factors as a
  plain Doolittle loop on the dense matrix, and L U = A to rounding;
* with lowrank blocks, L U approximates A to the truncation accuracy, for both arithmetics;
* the accumulator arithmetic truncates less often than the standard one and, with compressed
  storage, compresses less often and ends with a smaller error || I - A (L U)^{-1} || (the
  observation of Section 4.1).
"""
import numpy as np
import pytest

import synth
from oracle import hlu
from oracle import hmatrix as hm


@pytest.fixture(scope="module")
def problem():
    p = synth.exp2d_problem(512, seed=4)
    root, perm = hm.build_cluster_tree(p.points, 64)
    return p, root, perm


def _dense(H, perm):
    return hm.to_dense(H, decoded=False)[np.ix_(perm, perm)]   # cluster order


def _doolittle(A):
    n = A.shape[0]
    L, U = np.eye(n), np.zeros((n, n))
    for i in range(n):
        U[i, i:] = A[i, i:] - L[i, :i] @ U[:i, i:]
        L[i + 1:, i] = (A[i + 1:, i] - L[i + 1:, :i] @ U[:i, i]) / U[i, i]
    return L, U


@pytest.mark.parametrize("accumulate", [False, True])
def test_dense_partition_is_textbook_lu(problem, accumulate):
    p, root, perm = problem
    H = hm.build_hmatrix(p, 1e-6, leaf_size=64, eta=0.0, method="svd")
    assert all(b.kind == hm.DENSE for b in H.blocks) and len(H.blocks) > 16
    A = _dense(H, perm)
    T, ar = hlu.factorize(H, root, 1e-6, accumulate, compress=False)
    L, U = hlu.lu_dense_factors(T)
    Lr, Ur = _doolittle(A)
    assert np.max(np.abs(L - Lr)) <= 1e-11 and np.max(np.abs(U - Ur)) <= 1e-11 * np.max(np.abs(Ur))
    assert np.linalg.norm(A - L @ U) <= 1e-14 * np.linalg.norm(A) * A.shape[0]
    assert ar.truncations == 0


@pytest.mark.parametrize("accumulate", [False, True])
def test_h_partition_accuracy(problem, accumulate):
    p, root, perm = problem
    eps = 1e-6
    H = hm.build_hmatrix(p, eps, leaf_size=64, eta=2.0, method="svd")
    assert any(b.kind == hm.LOWRANK for b in H.blocks)
    A = _dense(H, perm)
    T, ar = hlu.factorize(H, root, eps, accumulate, compress=False)
    L, U = hlu.lu_dense_factors(T)
    assert np.linalg.norm(A - L @ U, 2) <= 10 * eps * np.linalg.norm(A, 2)
    assert ar.truncations > 0


def test_accumulator_truncates_and_compresses_less_and_errs_less(problem):
    p, root, perm = problem
    eps = 1e-6
    H = hm.build_hmatrix(p, eps, leaf_size=64, eta=2.0, method="svd")
    A = _dense(H, perm)
    res = {}
    for acc in (False, True):
        for comp in (False, True):
            T, ar = hlu.factorize(H, root, eps, acc, comp)
            L, U = hlu.lu_dense_factors(T)
            res[acc, comp] = (hlu.inverse_error(A, L, U), ar.truncations, ar.compressions)
    assert res[True, False][1] < res[False, False][1]          # fewer truncations
    assert res[True, True][2] < res[False, True][2]            # fewer compressions
    assert res[True, True][0] < res[False, True][0]            # compressed: accumulator errs less
    for v in res.values():
        assert v[0] < 1e-2


@pytest.mark.parametrize("seed", [4, 5, 6, 7])
def test_accumulator_error_margin_over_seeds(seed):
    """With compressed storage the accumulator arithmetic's ||I - A (L U)^-1|| is below 0.85 of
    the standard arithmetic's on every seed (measured ratios 0.55-0.80), not just smaller once."""
    p = synth.exp2d_problem(512, seed=seed)
    root, perm = hm.build_cluster_tree(p.points, 64)
    H = hm.build_hmatrix(p, 1e-6, leaf_size=64, eta=2.0, method="svd")
    A = _dense(H, perm)
    err = {}
    for acc in (False, True):
        T, _ = hlu.factorize(H, root, 1e-6, acc, True)
        L, U = hlu.lu_dense_factors(T)
        err[acc] = hlu.inverse_error(A, L, U)
    assert err[True] < 0.85 * err[False], err
