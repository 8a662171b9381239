"""FP64 H-matrix-vector product over the decoded compressed H-matrix (oracle; test
infrastructure only).

Section 5.4 multiplies the compressed H-matrix with a vector: every leaf block b = (tau,
sigma) adds A~_b x|sigma to y|tau, where A~_b is the decoded dense block D~_b or the decoded
lowrank block W~_b Sigma_b X~_b^T. The oracle writes this sum out as defined: it decodes every
unit with the oracle decoder, forms t_b = Sigma_b (X~_b^T x|sigma) and W~_b t_b (or D~_b x|sigma)
with exactly rounded sums of the FP64 products (``math.fsum``), and adds every contribution
of an output entry, together with y_in, in one exactly rounded sum. Index order: blocks live in
cluster order; x is read and y written through perm (perm[p] = original index).
"""
from __future__ import annotations

import math

import numpy as np

from . import hmatrix as hm


def _exact_rows(M: np.ndarray, v: np.ndarray) -> np.ndarray:
    """Row-wise exactly rounded sums of the FP64 products M[r, j] * v[j]."""
    P = M * v[None, :]
    return np.array([math.fsum(P[r]) for r in range(P.shape[0])])


def block_contributions(C: hm.CHMatrix, x: np.ndarray):
    """Yield (row0, contribution vector) for every block, in block order."""
    xp = x[C.perm]
    for b in C.blocks:
        xs = xp[b.col0:b.col0 + b.ncols]
        if b.kind == hm.DENSE:
            D = hm.decode_block(b)
            yield b.row0, _exact_rows(D, xs)
        else:
            if b.rank == 0:
                yield b.row0, np.zeros(b.nrows)
                continue
            W, S, X = hm.decode_block(b)
            s = _exact_rows(X.T, xs)          # X~^T x|sigma
            t = S * s                          # t_b = Sigma_b (X~^T x)
            yield b.row0, _exact_rows(W, t)


def matvec(C: hm.CHMatrix, x: np.ndarray, y: np.ndarray | None = None) -> np.ndarray:
    """y_out = y_in + A~ x in original index order (FP64, exactly rounded final sums)."""
    n = C.n
    x = np.asarray(x, dtype=np.float64)
    y_in = np.zeros(n) if y is None else np.asarray(y, dtype=np.float64)
    terms = [[] for _ in range(n)]
    for row0, c in block_contributions(C, x):
        for r, val in enumerate(c):
            terms[row0 + r].append(float(val))
    out = y_in.copy()
    for p in range(n):
        i = int(C.perm[p])
        out[i] = math.fsum([float(y_in[i])] + terms[p])
    return out


def matvec_multi(C: hm.CHMatrix, X: np.ndarray, Y: np.ndarray | None = None) -> np.ndarray:
    """Y_out = Y_in + A~ X for an n x r block of right-hand sides, one column at a time."""
    X = np.asarray(X, dtype=np.float64)
    Y = np.zeros_like(X) if Y is None else np.asarray(Y, dtype=np.float64)
    return np.stack([matvec(C, X[:, j], Y[:, j]) for j in range(X.shape[1])], axis=1)


def rows_of(C: hm.CHMatrix, x: np.ndarray, rows: np.ndarray, y: np.ndarray | None = None) -> np.ndarray:
    """Entries ``rows`` (original indices) of y_in + A~ x, computed row by row."""
    inv = np.empty(C.n, dtype=np.int64)
    inv[C.perm] = np.arange(C.n)
    xp = np.asarray(x, dtype=np.float64)[C.perm]
    out = []
    for i in rows:
        p = int(inv[i])
        terms = [0.0 if y is None else float(y[i])]
        for b in C.blocks:
            if not (b.row0 <= p < b.row0 + b.nrows):
                continue
            r = p - b.row0
            xs = xp[b.col0:b.col0 + b.ncols]
            if b.kind == hm.DENSE:
                D = hm.decode_block(b)
                terms.append(math.fsum(D[r] * xs))
            elif b.rank:
                W, S, X = hm.decode_block(b)
                t = S * np.array([math.fsum(X[:, k] * xs) for k in range(b.rank)])
                terms.append(math.fsum(W[r] * t))
        out.append(math.fsum(terms))
    return np.array(out)


def rows_exact(C: hm.CHMatrix, x: np.ndarray, rows: np.ndarray, y: np.ndarray | None = None) -> np.ndarray:
    """Entries ``rows`` (original indices) of y_in + A~ x with the terms of ``rows_of`` (each
    block's contribution to a row an exactly rounded sum, then all contributions and y_in in
    one exactly rounded sum), but every block that covers one of the rows is decoded, and its
    t_b = Sigma_b (X~_b^T x|sigma) formed, only once. C may hold just the blocks that cover the
    rows."""
    inv = np.empty(C.n, dtype=np.int64)
    inv[C.perm] = np.arange(C.n)
    xp = np.asarray(x, dtype=np.float64)[C.perm]
    rows = np.asarray(rows, dtype=np.int64)
    pos = inv[rows]
    order = np.argsort(pos, kind="stable")
    spos = pos[order]
    terms = [[0.0 if y is None else float(y[i])] for i in rows]
    for b in C.blocks:
        lo = int(np.searchsorted(spos, b.row0, side="left"))
        hi = int(np.searchsorted(spos, b.row0 + b.nrows, side="left"))
        if lo == hi:
            continue
        xs = xp[b.col0:b.col0 + b.ncols]
        if b.kind == hm.DENSE:
            D = hm.decode_block(b)
            for q in order[lo:hi]:
                terms[q].append(math.fsum(D[pos[q] - b.row0] * xs))
        elif b.rank:
            W, S, X = hm.decode_block(b)
            t = S * np.array([math.fsum(X[:, k] * xs) for k in range(b.rank)])
            for q in order[lo:hi]:
                terms[q].append(math.fsum(W[pos[q] - b.row0] * t))
    return np.array([math.fsum(tq) for tq in terms])


def abs_rows(C: hm.CHMatrix, x: np.ndarray, rows: np.ndarray) -> np.ndarray:
    """sum_j |A~_ij| |x_j| for the original indices ``rows`` (the scale of componentwise
    error bounds); C may hold just the blocks that cover the rows."""
    inv = np.empty(C.n, dtype=np.int64)
    inv[C.perm] = np.arange(C.n)
    xa = np.abs(np.asarray(x, dtype=np.float64))[C.perm]
    pos = inv[np.asarray(rows, dtype=np.int64)]
    out = np.zeros(pos.size)
    for b in C.blocks:
        sel = np.nonzero((pos >= b.row0) & (pos < b.row0 + b.nrows))[0]
        if sel.size == 0:
            continue
        xs = xa[b.col0:b.col0 + b.ncols]
        r = pos[sel] - b.row0
        if b.kind == hm.DENSE:
            out[sel] += np.abs(hm.decode_block(b)[r]) @ xs
        elif b.rank:
            W, S, X = hm.decode_block(b)
            out[sel] += np.abs((W[r] * S) @ X.T) @ xs
    return out


def dense_rows(problem, x: np.ndarray, rows: np.ndarray) -> np.ndarray:
    """(A x)[rows] by direct kernel evaluation of the full rows (the plain definition)."""
    x = np.asarray(x, dtype=np.float64)
    out = []
    allj = np.arange(problem.n)
    for i in rows:
        Ki = problem.entries(np.array([i]), allj)[0]
        out.append(math.fsum(Ki * x))
    return np.array(out)
