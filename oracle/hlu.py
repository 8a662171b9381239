"""H-LU factorisation over (compressed) H-matrices: oracle (test infrastructure only; the product
path never imports it).

Section 4.1 runs the LU factorisation of an H-matrix with compressed storage in two ways: with
the standard arithmetic of Algorithm 2 (every update is applied to its destination block at
once, a lowrank destination truncated by Algorithm 1 each time) and with the accumulator
arithmetic of Algorithm 3 (updates are collected top-down per block and applied in one step at
the leaf). With compression, storage is converted "semi-on-the-fly" (Section 4): a block is
decoded before it is used and re-encoded after it changed (AFL for dense blocks at eps,
AFL-APLR for lowrank blocks, Section 3.3), so the standard arithmetic compresses after every
update while the accumulator arithmetic compresses each block once, when it is final.

The paper gives the recursive multiplication (Algorithms 2 and 3) and notes that triangular
solves and the LU factorisation follow the same recursion; the LU used here is the usual
block recursion over the binary cluster tree, without pivoting:

    LU(A_00); A_01 := L_00^{-1} A_01; A_10 := A_10 U_00^{-1};
    A_11 := A_11 - A_10 A_01 (Algorithm 2 or 3); LU(A_11).

Matrices are plain FP64 numpy arrays; a lowrank block is M = U V^T (U = W Sigma, V = X after the
truncation of Algorithm 1, whose rank rule keeps sigma_i > eps sigma_0, Eq. 1).
"""
from __future__ import annotations

import numpy as np

from . import afl
from .hmatrix import DENSE, recompress, truncation_rank


class Node:
    """Block (tau, sigma) of the H-matrix: a dense leaf (D), a lowrank leaf (U, V with M = U V^T)
    or a 2 x 2 block of sons (sons[i][j] = (tau_i, sigma_j))."""

    def __init__(self, r0, nr, c0, nc):
        self.r0, self.nr, self.c0, self.nc = r0, nr, c0, nc
        self.kind = None        # "dense", "lowrank" or "node"
        self.D = None
        self.U = None
        self.V = None
        self.sons = None


def build_tree(H, root):
    """Block tree of the H-matrix H (oracle.hmatrix.HMatrix) over the cluster tree `root` (the
    tree H was built on): leaves from H.blocks, inner blocks split along both clusters' sons."""
    leaves = {(b.row0, b.nrows, b.col0, b.ncols): b for b in H.blocks}

    def rec(t, s):
        nd = Node(t.lo, t.size, s.lo, s.size)
        b = leaves.get((t.lo, t.size, s.lo, s.size))
        if b is not None:
            if b.kind == DENSE:
                nd.kind, nd.D = "dense", np.array(b.D, dtype=np.float64)
            else:
                nd.kind = "lowrank"
                nd.U = np.array(b.W * b.S[None, :] if b.rank else np.zeros((t.size, 0)))
                nd.V = np.array(b.X if b.rank else np.zeros((s.size, 0)))
            return nd
        nd.kind = "node"
        nd.sons = [[rec(t2, s2) for s2 in s.sons] for t2 in t.sons]
        return nd

    return rec(root, root)


def to_dense(nd) -> np.ndarray:
    if nd.kind == "dense":
        return nd.D.copy()
    if nd.kind == "lowrank":
        return nd.U @ nd.V.T
    top = np.hstack([to_dense(nd.sons[0][0]), to_dense(nd.sons[0][1])])
    bot = np.hstack([to_dense(nd.sons[1][0]), to_dense(nd.sons[1][1])])
    return np.vstack([top, bot])


def _split_rows(nd):
    return nd.sons[0][0].nr


def _split_cols(nd):
    return nd.sons[0][0].nc


def matmul(nd, X) -> np.ndarray:
    """nd @ X for a dense X with nd.nc rows."""
    if nd.kind == "dense":
        return nd.D @ X
    if nd.kind == "lowrank":
        return nd.U @ (nd.V.T @ X)
    c = _split_cols(nd)
    top = matmul(nd.sons[0][0], X[:c]) + matmul(nd.sons[0][1], X[c:])
    bot = matmul(nd.sons[1][0], X[:c]) + matmul(nd.sons[1][1], X[c:])
    return np.vstack([top, bot])


def rmatmul(nd, Y) -> np.ndarray:
    """nd^T @ Y for a dense Y with nd.nr rows."""
    if nd.kind == "dense":
        return nd.D.T @ Y
    if nd.kind == "lowrank":
        return nd.V @ (nd.U.T @ Y)
    r = _split_rows(nd)
    left = rmatmul(nd.sons[0][0], Y[:r]) + rmatmul(nd.sons[1][0], Y[r:])
    right = rmatmul(nd.sons[0][1], Y[:r]) + rmatmul(nd.sons[1][1], Y[r:])
    return np.vstack([left, right])


class Arith:
    """The arithmetic of one factorisation: truncation accuracy eps, optional compressed storage
    of the blocks, and counters (truncations, compressions)."""

    def __init__(self, eps: float, compress: bool = False):
        self.eps = eps
        self.compress = compress
        self.truncations = 0
        self.compressions = 0

    # ---- storage conversion (Section 4: decode before use, encode after an update) ----------
    def store(self, nd):
        """Round the leaf nd through its compressed storage format (AFL / AFL-APLR)."""
        if not self.compress or nd.kind == "node":
            return
        self.compressions += 1
        if nd.kind == "dense":
            shp = nd.D.shape
            nd.D = afl.decode(afl.encode(nd.D.ravel(order="F"), self.eps)).reshape(shp, order="F")
            return
        k = nd.U.shape[1]
        if k == 0:
            return
        # the APLR form W Sigma X^T of U V^T (orthonormal factors, Algorithm 1 without truncation)
        QU, RU = np.linalg.qr(nd.U)
        QV, RV = np.linalg.qr(nd.V)
        Us, s, Vst = np.linalg.svd(RU @ RV.T)
        W, X = QU @ Us, QV @ Vst.T
        if s[0] == 0.0:
            nd.U, nd.V = nd.U[:, :0], nd.V[:, :0]
            return
        us = afl.aplr_precisions(s, self.eps)
        Wd = np.stack([afl.decode(afl.encode(W[:, i], us[i])) for i in range(s.size)], axis=1)
        Xd = np.stack([afl.decode(afl.encode(X[:, i], us[i])) for i in range(s.size)], axis=1)
        nd.U, nd.V = Wd * s[None, :], Xd

    # ---- updates -------------------------------------------------------------------------
    def add(self, nd, P, alpha=1.0):
        """nd += alpha P, P = ("dense", D) or ("lowrank", U, V) over nd's rows and columns;
        a lowrank destination is truncated (Algorithm 1) after the update."""
        if nd.kind == "node":
            r, c = _split_rows(nd), _split_cols(nd)
            for i in range(2):
                for j in range(2):
                    rs = slice(0, r) if i == 0 else slice(r, None)
                    cs = slice(0, c) if j == 0 else slice(c, None)
                    if P[0] == "dense":
                        self.add(nd.sons[i][j], ("dense", P[1][rs, cs]), alpha)
                    else:
                        self.add(nd.sons[i][j], ("lowrank", P[1][rs], P[2][cs]), alpha)
            return
        if nd.kind == "dense":
            nd.D = nd.D + alpha * (P[1] if P[0] == "dense" else P[1] @ P[2].T)
            self.store(nd)
            return
        # lowrank destination
        self.truncations += 1
        if P[0] == "dense":
            M = nd.U @ nd.V.T + alpha * P[1]
            Uf, s, Vt = np.linalg.svd(M, full_matrices=False)
            k = truncation_rank(s, self.eps)
            nd.U, nd.V = Uf[:, :k] * s[None, :k], Vt[:k].T
        else:
            W, S, X = recompress(np.hstack([nd.U, alpha * P[1]]), np.hstack([nd.V, P[2]]), self.eps)
            nd.U, nd.V = W * S[None, :], X
        self.store(nd)

    @staticmethod
    def product(A, B):
        """A @ B as ("dense", D) or ("lowrank", U, V) (exact in FP64, no truncation)."""
        if A.kind == "lowrank":
            return ("lowrank", A.U, rmatmul(B, A.V))
        if B.kind == "lowrank":
            return ("lowrank", matmul(A, B.U), B.V)
        return ("dense", to_dense(A) @ to_dense(B))

    def hmul(self, alpha, A, B, C):
        """Algorithm 2: C := C + alpha A B, recursing while all three blocks have sons."""
        if A.kind == "node" and B.kind == "node" and C.kind == "node":
            for i in range(2):
                for j in range(2):
                    for l in range(2):
                        self.hmul(alpha, A.sons[i][l], B.sons[l][j], C.sons[i][j])
            return
        self.add(C, self.product(A, B), alpha)


# ---- triangular solves with the packed LU factors of a diagonal block -----------------------
def _lower_unit_solve_dense(L, B):
    """L^{-1} B, L the unit lower triangle of the factors held by diagonal block L."""
    if L.kind == "dense":
        n = L.D.shape[0]
        X = np.array(B, dtype=np.float64)
        for i in range(n):
            X[i] -= L.D[i, :i] @ X[:i]
        return X
    r = _split_rows(L)
    X0 = _lower_unit_solve_dense(L.sons[0][0], B[:r])
    X1 = _lower_unit_solve_dense(L.sons[1][1], B[r:] - matmul(L.sons[1][0], X0))
    return np.vstack([X0, X1])


def _upper_solve_right_dense(U, B):
    """B U^{-1}, U the upper triangle (with diagonal) of the factors held by diagonal block U."""
    if U.kind == "dense":
        n = U.D.shape[0]
        X = np.array(B, dtype=np.float64)
        for j in range(n):
            X[:, j] = (X[:, j] - X[:, :j] @ U.D[:j, j]) / U.D[j, j]
        return X
    c = _split_cols(U)
    X0 = _upper_solve_right_dense(U.sons[0][0], B[:, :c])
    X1 = _upper_solve_right_dense(U.sons[1][1], B[:, c:] - rmatmul(U.sons[0][1], X0.T).T)  # X0 U_01
    return np.hstack([X0, X1])


class HLU:
    """H-LU of a block tree in place: every diagonal leaf holds L \\ U packed (unit lower L),
    off-diagonal blocks hold the blocks of L (below) and U (above)."""

    def __init__(self, ar: Arith):
        self.ar = ar

    # L^{-1} B (B to the right of diagonal block L)
    def solve_lower(self, L, B):
        if B.kind == "dense":
            B.D = _lower_unit_solve_dense(L, B.D)
            self.ar.store(B)
        elif B.kind == "lowrank":
            B.U = _lower_unit_solve_dense(L, B.U)
            self.ar.store(B)
        else:
            for j in range(2):
                self.solve_lower(L.sons[0][0], B.sons[0][j])
                self.update(-1.0, L.sons[1][0], B.sons[0][j], B.sons[1][j])
                self.solve_lower(L.sons[1][1], B.sons[1][j])

    # B U^{-1} (B below diagonal block U)
    def solve_upper(self, U, B):
        if B.kind == "dense":
            B.D = _upper_solve_right_dense(U, B.D)
            self.ar.store(B)
        elif B.kind == "lowrank":
            B.V = _upper_solve_right_dense(U, B.V.T).T
            self.ar.store(B)
        else:
            for i in range(2):
                self.solve_upper(U.sons[0][0], B.sons[i][0])
                self.update(-1.0, B.sons[i][0], U.sons[0][1], B.sons[i][1])
                self.solve_upper(U.sons[1][1], B.sons[i][1])

    def update(self, alpha, A, B, C):
        self.ar.hmul(alpha, A, B, C)

    def factor(self, A):
        if A.kind == "dense":
            D = A.D
            n = D.shape[0]
            for k in range(n):  # Doolittle without pivoting, packed
                D[k + 1:, k] /= D[k, k]
                D[k + 1:, k + 1:] -= np.outer(D[k + 1:, k], D[k, k + 1:])
            self.ar.store(A)
            return
        self.factor(A.sons[0][0])
        self.solve_lower(A.sons[0][0], A.sons[0][1])
        self.solve_upper(A.sons[0][0], A.sons[1][0])
        self.update(-1.0, A.sons[1][0], A.sons[0][1], A.sons[1][1])
        self.factor(A.sons[1][1])


class HLUAccu(HLU):
    """The same factorisation with the accumulator arithmetic of Algorithm 3: an update
    C -= A B is recorded as pending at C; before a block is used (factored, solved, or an
    operand), its pending updates are evaluated top-down: products with a leaf operand go into
    the block's accumulator (a dense FP64 matrix, not compressed), products of two inner blocks
    are split over the sons, and a leaf applies its accumulator in one step."""

    def __init__(self, ar: Arith):
        super().__init__(ar)
        self.pending = {}   # id(node) -> list of (alpha, A, B)
        self.acc = {}       # id(node) -> dense accumulator

    def update(self, alpha, A, B, C):
        self.pending.setdefault(id(C), []).append((alpha, A, B))

    def _accumulate(self, C, M):
        a = self.acc.get(id(C))
        self.acc[id(C)] = M if a is None else a + M

    def settle(self, C):
        """Apply all updates pending at C or recorded in its accumulator (Algorithm 3)."""
        for alpha, A, B in self.pending.pop(id(C), []):
            self.settle(A)
            self.settle(B)
            if A.kind == "node" and B.kind == "node" and C.kind == "node":
                for i in range(2):
                    for j in range(2):
                        for l in range(2):
                            self.pending.setdefault(id(C.sons[i][j]), []).append((alpha, A.sons[i][l], B.sons[l][j]))
            else:
                P = Arith.product(A, B)
                self._accumulate(C, alpha * (P[1] if P[0] == "dense" else P[1] @ P[2].T))
        M = self.acc.pop(id(C), None)
        if C.kind == "node":
            if M is not None:
                r, c = _split_rows(C), _split_cols(C)
                for i in range(2):
                    for j in range(2):
                        rs = slice(0, r) if i == 0 else slice(r, None)
                        cs = slice(0, c) if j == 0 else slice(c, None)
                        self._accumulate(C.sons[i][j], M[rs, cs])
            for i in range(2):
                for j in range(2):
                    self.settle(C.sons[i][j])
        elif M is not None:
            self.ar.add(C, ("dense", M), 1.0)

    def solve_lower(self, L, B):
        self.settle(B)
        super().solve_lower(L, B)

    def solve_upper(self, U, B):
        self.settle(B)
        super().solve_upper(U, B)

    def factor(self, A):
        self.settle(A)
        super().factor(A)


def factorize(H, root, eps: float, accumulate: bool, compress: bool):
    """H-LU of the H-matrix H (over cluster tree `root`) at truncation accuracy eps; returns
    (block tree holding the factors, Arith with its counters)."""
    T = build_tree(H, root)
    ar = Arith(eps, compress)
    if compress:  # the matrix itself is stored compressed before the factorisation
        def rec(nd):
            if nd.kind == "node":
                for row in nd.sons:
                    for s in row:
                        rec(s)
            else:
                ar.store(nd)
        rec(T)
        ar.compressions = 0
    (HLUAccu(ar) if accumulate else HLU(ar)).factor(T)
    return T, ar


def lu_dense_factors(T):
    """(L, U) as dense matrices from a factored block tree (cluster order)."""
    M = to_dense(T)
    L = np.tril(M, -1) + np.eye(M.shape[0])
    U = np.triu(M)
    return L, U


def inverse_error(A: np.ndarray, L: np.ndarray, U: np.ndarray) -> float:
    """|| I - A (L U)^{-1} ||_2, the accuracy measure of Section 4.1."""
    n = A.shape[0]
    X = np.linalg.solve(L.T, np.linalg.solve(U.T, A.T)).T   # A (LU)^{-1} = A U^{-1} L^{-1}
    return float(np.linalg.norm(np.eye(n) - X, 2))
