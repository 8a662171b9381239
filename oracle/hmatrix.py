"""H-matrix construction and compression (oracle; test infrastructure only).

* Cluster tree (Def. 2.1): a binary tree of disjoint index sets whose sons partition their
  father. Split rule (the paper gives none): the bounding box of the cluster's points is cut
  at the midpoint of its longest edge (the first axis on ties); points with coordinate <= the
  midpoint go to the first son, in their father's order. If one side would be empty the
  cluster is split at the median of (coordinate, original index). Clusters with at most
  ``leaf_size`` indices are leaves.
* Block tree (Def. 2.2): (tau, sigma) is a leaf if it is admissible or one of tau, sigma is a
  leaf cluster; otherwise its sons are all pairs of sons. Standard admissibility (Section 5.1):
  min(diam tau, diam sigma) <= eta * dist(tau, sigma), with diam the diagonal of the bounding
  box and dist the Euclidean distance between the two boxes.
* H-matrix (Def. 2.3 with Eq. 1): admissible leaves are lowrank W Sigma X^T with orthonormal
  W, X (Section 3.3) and ||M - W Sigma X^T||_2 <= eps ||M||_2, i.e. sigma_i > eps * sigma_0 are
  kept; other leaves are dense.
* Lowrank approximation: truncated SVD of the full block (``method="svd"``), or ACA with
  partial pivoting (reference [Beb:2000] of Section 5.1) at eps/10 followed by SVD
  recompression (Algorithm 1: QR of both factors, SVD of R_U R_V^T, truncation), keeping
  Sigma separate from W as Section 4 allows.
* Compression (Section 3): a dense leaf is one AFL unit (column-major) at precision eps; a
  lowrank leaf stores every column of W and of X as its own AFL unit at u~_i = eps sigma_0 /
  sigma_i (APLR, Section 3.3); Sigma stays FP64.

All blocks are addressed in cluster order: block rows [row0, row0+nrows) and columns
[col0, col0+ncols) index ``perm``, where perm[p] is the original index at cluster position p.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import afl

DENSE = 0
LOWRANK = 1


@dataclass
class Cluster:
    lo: int
    hi: int
    bmin: np.ndarray
    bmax: np.ndarray
    sons: list = field(default_factory=list)
    level: int = 0

    @property
    def size(self) -> int:
        return self.hi - self.lo


def build_cluster_tree(points: np.ndarray, leaf_size: int = 64):
    """Return (root, perm) of the bounding-box bisection cluster tree (Def. 2.1)."""
    points = np.asarray(points, dtype=np.float64)
    n = points.shape[0]
    perm = np.arange(n, dtype=np.int64)

    def rec(lo: int, hi: int, level: int) -> Cluster:
        idx = perm[lo:hi].copy()
        P = points[idx]
        bmin = P.min(axis=0)
        bmax = P.max(axis=0)
        c = Cluster(lo, hi, bmin, bmax, [], level)
        if hi - lo <= leaf_size:
            return c
        ext = bmax - bmin
        d = int(np.argmax(ext))
        mid = 0.5 * (bmin[d] + bmax[d])
        first = P[:, d] <= mid
        nfirst = int(first.sum())
        if nfirst == 0 or nfirst == hi - lo:
            order = np.lexsort((idx, P[:, d]))
            perm[lo:hi] = idx[order]
            nfirst = (hi - lo) // 2
        else:
            perm[lo:hi] = np.concatenate([idx[first], idx[~first]])
        c.sons = [rec(lo, lo + nfirst, level + 1), rec(lo + nfirst, hi, level + 1)]
        return c

    root = rec(0, n, 0)
    return root, perm


def diam(c: Cluster) -> float:
    """Diagonal length of the cluster's bounding box."""
    s = 0.0
    for v in (c.bmax - c.bmin):
        s += float(v) * float(v)
    return math.sqrt(s)


def dist(a: Cluster, b: Cluster) -> float:
    """Euclidean distance between two bounding boxes (0 if they intersect)."""
    s = 0.0
    for k in range(a.bmin.size):
        g = max(0.0, float(b.bmin[k]) - float(a.bmax[k]), float(a.bmin[k]) - float(b.bmax[k]))
        s += g * g
    return math.sqrt(s)


def admissible(t: Cluster, s: Cluster, eta: float) -> bool:
    """Standard admissibility min(diam t, diam s) <= eta * dist(t, s) (Section 5.1)."""
    return min(diam(t), diam(s)) <= eta * dist(t, s)


def build_block_tree(rows: Cluster, cols: Cluster, eta: float = 2.0):
    """Leaves of the block tree (Def. 2.2) as (tau, sigma, is_admissible), depth-first."""
    leaves = []

    def rec(t: Cluster, s: Cluster):
        if admissible(t, s, eta):
            leaves.append((t, s, True))
        elif not t.sons or not s.sons:
            leaves.append((t, s, False))
        else:
            for t2 in t.sons:
                for s2 in s.sons:
                    rec(t2, s2)

    rec(rows, cols)
    return leaves


@dataclass
class Block:
    row0: int
    nrows: int
    col0: int
    ncols: int
    kind: int
    D: np.ndarray | None = None       # nrows x ncols (dense)
    W: np.ndarray | None = None       # nrows x k, orthonormal columns
    S: np.ndarray | None = None       # k singular values, descending
    X: np.ndarray | None = None       # ncols x k, orthonormal columns

    @property
    def rank(self) -> int:
        return 0 if self.S is None else int(self.S.size)


@dataclass
class HMatrix:
    n: int
    perm: np.ndarray
    blocks: list
    eps: float


def truncation_rank(s: np.ndarray, eps: float) -> int:
    """Number of singular values sigma_i > eps * sigma_0 (Eq. 1 in the spectral norm)."""
    if s.size == 0 or s[0] == 0.0:
        return 0
    return int(np.count_nonzero(s > eps * s[0]))


def lowrank_svd(M: np.ndarray, eps: float):
    """Truncated SVD of a full block: (W, S, X) with M ~ W diag(S) X^T."""
    U, s, Vt = np.linalg.svd(M, full_matrices=False)
    k = truncation_rank(s, eps)
    return U[:, :k].copy(), s[:k].copy(), Vt[:k].T.copy()


def recompress(U: np.ndarray, V: np.ndarray, eps: float):
    """Algorithm 1 (truncation via SVD) on U V^T, returning W, Sigma, X with Sigma separate."""
    if U.shape[1] == 0:
        return U[:, :0], np.zeros(0), V[:, :0]
    QU, RU = np.linalg.qr(U)
    QV, RV = np.linalg.qr(V)
    Us, s, Vst = np.linalg.svd(RU @ RV.T)
    k = truncation_rank(s, eps)
    return QU @ Us[:, :k], s[:k].copy(), QV @ Vst[:k].T


def aca(entry_rows, entry_cols, nrows: int, ncols: int, eps_aca: float, max_rank: int):
    """ACA with partial pivoting.

    ``entry_rows(i)`` returns row i of the block, ``entry_cols(j)`` column j. The first pivot
    row is 0; the next pivot row is the unused row where the newest column term is largest
    in magnitude. Iteration stops after a term with ||u_k|| ||v_k|| <= eps_aca ||S_k||_F
    (S_k the current approximation) or when every row has been used. Returns (U, V, ok)
    with block ~ U V^T; ok is False when ``max_rank`` terms did not reach the stop rule.
    """
    us, vs = [], []
    used = np.zeros(nrows, dtype=bool)
    norm2 = 0.0
    i = 0
    while True:
        if len(us) >= max_rank:
            return _stack(us, nrows), _stack(vs, ncols), False
        used[i] = True
        row = entry_rows(i).astype(np.float64)
        for u, v in zip(us, vs):
            row = row - u[i] * v
        j = int(np.argmax(np.abs(row)))
        if row[j] == 0.0:
            rest = np.flatnonzero(~used)
            if rest.size == 0:
                break
            i = int(rest[0])
            continue
        v = row / row[j]
        col = entry_cols(j).astype(np.float64)
        for u, vv in zip(us, vs):
            col = col - vv[j] * u
        u = col
        cross = 0.0
        for uu, vv in zip(us, vs):
            cross += float(uu @ u) * float(vv @ v)
        nu2 = float(u @ u) * float(v @ v)
        norm2 = norm2 + 2.0 * cross + nu2
        us.append(u)
        vs.append(v)
        if math.sqrt(nu2) <= eps_aca * math.sqrt(max(norm2, 0.0)):
            break
        cand = np.abs(u).copy()
        cand[used] = -1.0
        if np.all(used):
            break
        i = int(np.argmax(cand))
    return _stack(us, nrows), _stack(vs, ncols), True


def _stack(vs, n):
    if not vs:
        return np.zeros((n, 0))
    return np.stack(vs, axis=1)


def build_hmatrix(problem, eps: float, leaf_size: int = 64, eta: float = 2.0,
                  method: str = "svd") -> HMatrix:
    """Build the FP64 H-matrix of ``problem`` (a ``synth.Problem``) at accuracy eps."""
    root, perm = build_cluster_tree(problem.points, leaf_size)
    leaves = build_block_tree(root, root, eta)
    blocks = []
    for t, s, adm in leaves:
        I = perm[t.lo:t.hi]
        J = perm[s.lo:s.hi]
        if not adm:
            blocks.append(Block(t.lo, t.size, s.lo, s.size, DENSE, D=problem.entries(I, J)))
            continue
        if method == "svd":
            W, S, X = lowrank_svd(problem.entries(I, J), eps)
        elif method == "aca":
            cap = max(1, min(t.size, s.size) // 2)
            U, V, ok = aca(lambda i: problem.entries(I[i:i + 1], J)[0],
                           lambda j: problem.entries(I, J[j:j + 1])[:, 0],
                           t.size, s.size, eps / 10.0, cap)
            if ok:
                W, S, X = recompress(U, V, eps)
            else:
                W, S, X = lowrank_svd(problem.entries(I, J), eps)
        else:
            raise ValueError(method)
        blocks.append(Block(t.lo, t.size, s.lo, s.size, LOWRANK, W=W, S=S, X=X))
    return HMatrix(problem.n, perm, blocks, eps)


@dataclass
class CBlock:
    """A compressed block: dense -> units = [D]; lowrank -> units = W columns + X columns."""
    row0: int
    nrows: int
    col0: int
    ncols: int
    kind: int
    S: np.ndarray | None
    units: list

    @property
    def rank(self) -> int:
        return 0 if self.S is None else int(self.S.size)


@dataclass
class CHMatrix:
    n: int
    perm: np.ndarray
    blocks: list
    eps: float


def compress(H: HMatrix, eps: float | None = None, precision_override: float | None = None,
             fmt: str = "afl") -> CHMatrix:
    """AFL (dense) / AFL-APLR (lowrank) compression of every leaf; fmt selects AFL or one of
    its byte-aligned variants AFLP, BFL, DFL (Section 3.2), with the same precisions, or the
    mixed precision comparison format MP-D-S-H ("mp", Section 3.3).

    ``precision_override`` replaces every precision (tests use 2^-60 to make m = 52).
    """
    eps = H.eps if eps is None else eps
    out = []
    for b in H.blocks:
        if b.kind == DENSE:
            u = eps if precision_override is None else precision_override
            if fmt == "mp":   # the mixed precision comparison keeps dense leaves in FP64
                units = [afl.encode_mp(b.D.ravel(order="F"), u, "mp64")]
            else:
                units = [afl.encode(b.D.ravel(order="F"), u, fmt)]
            out.append(CBlock(b.row0, b.nrows, b.col0, b.ncols, DENSE, None, units))
        else:
            us = afl.aplr_precisions(b.S, eps)
            if precision_override is not None:
                us = np.full_like(us, precision_override)
            units = [afl.encode(b.W[:, i], us[i], fmt) for i in range(b.rank)]
            units += [afl.encode(b.X[:, i], us[i], fmt) for i in range(b.rank)]
            out.append(CBlock(b.row0, b.nrows, b.col0, b.ncols, LOWRANK, b.S.copy(), units))
    return CHMatrix(H.n, H.perm.copy(), out, eps)


def decode_block(cb: CBlock):
    """FP64 factors of a compressed block: D~ (dense) or (W~, S, X~) (lowrank)."""
    if cb.kind == DENSE:
        return afl.decode(cb.units[0]).reshape(cb.nrows, cb.ncols, order="F")
    k = cb.rank
    W = np.stack([afl.decode(u) for u in cb.units[:k]], axis=1) if k else np.zeros((cb.nrows, 0))
    X = np.stack([afl.decode(u) for u in cb.units[k:]], axis=1) if k else np.zeros((cb.ncols, 0))
    return W, cb.S, X


def to_dense(H, decoded: bool = True) -> np.ndarray:
    """Assemble the full n x n matrix in ORIGINAL index order (small n only)."""
    A = np.zeros((H.n, H.n))
    P = H.perm
    for b in H.blocks:
        if isinstance(b, CBlock):
            if b.kind == DENSE:
                M = decode_block(b)
            else:
                W, S, X = decode_block(b)
                M = (W * S) @ X.T
        else:
            M = b.D if b.kind == DENSE else (b.W * b.S) @ b.X.T
        A[np.ix_(P[b.row0:b.row0 + b.nrows], P[b.col0:b.col0 + b.ncols])] = M
    return A


def storage_bytes(C: CHMatrix, header_bytes: int = 16) -> dict:
    """FP64 vs compressed storage: FP64 = 8 per value (+8 per singular value); compressed =
    unpadded stream bytes + one header per unit + 8 per singular value."""
    fp64 = 0
    comp = 0
    for b in C.blocks:
        if b.kind == DENSE:
            fp64 += 8 * b.nrows * b.ncols
        else:
            fp64 += 8 * b.rank * (b.nrows + b.ncols + 1)
            comp += 8 * b.rank
        for u in b.units:
            comp += afl.stream_bytes(u) + header_bytes
    return {"fp64": fp64, "compressed": comp, "ratio": comp / fp64 if fp64 else 0.0}
