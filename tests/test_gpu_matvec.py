"""GPU H-matrix-vector product against the CPU oracle, element by element (Section 5.4).

Oracle-built H-matrices (the library's host encoder is byte-exact with the oracle encoder) are
uploaded through the C ABI; y_out = y_in + A~ x on the GPU is compared with the oracle's
exactly rounded product: relative 1e-12 for FP64 accumulation and 1e-6 for FP32 in-block
accumulation (normwise, and componentwise against sum |A~_ij x_j|). Cases span several
tiles and ragged tails (leaf rows 18-64, lowrank blocks wider than one 256-row item), tiny
and degenerate matrices, wide codes (eps = 1e-8), the plain FP64 storage and determinism.
"""
import math

import numpy as np
import pytest

import synth
from oracle import afl
from oracle import hmatrix as ohm
from oracle import matvec as omv
from tests._util import oracle_blocks

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
hg = pytest.importorskip("paper_2308_10960_gb300")

TOL = {"fp64": 1e-12, "fp32": 1e-6}


def _abs_product(C, x):
    """sum_j |A~_ij| |x_j| per row (original order), for componentwise bounds."""
    Cabs = ohm.CHMatrix(C.n, C.perm, C.blocks, C.eps)
    out = np.zeros(C.n)
    xp = np.abs(x)[C.perm]
    for b in C.blocks:
        if b.kind == ohm.DENSE:
            D = np.abs(ohm.decode_block(b))
            out[C.perm[b.row0:b.row0 + b.nrows]] += D @ xp[b.col0:b.col0 + b.ncols]
        elif b.rank:
            W, S, X = ohm.decode_block(b)
            M = np.abs((W * S) @ X.T)
            out[C.perm[b.row0:b.row0 + b.nrows]] += M @ xp[b.col0:b.col0 + b.ncols]
    return out


def _run(A, x, y0, acc):
    xd = torch.from_numpy(x).cuda()
    yd = torch.from_numpy(y0.copy()).cuda()
    A.matvec(xd, yd, acc=acc)
    A.check()
    torch.cuda.synchronize()
    return yd.cpu().numpy()


def _check(got, ref, absprod, acc, y0=None):
    rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert rel <= TOL[acc], (acc, rel)
    scale = absprod + (np.abs(y0) if y0 is not None else 0.0)
    comp = np.max(np.abs(got - ref) / np.maximum(scale, 1e-300))
    assert comp <= 10 * TOL[acc], (acc, comp)


@pytest.mark.parametrize("case", ["exp2d", "matern"])
@pytest.mark.parametrize("acc", ["fp64", "fp32"])
def test_matvec_matches_oracle(case, acc, exp2d_case, matern_small_case):
    p, H, C = exp2d_case if case == "exp2d" else matern_small_case
    x = synth.rhs(p.n, 1)
    y0 = synth.rhs(p.n, 2)
    ref = omv.matvec(C, x, y0)
    A = hg.upload(p.n, H.perm, oracle_blocks(H), H.eps)
    got = _run(A, x, y0, acc)
    _check(got, ref, _abs_product(C, x), acc, y0)
    A.free()


def test_plain_fp64_storage_matches_uncompressed(matern_small_case):
    p, H, C = matern_small_case
    x = synth.rhs(p.n, 3)
    Cfull = ohm.compress(H, precision_override=2.0 ** -60)   # m = 52: A~ equals the FP64 H-matrix
    ref = omv.matvec(Cfull, x)
    A = hg.upload(p.n, H.perm, oracle_blocks(H), H.eps, fmt="fp64")
    got = _run(A, x, np.zeros(p.n), "fp64")
    _check(got, ref, _abs_product(Cfull, x), "fp64")
    A.free()


def test_deterministic_bits(exp2d_case):
    p, H, C = exp2d_case
    A = hg.upload(p.n, H.perm, oracle_blocks(H), H.eps)
    x = synth.rhs(p.n, 1)
    for acc in ("fp32", "fp64"):
        r1 = _run(A, x, np.zeros(p.n), acc)
        r2 = _run(A, x, np.zeros(p.n), acc)
        assert np.array_equal(r1.view(np.int64), r2.view(np.int64))
    A.free()


def test_wide_codes_eps_1e10():
    # eps = 1e-10: dense codes have m = 34 > 23 and w > 32 (the FP32 path's generic decoder)
    p = synth.exp2d_problem(1500, seed=3)
    H = ohm.build_hmatrix(p, 1e-10, method="svd")
    C = ohm.compress(H)
    assert max(u.w for cb in C.blocks for u in cb.units) > 32
    x = synth.rhs(p.n, 1)
    ref = omv.matvec(C, x)
    A = hg.upload(p.n, H.perm, oracle_blocks(H), 1e-10)
    ap = _abs_product(C, x)
    for acc in ("fp64", "fp32"):
        _check(_run(A, x, np.zeros(p.n), acc), ref, ap, acc)
    A.free()


@pytest.mark.parametrize("eps", [1e-4, 1e-8])
def test_low_and_high_accuracy(eps):
    # eps = 1e-4: short codes (m <= 14); eps = 1e-8: dense codes have m = 27 > 23 within 32 bits,
    # and warps whose lanes all have w <= 32 and e <= 4 (or the FP32 fast layout) decode in FP32
    # operations to the FP64 route's values
    p = synth.exp2d_problem(2048, seed=5)
    H = ohm.build_hmatrix(p, eps, method="svd")
    C = ohm.compress(H)
    units = [u for cb in C.blocks for u in cb.units]
    if eps < 1e-7:
        assert any(23 < u.m and u.w <= 32 and u.e <= 4 for u in units)
    else:
        assert max(u.m for u in units) <= 14
    x = synth.rhs(p.n, 2)
    y0 = synth.rhs(p.n, 3)
    ref = omv.matvec(C, x, y0)
    A = hg.upload(p.n, H.perm, oracle_blocks(H), eps)
    ap = _abs_product(C, x) + np.abs(y0)
    for acc in ("fp64", "fp32"):
        _check(_run(A, x, y0, acc), ref, ap, acc)
    A.free()


def _custom(n, blocks, eps=1e-6):
    C = ohm.CHMatrix(n, np.arange(n), [], eps)
    for b in blocks:
        if b["kind"] == 0:
            C.blocks.append(ohm.CBlock(b["row0"], b["nrows"], b["col0"], b["ncols"], 0, None,
                                       [afl.encode(np.asarray(b["D"]).ravel(order="F"), eps)]))
        else:
            S = np.asarray(b["S"])
            us = afl.aplr_precisions(S, eps)
            units = [afl.encode(b["W"][:, i], us[i]) for i in range(S.size)]
            units += [afl.encode(b["X"][:, i], us[i]) for i in range(S.size)]
            C.blocks.append(ohm.CBlock(b["row0"], b["nrows"], b["col0"], b["ncols"], 1, S, units))
    return C


def test_degenerate_blocks():
    g = np.random.default_rng(5)
    n = 130
    Wq, _ = np.linalg.qr(g.standard_normal((65, 3)))
    Xq, _ = np.linalg.qr(g.standard_normal((65, 3)))
    blocks = [
        {"row0": 0, "nrows": 65, "col0": 0, "ncols": 65, "kind": 0, "D": g.standard_normal((65, 65))},
        {"row0": 0, "nrows": 65, "col0": 65, "ncols": 65, "kind": 1, "W": Wq, "S": np.array([3.0, 1e-3, 2e-6]),
         "X": Xq},
        {"row0": 65, "nrows": 65, "col0": 0, "ncols": 65, "kind": 1, "W": np.zeros((65, 0)), "S": np.zeros(0),
         "X": np.zeros((65, 0))},                                         # rank 0
        {"row0": 65, "nrows": 65, "col0": 65, "ncols": 1, "kind": 0, "D": np.zeros((65, 1))},   # all-zero unit
        {"row0": 65, "nrows": 65, "col0": 66, "ncols": 64, "kind": 0, "D": g.standard_normal((65, 64))},
    ]
    C = _custom(n, blocks)
    x = synth.rhs(n, 1)
    y0 = synth.rhs(n, 2)
    ref = omv.matvec(C, x, y0)
    A = hg.upload(n, None, blocks, 1e-6)
    ap = _abs_product(C, x)
    for acc in ("fp64", "fp32"):
        _check(_run(A, x, y0, acc), ref, ap, acc, y0)
    A.free()


@pytest.mark.parametrize("n", [1, 2, 64, 65])
def test_tiny_single_dense(n):
    g = np.random.default_rng(n)
    D = g.standard_normal((n, n))
    blocks = [{"row0": 0, "nrows": n, "col0": 0, "ncols": n, "kind": 0, "D": D}]
    C = _custom(n, blocks)
    x = g.standard_normal(n)
    ref = omv.matvec(C, x)
    A = hg.upload(n, None, blocks, 1e-6)
    for acc in ("fp64", "fp32"):
        got = _run(A, x, np.zeros(n), acc)
        assert np.linalg.norm(got - ref) <= TOL[acc] * max(np.linalg.norm(ref), 1e-300) * 10
    A.free()


def test_permutation_and_host_api(exp2d_case):
    p, H, C = exp2d_case
    x = synth.rhs(p.n, 7)
    y0 = synth.rhs(p.n, 8)
    ref = omv.matvec(C, x, y0)
    A = hg.upload(p.n, H.perm, oracle_blocks(H), H.eps)
    yh = y0.copy()
    A.matvec_host(x, yh, acc="fp64")
    assert np.linalg.norm(yh - ref) / np.linalg.norm(ref) <= 1e-12
    A.free()
