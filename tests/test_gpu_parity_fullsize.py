"""Oracle parity on the benchmarked matrices (Section 5.4 product over the stored AFL-APLR
matrix of Sections 3.2-3.3): the n = 262144 Laplace sphere built natively, as the benchmark
times it, at eps = 1e-6 and at eps = 1e-8 (the widest codes), and rows of the n = 2^21 case.

The oracle cannot build these matrices, so it checks the stored one: the library's host
builder gives the FP64 blocks (W, Sigma, X, D), the oracle encodes them with its own encoder
and decoder (readings s1-s6), and
* decoded units: every value the GPU decodes (hlr_decode_units) equals the oracle's decode, bit
  for bit, on a seeded sample of blocks (>= 2000 units);
* products: y = A~ x from the benchmarked launch (FP32 in-block and FP64 accumulation) on all
  rows of seeded leaf clusters (>= 512 rows) against the oracle's exactly rounded rows over
  the same stored blocks: normwise 1e-6 (FP32) / 1e-12 (FP64) and componentwise 10x that
  against sum_j |A~_ij x_j|.
"""
import numpy as np
import pytest

import synth
from oracle import afl
from oracle import hmatrix as ohm
from oracle import matvec as omv

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
hg = pytest.importorskip("paper_2308_10960_gb300")

TOL = {"fp32": 1e-6, "fp64": 1e-12}


def _leaf_rows(Hh, rng, min_rows):
    """Original indices of every row of seeded leaf clusters (the row ranges of the dense
    diagonal blocks, <= 64 rows each), as many as give at least `min_rows` rows, and the block
    indices that cover them."""
    st = Hh.structure()
    diag = np.nonzero((st[:, 4] == hg.HLR_DENSE) & (st[:, 0] == st[:, 2]) & (st[:, 1] == st[:, 3]))[0]
    order = rng.permutation(diag)
    pick = []
    while sum(st[i, 1] for i in pick) < min_rows:
        pick.append(order[len(pick)])
    pos = np.concatenate([np.arange(st[i, 0], st[i, 0] + st[i, 1]) for i in pick])
    cover = np.nonzero([np.any((pos >= r0) & (pos < r0 + nr)) for r0, nr in zip(st[:, 0], st[:, 1])])[0]
    return Hh.perm[pos], cover


def _oracle_blocks(Hh, idx, eps):
    """The oracle's compression of blocks idx of the library-built matrix (cluster order)."""
    blocks = []
    for i in idx:
        b = Hh.block(int(i))
        if b["kind"] == hg.HLR_DENSE:
            blocks.append(ohm.Block(b["row0"], b["nrows"], b["col0"], b["ncols"], ohm.DENSE, D=b["D"]))
        else:
            blocks.append(ohm.Block(b["row0"], b["nrows"], b["col0"], b["ncols"], ohm.LOWRANK, W=b["W"], S=b["S"],
                                    X=b["X"]))
    return ohm.compress(ohm.HMatrix(Hh.n, Hh.perm, blocks, eps))


def _check_rows(y, ref, absr, acc):
    rel = np.linalg.norm(y - ref) / np.linalg.norm(ref)
    comp = np.max(np.abs(y - ref) / absr)
    assert rel <= TOL[acc], (acc, rel)
    assert comp <= 10 * TOL[acc], (acc, comp)
    return rel, comp


def _products(A, x):
    n = x.size
    xd = torch.from_numpy(x).cuda()
    out = {}
    for acc in ("fp32", "fp64"):
        yd = torch.zeros(n, dtype=torch.float64, device="cuda")
        A.matvec(xd, yd, acc=acc)
        A.check()
        out[acc] = yd.cpu().numpy()
    return out


@pytest.mark.parametrize("eps", [1e-6, 1e-8])
def test_benchmarked_matrix_units_and_rows(eps):
    n = 262144
    p = synth.laplace_problem(n)
    Hh = hg.build_kernel_hmatrix(p.points, "laplace", eps, diag=p.params["diag"], eta=2.0, leaf_size=64)
    A = Hh.upload("afl", decode_map=True)
    try:
        rng = np.random.default_rng(11)
        # ---- decoded units, bit for bit
        off, prec = Hh.unit_offsets("afl")
        st = Hh.structure()
        nunits_blk = np.where(st[:, 4] == hg.HLR_DENSE, 1, 2 * st[:, 5])
        first = np.concatenate([[0], np.cumsum(nunits_blk)[:-1]])
        dec = torch.empty(int(off[-1]), dtype=torch.float64, device="cuda")
        A.decode_units(dec)
        torch.cuda.synchronize()
        order = rng.permutation(st.shape[0])
        checked = 0
        for i in order:
            if nunits_blk[i] == 0:
                continue
            b = Hh.block(int(i))
            if b["kind"] == hg.HLR_DENSE:
                vals = [b["D"].ravel(order="F")]
            else:
                vals = [b["W"][:, k] for k in range(b["S"].size)] + [b["X"][:, k] for k in range(b["S"].size)]
            for k, a in enumerate(vals):
                u = first[i] + k
                want = afl.decode(afl.encode(np.ascontiguousarray(a), float(prec[u])))
                got = dec[int(off[u]):int(off[u + 1])].cpu().numpy()
                assert np.array_equal(got.view(np.int64), want.view(np.int64)), (int(i), k)
            checked += len(vals)
            if checked >= 2000:
                break
        assert checked >= 2000
        del dec
        torch.cuda.empty_cache()
        # ---- products on >= 512 rows of seeded leaf clusters
        rows, cover = _leaf_rows(Hh, rng, 512)
        assert rows.size >= 512
        C = _oracle_blocks(Hh, cover, eps)
        x = synth.rhs(n, 1)
        ref = omv.rows_exact(C, x, rows)
        absr = omv.abs_rows(C, x, rows)
        ys = _products(A, x)
        for acc in ("fp32", "fp64"):
            _check_rows(ys[acc][rows], ref, absr, acc)
    finally:
        A.free()
        Hh.free()


@pytest.mark.slow
def test_scale_matrix_rows():
    """n = 2^21 (the scale workload): all rows of seeded leaf clusters (>= 192 rows) against the
    oracle."""
    n = 2 ** 21
    eps = 1e-6
    p = synth.laplace_problem(n)
    Hh = hg.build_kernel_hmatrix(p.points, "laplace", eps, diag=p.params["diag"], eta=2.0, leaf_size=64)
    A = Hh.upload("afl")
    try:
        rows, cover = _leaf_rows(Hh, np.random.default_rng(12), 192)
        C = _oracle_blocks(Hh, cover, eps)
        x = synth.rhs(n, 1)
        ref = omv.rows_exact(C, x, rows)
        absr = omv.abs_rows(C, x, rows)
        ys = _products(A, x)
        for acc in ("fp32", "fp64"):
            _check_rows(ys[acc][rows], ref, absr, acc)
    finally:
        A.free()
        Hh.free()
