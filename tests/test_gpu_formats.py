"""The byte-aligned AFL variants on the GPU (Section 3.2): AFLP, BFL, DFL, and the mixed precision
comparison format MP-D-S-H (Section 3.3). Units decode bit for bit like the oracle's decoder,
products match the oracle's product of the same compressed matrix (1e-6 with FP32 accumulation,
1e-12 with FP64), multi-column requests and CG work on them."""
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

FMTS = ["aflp", "bfl", "dfl", "mp"]


@pytest.mark.parametrize("fmt", FMTS)
@pytest.mark.parametrize("case", ["exp2d", "matern"])
def test_format_decode_and_product(fmt, case, exp2d_case, matern_small_case):
    p, H, _ = exp2d_case if case == "exp2d" else matern_small_case
    C = ohm.compress(H, fmt=fmt)
    A = hg.upload(p.n, H.perm, oracle_blocks(H), H.eps, fmt=fmt)
    try:
        out = torch.empty(A.info["values"], dtype=torch.float64, device="cuda")
        A.decode_units(out)
        ref = np.concatenate([afl.decode(u) for cb in C.blocks for u in cb.units])
        assert np.array_equal(out.cpu().numpy().view(np.int64), ref.view(np.int64))
        x = np.random.default_rng(5).standard_normal(p.n)
        y0 = np.random.default_rng(6).standard_normal(p.n)
        yref = omv.matvec(C, x, y0)
        for acc, tol in (("fp32", 1e-6), ("fp64", 1e-12)):
            yd = torch.from_numpy(y0.copy()).cuda()
            A.matvec(torch.from_numpy(x).cuda(), yd, acc=acc)
            A.check()
            got = yd.cpu().numpy()
            assert np.linalg.norm(got - yref) / np.linalg.norm(yref) <= tol, (fmt, acc)
    finally:
        A.free()


@pytest.mark.parametrize("fmt", ["bfl", "dfl", "mp"])
def test_format_multi_column_and_cg(fmt, matern_small_case):
    p, H, _ = matern_small_case
    C = ohm.compress(H, fmt=fmt)
    Ad = ohm.to_dense(C)
    A = hg.upload(p.n, H.perm, oracle_blocks(H), H.eps, fmt=fmt)
    try:
        X = np.random.default_rng(7).standard_normal((8, p.n))
        Yd = torch.zeros((8, p.n), dtype=torch.float64, device="cuda")
        hg.matvec_batched([A], [torch.from_numpy(X).cuda()], [Yd])
        A.check()
        Y = Yd.cpu().numpy()
        ref = (Ad @ X.T).T
        for j in range(8):
            assert np.linalg.norm(Y[j] - ref[j]) / np.linalg.norm(ref[j]) <= 1e-6
        b = synth.rhs(p.n, 9)
        xd = torch.zeros(p.n, dtype=torch.float64, device="cuda")
        it, rel = A.solve_cg(torch.from_numpy(b).cuda(), xd, rtol=1e-8, maxit=20000, acc="fp32")
        x = xd.cpu().numpy()
        assert np.linalg.norm(b - Ad @ x) / np.linalg.norm(b) <= 1.5e-8 and rel <= 1e-8
    finally:
        A.free()


def test_mp_all_three_precisions():
    """MP at eps = 1e-9: lowrank columns in FP16, FP32 and FP64 (dense leaves FP64) in one matrix;
    the per-lane decode picks the IEEE layout from the lane's exponent width."""
    p = synth.exp2d_problem(2048, seed=3)
    H = ohm.build_hmatrix(p, 1e-9, leaf_size=64, eta=2.0, method="svd")
    C = ohm.compress(H, fmt="mp")
    kinds = {u.fmt for b in C.blocks if b.kind == ohm.LOWRANK for u in b.units}
    assert kinds == {"mp16", "mp32", "mp64"}
    A = hg.upload(p.n, H.perm, oracle_blocks(H), H.eps, fmt="mp")
    try:
        out = torch.empty(A.info["values"], dtype=torch.float64, device="cuda")
        A.decode_units(out)
        ref = np.concatenate([afl.decode(u) for cb in C.blocks for u in cb.units])
        assert np.array_equal(out.cpu().numpy().view(np.int64), ref.view(np.int64))
        x = np.random.default_rng(15).standard_normal(p.n)
        y0 = np.random.default_rng(16).standard_normal(p.n)
        yref = omv.matvec(C, x, y0)
        for acc, tol in (("fp32", 1e-6), ("fp64", 1e-12)):
            yd = torch.from_numpy(y0.copy()).cuda()
            A.matvec(torch.from_numpy(x).cuda(), yd, acc=acc)
            A.check()
            got = yd.cpu().numpy()
            assert np.linalg.norm(got - yref) / np.linalg.norm(yref) <= tol, acc
    finally:
        A.free()
