"""CG on the compressed operator (hlr_solve_cg) against the oracle: the returned x has a true
residual ||b - A~ x|| / ||b|| <= 1e-8 computed by the ORACLE product, and agrees with the
direct solution of A~ x = b within the conditioning bound."""
import numpy as np
import pytest

import synth
from oracle import hmatrix as ohm
from oracle import matvec as omv
from tests._util import oracle_blocks

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
hg = pytest.importorskip("paper_2308_10960_gb300")


def test_cg_true_residual_and_solution():
    p = synth.matern_problem(2000, seed=100)
    H = ohm.build_hmatrix(p, 1e-6, method="aca")
    C = ohm.compress(H)
    A = hg.upload(p.n, H.perm, oracle_blocks(H), 1e-6)
    b = synth.rhs(p.n, 9)
    bd = torch.from_numpy(b).cuda()
    xd = torch.zeros(p.n, dtype=torch.float64, device="cuda")
    it, rel = A.solve_cg(bd, xd, rtol=1e-8, maxit=2000, acc="fp64")
    x = xd.cpu().numpy()
    r = b - omv.matvec(C, x)
    assert np.linalg.norm(r) / np.linalg.norm(b) <= 1.5e-8
    assert abs(rel - np.linalg.norm(r) / np.linalg.norm(b)) <= 1e-10
    At = ohm.to_dense(C)
    xs = np.linalg.solve(At, b)
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) <= np.linalg.cond(At) * 2e-8
    assert it > 0
    A.free()


def test_cg_noconv_reports_last_iterate():
    p = synth.matern_problem(1500, seed=101)
    H = ohm.build_hmatrix(p, 1e-6, method="aca")
    A = hg.upload(p.n, H.perm, oracle_blocks(H), 1e-6)
    bd = torch.from_numpy(synth.rhs(p.n, 9)).cuda()
    xd = torch.zeros(p.n, dtype=torch.float64, device="cuda")
    with pytest.raises(hg.HlrError) as ei:
        A.solve_cg(bd, xd, rtol=1e-14, maxit=3, acc="fp64")
    assert ei.value.code == -5
    assert torch.count_nonzero(xd).item() > 0
    A.free()


@pytest.mark.parametrize("n,seed", [(2000, 100), (3000, 103)])
def test_cg_fp32_refinement_reaches_true_residual(n, seed):
    """FP32-accumulation products inside CG, FP64 true residual between corrections: the
    returned x meets rtol on the TRUE residual (computed here from the oracle's decoded
    matrix) and agrees with the FP64-product CG solution."""
    p = synth.matern_problem(n, seed=seed)
    H = ohm.build_hmatrix(p, 1e-6, method="aca")
    C = ohm.compress(H)
    A = hg.upload(p.n, H.perm, oracle_blocks(H), 1e-6)
    b = synth.rhs(p.n, 9)
    bd = torch.from_numpy(b).cuda()
    x32 = torch.zeros(p.n, dtype=torch.float64, device="cuda")
    it32, rel32 = A.solve_cg(bd, x32, rtol=1e-8, maxit=20000, acc="fp32")
    x64 = torch.zeros(p.n, dtype=torch.float64, device="cuda")
    it64, rel64 = A.solve_cg(bd, x64, rtol=1e-8, maxit=20000, acc="fp64")
    At = ohm.to_dense(C)
    x = x32.cpu().numpy()
    true = np.linalg.norm(b - At @ x) / np.linalg.norm(b)
    assert true <= 1.5e-8 and rel32 <= 1e-8 and abs(rel32 - true) <= 1e-10
    xs = x64.cpu().numpy()
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) <= np.linalg.cond(At) * 4e-8
    assert it32 > 0 and it64 > 0
    A.free()
