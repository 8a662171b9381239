"""HLR_SM_SHARE: the persistent product kernels on a share of their CTA slots (each CTA walking
the work lists of several slots) give the same bits as on all of them, for single products,
batched multi-right-hand-side products and CG solves (the serving loop runs solves on a share
so that products keep the rest of every SM)."""
import numpy as np
import pytest

import synth
from oracle import hmatrix as ohm
from tests._util import oracle_blocks

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
hg = pytest.importorskip("paper_2308_10960_gb300")


@pytest.fixture(scope="module")
def mat():
    p = synth.matern_problem(3000, seed=100)
    H = ohm.build_hmatrix(p, 1e-6, leaf_size=64, eta=2.0, method="aca")
    A = hg.upload(p.n, H.perm, oracle_blocks(H), 1e-6)
    yield p, A
    A.free()


def _bits(t):
    return t.cpu().numpy().view(np.int64)


def test_products_same_bits_on_a_share(mat):
    p, A = mat
    x = torch.from_numpy(synth.rhs(p.n, 1)).cuda()
    for acc in ("fp32", "fp64"):
        ref = torch.zeros(p.n, dtype=torch.float64, device="cuda")
        A.matvec(x, ref, acc=acc)
        for share in (1, 3, 7):
            y = torch.zeros(p.n, dtype=torch.float64, device="cuda")
            A.matvec(x, y, acc=acc, sm_share=share)
            A.check()
            assert np.array_equal(_bits(y), _bits(ref)), (acc, share)
    X = torch.from_numpy(synth.rhs(p.n * 11, 5)).cuda().view(11, p.n)
    Y0 = torch.zeros_like(X)
    hg.matvec_batched([A], [X], [Y0])
    Y1 = torch.zeros_like(X)
    hg.matvec_batched([A], [X], [Y1], sm_share=2)
    assert np.array_equal(_bits(Y1), _bits(Y0))
    with pytest.raises(hg.HlrError):
        A.matvec(x, ref, sm_share=9)


def test_cg_same_solution_on_a_share(mat):
    p, A = mat
    b = torch.from_numpy(synth.rhs(p.n, 8)).cuda()
    for acc in ("fp64", "fp32"):
        x0 = torch.zeros(p.n, dtype=torch.float64, device="cuda")
        it0, rel0 = A.solve_cg(b, x0, rtol=1e-8, maxit=5000, acc=acc)
        x1 = torch.zeros(p.n, dtype=torch.float64, device="cuda")
        it1, rel1 = A.solve_cg(b, x1, rtol=1e-8, maxit=5000, acc=acc, sm_share=4)
        assert rel0 <= 1e-8 and (it1, rel1) == (it0, rel0)
        assert np.array_equal(_bits(x1), _bits(x0))
