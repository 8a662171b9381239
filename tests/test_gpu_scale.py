"""The scale case: n = 2^21 Fibonacci points on the sphere, 1/(4 pi r) with the sampled mean row
sum on the diagonal, eps = 1e-6. Sampled rows of the single-column product (1024 rows,
default_rng(6)) and of three columns of a 32-column product (128 rows) against direct kernel
evaluation by the oracle: |y_i - (A x)_i| <= C eps sum_j |A_ij x_j|, C = 30, as for n = 262144."""
import numpy as np
import pytest

import synth
from oracle import matvec as omv

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
torch = pytest.importorskip("torch")
hg = pytest.importorskip("paper_2308_10960_gb300")

N = 2 ** 21
EPS = 1e-6


def _abs_rows(p, x, rows):
    allj = np.arange(p.n)
    return np.array([np.sum(np.abs(p.entries(np.array([i]), allj)[0]) * np.abs(x)) for i in rows])


def test_scale_sampled_rows():
    p = synth.laplace_problem(N)
    Hh = hg.build_kernel_hmatrix(p.points, "laplace", EPS, diag=p.params["diag"])
    A = Hh.upload("afl")
    Hh.free()
    try:
        x = synth.rhs(N, 1)
        yd = torch.zeros(N, dtype=torch.float64, device="cuda")
        A.matvec(torch.from_numpy(x).cuda(), yd, acc="fp32")
        A.check()
        y = yd.cpu().numpy()
        rows = np.sort(np.random.default_rng(6).choice(N, size=1024, replace=False))
        ref = omv.dense_rows(p, x, rows)
        err = np.abs(y[rows] - ref) / _abs_rows(p, x, rows)
        assert err.max() <= 30 * EPS, err.max()

        X = synth.rhs(N * 32, 3).reshape(32, N)
        Yd = torch.zeros((32, N), dtype=torch.float64, device="cuda")
        hg.matvec_batched([A], [torch.from_numpy(X).cuda()], [Yd])
        A.check()
        Y = Yd.cpu().numpy()
        rows = rows[::16]
        for j in (0, 13, 31):
            ref = omv.dense_rows(p, X[j], rows)
            err = np.abs(Y[j][rows] - ref) / _abs_rows(p, X[j], rows)
            assert err.max() <= 30 * EPS, (j, err.max())
    finally:
        A.free()
