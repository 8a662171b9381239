"""Full-size checks at the benchmark workload (n = 262144 sphere, eps = 1e-6, the launch
configuration bench.py times), where the oracle cannot build the whole matrix:

* sampled rows of y against direct kernel evaluation by the oracle (A x by its plain
  definition): |y_i - (A x)_i| <= C eps sum_j |A_ij x_j| on 256 seeded rows, C = 30;
* FP32 in-block vs FP64 accumulation on the same stored matrix: relative 1e-6;
* plain FP64 storage vs compressed (FP64 accumulation): within C eps;
* determinism of the FP32 path.
"""
import numpy as np
import pytest

import synth
from oracle import matvec as omv

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
hg = pytest.importorskip("paper_2308_10960_gb300")

N = 262144
EPS = 1e-6


@pytest.fixture(scope="module")
def big():
    p = synth.laplace_problem(N)
    Hh = hg.build_kernel_hmatrix(p.points, "laplace", EPS, diag=p.params["diag"])
    A = Hh.upload("afl")
    Ap = Hh.upload("fp64")
    yield p, A, Ap
    A.free()
    Ap.free()
    Hh.free()


def _abs_rows(p, x, rows):
    allj = np.arange(p.n)
    return np.array([np.sum(np.abs(p.entries(np.array([i]), allj)[0]) * np.abs(x)) for i in rows])


def test_sampled_rows_against_dense_kernel(big):
    p, A, Ap = big
    x = synth.rhs(N, 1)
    xd = torch.from_numpy(x).cuda()
    rows = np.sort(np.random.default_rng(6).choice(N, size=256, replace=False))
    ref = omv.dense_rows(p, x, rows)
    absr = _abs_rows(p, x, rows)
    for M, acc in ((A, "fp32"), (A, "fp64"), (Ap, "fp64")):
        yd = torch.zeros(N, dtype=torch.float64, device="cuda")
        M.matvec(xd, yd, acc=acc)
        y = yd.cpu().numpy()
        err = np.abs(y[rows] - ref) / absr
        assert err.max() <= 30 * EPS, (acc, err.max())
        assert np.linalg.norm(y[rows] - ref) / np.linalg.norm(ref) <= 30 * EPS


def test_fp32_vs_fp64_and_plain(big):
    p, A, Ap = big
    x = torch.from_numpy(synth.rhs(N, 1)).cuda()
    out = {}
    for name, M, acc in (("fp32", A, "fp32"), ("fp64", A, "fp64"), ("plain", Ap, "fp64")):
        y = torch.zeros(N, dtype=torch.float64, device="cuda")
        M.matvec(x, y, acc=acc)
        out[name] = y.cpu().numpy()
    r = lambda a, b: np.linalg.norm(a - b) / np.linalg.norm(b)
    assert r(out["fp32"], out["fp64"]) <= 1e-6
    assert r(out["fp64"], out["plain"]) <= 30 * EPS
    y2 = torch.zeros(N, dtype=torch.float64, device="cuda")
    A.matvec(x, y2, acc="fp32")
    assert np.array_equal(y2.cpu().numpy().view(np.int64), out["fp32"].view(np.int64))
