"""Products of different matrices running at the same time on one GPU (different streams, as in
the serving loop) give the same bits as each product alone, and concurrent CG solves the same
iterates. Regression test of the ring-slot hand-back: the consumers read a slot with ordinary
shared loads and the next TMA copy writes it through the async proxy, so each lane fences
before its warp releases the slot (without it, products that shared SMs with another kernel
occasionally decoded the next piece into the first rows of a leaf)."""
import threading

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
hg = pytest.importorskip("paper_2308_10960_gb300")


@pytest.fixture(scope="module")
def mats():
    out = []
    for i, n in enumerate((28526, 37641)):
        p = synth.matern_problem(n, seed=202 + i)
        H = hg.build_kernel_hmatrix(p.points, "matern15", 1e-6, scale=p.params["scale"], diag=p.params["diag"])
        out.append((H, H.upload("afl")))
    yield out
    for H, A in out:
        A.free()
        H.free()


def _run_threads(fn, k):
    errs = {}
    th = [threading.Thread(target=fn, args=(i, errs)) for i in range(k)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    return errs


@pytest.mark.parametrize("acc", ["fp32", "fp64"])
def test_concurrent_products_match_alone(mats, acc):
    refs = []
    for k, (H, A) in enumerate(mats):
        x = torch.from_numpy(synth.rhs(H.n, 11 + k)).cuda()
        y = torch.zeros(H.n, dtype=torch.float64, device="cuda")
        A.matvec(x, y, acc=acc)
        torch.cuda.synchronize()
        refs.append((x, y.cpu().numpy().view(np.int64)))

    def work(k, errs):
        H, A = mats[k]
        x, ref = refs[k]
        s = torch.cuda.Stream()
        bad = 0
        with torch.cuda.stream(s):
            for _ in range(150):
                y = torch.zeros(H.n, dtype=torch.float64, device="cuda")
                A.matvec(x, y, acc=acc, stream=s)
                s.synchronize()
                bad += int(not np.array_equal(y.cpu().numpy().view(np.int64), ref))
        errs[k] = bad

    errs = _run_threads(work, 2)
    assert errs == {0: 0, 1: 0}


def test_concurrent_solves_match_alone(mats):
    alone = []
    bs = []
    for k, (H, A) in enumerate(mats):
        b = torch.from_numpy(synth.rhs(H.n, 7000 + k)).cuda()
        x = torch.zeros(H.n, dtype=torch.float64, device="cuda")
        alone.append((A.solve_cg(b, x, rtol=1e-8, maxit=20000, acc="fp32"), x.cpu().numpy().view(np.int64)))
        bs.append(b)

    def work(k, res):
        H, A = mats[k]
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            x = torch.zeros(H.n, dtype=torch.float64, device="cuda")
            r = A.solve_cg(bs[k], x, rtol=1e-8, maxit=20000, acc="fp32", stream=s, sm_share=4)
        s.synchronize()
        res[k] = (r, x.cpu().numpy().view(np.int64))

    res = _run_threads(work, 2)
    for k in range(2):
        assert res[k][0] == alone[k][0] and res[k][0][1] <= 1e-8
        assert np.array_equal(res[k][1], alone[k][1])
