"""Work-layout tunings of the AFL kernels (rows per lane, task rows, piece size, CTAs per SM)
give the same decoded values bit for bit and products within the FP32 tolerance of the oracle;
the autotuner picks one of its candidates."""
import numpy as np
import pytest

from oracle import afl
from oracle import matvec as omv
from tests._util import oracle_blocks

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
hg = pytest.importorskip("paper_2308_10960_gb300")
from paper_2308_10960_gb300 import tune  # noqa: E402

LAYOUTS = [(32, 64, 16), (128, 64, 16), (64, 32, 16), (32, 32, 4), (128, 32, 8), (64, 64, 16, 2), (32, 64, 16, 3)]


@pytest.mark.parametrize("layout", LAYOUTS)
def test_tuned_layouts_match_oracle(layout, matern_small_case):
    p, H, C = matern_small_case
    A = hg.upload(p.n, H.perm, oracle_blocks(H), H.eps, tuning=hg.tuning_code(*layout))
    try:
        out = torch.empty(A.info["values"], dtype=torch.float64, device="cuda")
        A.decode_units(out)
        ref = np.concatenate([afl.decode(u) for cb in C.blocks for u in cb.units])
        assert np.array_equal(out.cpu().numpy().view(np.int64), ref.view(np.int64))
        x = np.random.default_rng(3).standard_normal(p.n)
        y0 = np.random.default_rng(4).standard_normal(p.n)
        yref = omv.matvec(C, x, y0)
        for acc, tol in (("fp32", 1e-6), ("fp64", 1e-12)):
            yd = torch.from_numpy(y0.copy()).cuda()
            A.matvec(torch.from_numpy(x).cuda(), yd, acc=acc)
            A.check()
            got = yd.cpu().numpy()
            assert np.linalg.norm(got - yref) / np.linalg.norm(yref) <= tol, (layout, acc)
        if len(layout) == 4:
            # a launch shape with fewer CTAs per SM: the multi-column passes too (one wide pass)
            X = np.random.default_rng(5).standard_normal((12, p.n))
            Y = torch.zeros((12, p.n), dtype=torch.float64, device="cuda")
            hg.matvec_batched([A], [torch.from_numpy(X).cuda()], [Y], acc="fp32")
            A.check()
            got = Y.cpu().numpy()
            for j in (0, 7, 11):
                yj = omv.matvec(C, X[j])
                assert np.linalg.norm(got[j] - yj) / np.linalg.norm(yj) <= 1e-6, (layout, j)
    finally:
        A.free()


class _Host:
    def __init__(self, p, H):
        self.p, self.H = p, H

    def upload(self, fmt="afl", tuning=0, stream=None):
        return hg.upload(self.p.n, self.H.perm, oracle_blocks(self.H), self.H.eps, fmt=fmt, tuning=tuning,
                         stream=stream)


def test_autotuner_picks_a_candidate(exp2d_case):
    p, H, C = exp2d_case
    t = tune.Autotuner(candidates=[(64, 64, 16), (32, 64, 16), (64, 32, 8), (64, 64, 16, 3)], reps=5)
    for nrhs in (1, 8, 32):
        res = t.tune(_Host(p, H), nrhs=nrhs)
        assert res.best in t.candidates and set(res.ms) == set(t.candidates)
        assert all(v > 0 for v in res.ms.values())
        assert t.table[res.rank_class] == res.best
    # a second matrix of a known class takes the stored choice without timing
    code, rc, res = t.choose(_Host(p, H), nrhs=8)
    assert res is None and code == hg.tuning_code(*t.table[rc])
