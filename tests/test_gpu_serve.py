"""Serving loop on the GPU: Poisson arrivals of products and CG solves against three resident
matrices under a budget that holds only two of them. Every product matches the oracle's decoded
matrix (Section 5.4), every solve reaches a true relative residual of 1e-8, and every request
gives the same bits alone as in the mix."""
import numpy as np
import pytest

import synth
from oracle import hmatrix as ohm
from tests._util import oracle_blocks

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
hg = pytest.importorskip("paper_2308_10960_gb300")
from paper_2308_10960_gb300 import serve  # noqa: E402


class OracleBuilt:
    """An oracle-built H-matrix with the ``upload(fmt, stream=...)`` face of HostHMatrix."""

    def __init__(self, H):
        self.H = H

    def upload(self, fmt="afl", stream=None):
        return hg.upload(self.H.n, self.H.perm, oracle_blocks(self.H), self.H.eps, fmt=fmt, stream=stream)


@pytest.fixture(scope="module")
def setup(exp2d_case, matern_small_case):
    p3 = synth.matern_problem(2500, seed=102)
    H3 = ohm.build_hmatrix(p3, 1e-6, method="aca")
    C3 = ohm.compress(H3)
    cases = {"exp2d": exp2d_case[1:], "matern": matern_small_case[1:], "matern2": (H3, C3)}
    host = {k: OracleBuilt(H) for k, (H, C) in cases.items()}
    dense = {k: ohm.to_dense(C) for k, (H, C) in cases.items()}
    return host, dense


def _requests(host, dense, count, seed):
    g = np.random.default_rng(seed)
    names = sorted(host)
    arr = serve.poisson_arrivals(count, 400.0, seed)
    reqs = []
    for i in range(count):
        m = names[i % len(names)] if i < 6 else names[g.integers(len(names))]
        kind = "solve" if (i % 7 == 3) else "matvec"
        x = torch.from_numpy(g.standard_normal(dense[m].shape[0])).cuda()
        reqs.append(serve.Request(i, kind, m, x, arrival=arr[i], rtol=1e-8, maxit=20000))
    return reqs


def test_serving_mix_matches_oracle_and_alone(setup):
    host, dense = setup
    be = serve.GpuBackend(host)
    sizes = sorted(be.device_bytes(m) for m in host)
    budget = sizes[-1] + sizes[-2]              # two of the three fit
    reqs = _requests(host, dense, 42, 11)
    st = serve.Server(be, budget_bytes=budget, cg_workers=2, max_rhs=32).run(reqs)
    assert st.failed == 0 and st.completed == len(reqs)
    assert st.peak_resident_bytes <= budget and st.evictions > 0
    assert st.latency["matvec"]["p99"] >= st.latency["matvec"]["p50"] > 0
    for r in reqs:
        A = dense[r.matrix]
        x = r.x.cpu().numpy()
        y = r.y.cpu().numpy()
        if r.kind == "matvec":
            ref = A @ x
            assert np.linalg.norm(y - ref) / np.linalg.norm(ref) <= 1e-6
            assert np.max(np.abs(y - ref) / (np.abs(A) @ np.abs(x))) <= 1e-5
        else:
            assert np.linalg.norm(x - A @ y) / np.linalg.norm(x) <= 1.5e-8, r.rid
    # each request alone, through the same backend and kernels
    for r in reqs:
        alone = serve.Request(0, r.kind, r.matrix, r.x, rtol=r.rtol, maxit=r.maxit)
        serve.Server(be, budget_bytes=budget).run([alone], realtime=False)
        assert torch.equal(alone.y, r.y), (r.rid, r.kind)
    be.close()
