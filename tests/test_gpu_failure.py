"""Failure detection on the GPU without a fault: the product kernels never wait without a limit;
a wait that gives up is recorded in the handle's status word and reported by hlr_check as
HLR_ERR_TIMEOUT. hlr_selftest_wait runs that very bounded wait on a barrier that nothing
completes, with a short limit, so the failure path is exercised while the context, the handle
and its data stay usable."""
import numpy as np
import pytest

import synth
from oracle import hmatrix as ohm
from tests._util import oracle_blocks

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
hg = pytest.importorskip("paper_2308_10960_gb300")
from paper_2308_10960_gb300 import _binding as B  # noqa: E402


def _matrix():
    p = synth.exp2d_problem(1024, seed=0)
    H = ohm.build_hmatrix(p, 1e-6, leaf_size=64, eta=2.0, method="svd")
    return p, H


def test_expired_wait_is_reported_once_and_leaves_the_handle_usable():
    p, H = _matrix()
    A = hg.upload(p.n, H.perm, oracle_blocks(H), 1e-6)
    try:
        x = torch.from_numpy(synth.rhs(p.n, 1)).cuda()
        y0 = torch.zeros(p.n, dtype=torch.float64, device="cuda")
        A.matvec(x, y0, acc="fp32")
        A.check()                                  # a normal product reports nothing
        ref = y0.cpu().numpy()
        for cycles in (20_000, 2_000_000):         # ~10 us and ~1 ms at the SM clock
            A.selftest_wait(cycles)
            with pytest.raises(hg.HlrError) as ei:
                A.check()
            assert ei.value.code == B.HLR_ERR_TIMEOUT
            A.check()                              # the check cleared the status word
        y1 = torch.zeros(p.n, dtype=torch.float64, device="cuda")
        A.matvec(x, y1, acc="fp32")
        A.check()
        assert np.array_equal(y1.cpu().numpy().view(np.int64), ref.view(np.int64))
        with pytest.raises(hg.HlrError):
            A.selftest_wait(10)                    # below the accepted range
    finally:
        A.free()
