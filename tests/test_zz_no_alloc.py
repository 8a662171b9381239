"""hlr_decode_units_static (decoding without any device allocation) against hlr_decode_units.

Two calls in a row on different matrices (so the second call overwrites the shared static map
of the first), each compared bit for bit with the allocating entry point; a matrix whose map
does not fit the static array is rejected with HLR_ERR_UNSUPPORTED. This file is collected last
and also passes on its own in a fresh process.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
hg = pytest.importorskip("paper_2308_10960_gb300")
from paper_2308_10960_gb300 import _binding as B  # noqa: E402


def _matrix(n, fmt):
    p = synth.laplace_problem(n)
    H = hg.build_kernel_hmatrix(p.points, "laplace", 1e-6, diag=p.params["diag"])
    A = H.upload(fmt=fmt)
    H.free()
    return A


def _decode_both(A):
    v = A.info["values"]
    ref = torch.full((v,), float("nan"), dtype=torch.float64, device="cuda")
    A.decode_units(ref)
    got = torch.full((v,), float("nan"), dtype=torch.float64, device="cuda")
    A.decode_units_static(got)
    torch.cuda.synchronize()
    return ref.cpu().numpy(), got.cpu().numpy()


def test_static_decode_two_calls_match_allocating_decode():
    mats = [_matrix(2048, "afl"), _matrix(2048, "fp64")]
    try:
        for A in mats:
            ref, got = _decode_both(A)
            assert ref.size == A.info["values"] > 0
            assert np.array_equal(got.view(np.int64), ref.view(np.int64))
        # the first matrix again, after the second one's map has replaced its own
        ref, got = _decode_both(mats[0])
        assert np.array_equal(got.view(np.int64), ref.view(np.int64))
    finally:
        for A in mats:
            A.free()


def test_static_decode_rejects_oversized_map_and_small_output():
    A = _matrix(16384, "afl")
    try:
        out = torch.empty(A.info["values"], dtype=torch.float64, device="cuda")
        with pytest.raises(B.HlrError) as ei:
            A.decode_units_static(out)
        assert ei.value.code == B.HLR_ERR_UNSUPPORTED and "static scratch" in str(ei.value)
        small = torch.empty(8, dtype=torch.float64, device="cuda")
        with pytest.raises(B.HlrError) as ei:
            A.decode_units_static(small)
        assert ei.value.code == B.HLR_ERR_INVALID
    finally:
        A.free()
