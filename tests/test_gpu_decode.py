"""GPU decoding is bit-exact with the oracle decoder (Section 3.2).

Streams are produced by the ORACLE encoder and decoded on the GPU by hlr_afl_decode_device;
whole uploaded H-matrices are decoded by hlr_decode_units and compared, unit by unit, with the
oracle's decoding of its own compression of the same FP64 H-matrix.
"""
import numpy as np
import pytest

import synth
from oracle import afl
from oracle import hmatrix as ohm
from tests._util import oracle_blocks

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
hg = pytest.importorskip("paper_2308_10960_gb300")


def _gpu_decode(unit):
    data = np.frombuffer(unit.data, dtype=np.uint8)
    buf = torch.zeros(max(16, data.size + 16), dtype=torch.uint8, device="cuda")
    if data.size:
        buf[: data.size] = torch.from_numpy(data.copy()).cuda()
    out = torch.full((max(unit.n, 1),), np.nan, dtype=torch.float64, device="cuda")
    hg.afl_decode_device(buf, unit.n, unit.m_min, unit.e, unit.m, out)
    torch.cuda.synchronize()
    return out[: unit.n].cpu().numpy()


def _cases():
    g = np.random.default_rng(99)
    yield g.standard_normal(1)
    yield g.standard_normal(1000)
    yield np.exp(g.uniform(-300, 300, size=257)) * g.choice([-1.0, 1.0], size=257)
    z = g.standard_normal(333)
    z[::4] = 0.0
    yield z
    yield np.zeros(40)
    yield np.array([1.0, 2.0 - 2.0 ** -40, -(4.0 - 2.0 ** -30), 7.999999])


@pytest.mark.parametrize("m", [0, 1, 2, 7, 10, 19, 20, 23, 24, 27, 31, 40, 47, 51, 52])
def test_decode_stream_bit_exact(m):
    u = 1.0 if m == 0 else 2.0 ** -m
    for a in _cases():
        unit = afl.encode(a, u)
        ref = afl.decode(unit)
        got = _gpu_decode(unit)
        assert np.array_equal(got.view(np.int64), ref.view(np.int64)), (m, unit.e, unit.w)


@pytest.mark.parametrize("case", ["exp2d", "matern"])
def test_decode_units_bit_exact(case, exp2d_case, matern_small_case):
    p, H, C = exp2d_case if case == "exp2d" else matern_small_case
    A = hg.upload(p.n, H.perm, oracle_blocks(H), H.eps)
    out = torch.empty(A.info["values"], dtype=torch.float64, device="cuda")
    A.decode_units(out)
    got = out.cpu().numpy()
    ref = np.concatenate([afl.decode(u) for cb in C.blocks for u in cb.units])
    assert got.size == ref.size
    assert np.array_equal(got.view(np.int64), ref.view(np.int64))
    A.free()
