"""The GPU encoder hlr_encode_device (Section 3.2 per unit, Section 3.3 for the APLR precisions
and the MP layout) against the oracle's encoder: every unit of a compressed H-matrix, in every
compressed format, byte for byte, plus the parameters; rejected units (NaN, values beyond the
format, bad precisions) are marked and get no stream; empty and all-zero units."""
import numpy as np
import pytest

from oracle import afl
from oracle import hmatrix as ohm
from tests._util import oracle_blocks

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
hg = pytest.importorskip("paper_2308_10960_gb300")

FMTS = ["afl", "aflp", "bfl", "dfl", "mp"]


def _run(vals, off, prec, fmt):
    v = torch.from_numpy(np.ascontiguousarray(vals, dtype=np.float64)).cuda()
    o = torch.from_numpy(np.ascontiguousarray(off, dtype=np.int64)).cuda()
    u = torch.from_numpy(np.ascontiguousarray(prec, dtype=np.float64)).cuda()
    mm, e, m, oo, out = hg.encode_device(v, o, u, fmt)
    torch.cuda.synchronize()
    return mm.cpu().numpy(), e.cpu().numpy(), m.cpu().numpy(), oo.cpu().numpy(), out.cpu().numpy()


def _check_units(vals, off, prec, fmt, oracle_units):
    mm, e, m, oo, out = _run(vals, off, prec, fmt)
    for k, ref in enumerate(oracle_units):
        if ref is None:
            assert e[k] == -1 and oo[k + 1] == oo[k], (fmt, k)
            continue
        assert (e[k], m[k]) == (ref.e, ref.m) and mm[k] == ref.m_min, (fmt, k)
        assert out[oo[k]:oo[k + 1]].tobytes() == ref.data, (fmt, k)
    assert oo[-1] == sum(len(r.data) for r in oracle_units if r is not None)


@pytest.mark.parametrize("fmt", FMTS)
def test_encode_device_matches_oracle_units(fmt, exp2d_case):
    p, H, _ = exp2d_case
    C = ohm.compress(H, fmt=fmt)
    ref = [u for cb in C.blocks for u in cb.units]
    vals, off, prec = hg.unit_arrays(oracle_blocks(H), H.eps, fmt)
    assert len(ref) == prec.size
    _check_units(vals, off, prec, fmt, ref)


@pytest.mark.parametrize("fmt", FMTS)
def test_encode_device_edge_units(fmt):
    g = np.random.default_rng(31)
    t = 2.0 ** -11
    units = [
        (np.zeros(0), 1e-6),                                  # empty
        (np.zeros(37), 1e-6),                                 # all zero
        (np.array([0.0, -0.0, 1.0 + t, 1.0 + 3 * t, 2.0 ** -25, 65504.0, -65519.99, 1e-30]), 0.25),
        (g.standard_normal(1000) * np.exp(g.uniform(-30, 30, 1000)), 1e-9),
        (g.standard_normal(1) * 3.0, 0.9),                    # one value, m = 0 or 1
        (g.standard_normal(4097), 2.0 ** -24),
        (np.array([1.0, np.nan, 2.0]), 1e-6),                 # rejected: NaN
        (np.array([1.0, 2.0]), 0.0),                          # rejected: precision not positive
        (g.standard_normal(300) * 1e-3, 2.0 ** -11),
        (np.array([1e300, -1e300, 1e-300]), 1e-6),           # beyond FP32 / FP16 for BFL and MP16
    ]
    vals = np.concatenate([a for a, _ in units])
    off = np.zeros(len(units) + 1, dtype=np.int64)
    np.cumsum([a.size for a, _ in units], out=off[1:])
    prec = np.array([u for _, u in units])
    ref = []
    for a, u in units:
        try:
            ref.append(afl.encode(a, u, fmt) if u > 0 else None)
        except ValueError:
            ref.append(None)
    _check_units(vals, off, prec, fmt, ref)


def test_encode_device_graph_capture(exp2d_case):
    p, H, _ = exp2d_case
    vals, off, prec = hg.unit_arrays(oracle_blocks(H)[:200], H.eps)
    v = torch.from_numpy(vals).cuda()
    o = torch.from_numpy(off).cuda()
    u = torch.from_numpy(prec).cuda()
    eager = hg.encode_device(v, o, u)
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        cap = hg.encode_device(v, o, u, stream=s)
    g.replay()
    torch.cuda.synchronize()
    n = int(eager[3][-1])
    assert torch.equal(eager[4][:n], cap[4][:n]) and torch.equal(eager[3], cap[3])


@pytest.mark.parametrize("fmt", ["afl", "aflp"])
def test_encode_device_rounding_boundaries(fmt):
    """Values whose scaled magnitude |a| / m_min + 1 lies at or within a few ulps of the half-way
    point of the m-bit rounding (Section 3.2), for every m from 0 to 52, plus random values:
    the GPU quotient must round exactly like the IEEE division of the host encoder."""
    g = np.random.default_rng(41)
    units, precs = [], []
    for m in range(0, 53):
        u = 2.0 ** -m
        for m_min in (3.0, 0.7, 1.0 / 3.0, 5e-200, 7e150):
            k = g.integers(0, 2 ** min(m, 40), 200).astype(np.float64)
            v = (1.0 + (2.0 * k + 1.0) * 2.0 ** -(m + 1)) * 2.0 ** g.integers(1, 12, k.size)  # half-way at m bits
            v = v * (1.0 + g.integers(-6, 7, k.size) * 2.0 ** -52)                      # and a few ulps off
            t = v - 1.0
            a = np.concatenate([[m_min], m_min * t, -m_min * t[::3]])
            a = a[np.isfinite(a)]
            units.append(a)
            precs.append(u)
        units.append(g.standard_normal(777) * np.exp(g.uniform(-8, 8, 777)))
        precs.append(u)
    vals = np.concatenate(units)
    off = np.zeros(len(units) + 1, dtype=np.int64)
    np.cumsum([x.size for x in units], out=off[1:])
    ref = [afl.encode(x, p, fmt) for x, p in zip(units, precs)]
    _check_units(vals, off, np.array(precs), fmt, ref)


@pytest.mark.parametrize("fmt", FMTS)
def test_upload_with_device_encoding_is_the_same_matrix(fmt, exp2d_case):
    """HLR_ENCODE_DEVICE (compression on the GPU during the upload, Section 5.3) gives the
    matrix the host encoder gives: the same decoded values and the same products, bit for bit,
    and the same stored byte counts."""
    p, H, C = exp2d_case
    A = hg.upload(p.n, H.perm, oracle_blocks(H), H.eps, fmt=fmt)
    D = hg.upload(p.n, H.perm, oracle_blocks(H), H.eps, fmt=fmt, tuning=hg.HLR_ENCODE_DEVICE)
    try:
        for k in ("stream_bytes", "header_bytes", "algorithmic_bytes", "nunits", "values"):
            assert A.info[k] == D.info[k], k
        da = torch.empty(A.info["values"], dtype=torch.float64, device="cuda")
        dd = torch.empty_like(da)
        A.decode_units(da)
        D.decode_units(dd)
        assert torch.equal(da.view(torch.int64), dd.view(torch.int64))
        x = torch.from_numpy(np.random.default_rng(5).standard_normal(p.n)).cuda()
        for acc in ("fp32", "fp64"):
            ya = torch.zeros(p.n, dtype=torch.float64, device="cuda")
            yd = torch.zeros_like(ya)
            A.matvec(x, ya, acc=acc)
            D.matvec(x, yd, acc=acc)
            A.check()
            D.check()
            assert torch.equal(ya.view(torch.int64), yd.view(torch.int64)), acc
    finally:
        A.free()
        D.free()


def test_upload_with_device_encoding_rejects_non_finite():
    bl = [{"row0": 0, "nrows": 4, "col0": 0, "ncols": 4, "kind": hg.HLR_DENSE,
           "D": np.array([[1.0, 2.0, np.nan, 3.0]] * 4)}]
    with pytest.raises(hg.HlrError, match="NaN or Inf"):
        hg.upload(4, None, bl, 1e-6, tuning=hg.HLR_ENCODE_DEVICE)
