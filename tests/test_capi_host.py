"""Host-side tests of the native library (no GPU): the shared library loads and exports every
symbol include/hlr.h declares; the host AFL encoder is byte-exact with the oracle encoder; the
native construction reproduces the oracle's cluster tree, block tree and ranks and meets Eq. 1;
upload rejects invalid descriptors before touching the GPU."""
import ctypes
import os

import numpy as np
import pytest

import synth
from oracle import afl
from oracle import hmatrix as ohm
from tests._util import header_symbols, oracle_blocks

hg = pytest.importorskip("paper_2308_10960_gb300")


def test_every_declared_symbol_is_exported():
    lib = ctypes.CDLL(hg.lib_path())
    names = header_symbols()
    assert len(names) >= 13
    for n in names:
        assert hasattr(lib, n), n
    from paper_2308_10960_gb300 import _binding
    assert sorted(s[0] for s in _binding.SIGNATURES) == names


def _enc_cases():
    g = np.random.default_rng(21)
    yield g.standard_normal(1)
    yield g.standard_normal(777)
    yield np.exp(g.uniform(-60, 60, size=333)) * g.choice([-1.0, 1.0], size=333)
    z = g.standard_normal(129)
    z[::3] = 0.0
    yield z
    yield np.zeros(17)
    yield np.array([1.0, 2.0 - 2.0 ** -40, -(4.0 - 2.0 ** -30), 7.999999, -0.0])


@pytest.mark.parametrize("m", list(range(0, 53, 1)))
def test_host_encoder_byte_exact_with_oracle(m):
    u = 1.0 if m == 0 else 2.0 ** -m * 1.3
    for a in _enc_cases():
        mm, e, mb, data = hg.afl_encode(a, u)
        o = afl.encode(a, u)
        assert (mm, e, mb) == (o.m_min, o.e, o.m)
        assert data == o.data


def test_host_encoder_precisions_like_aplr():
    g = np.random.default_rng(4)
    s = np.sort(np.exp(g.uniform(-12, 0, size=20)))[::-1]
    for ui in afl.aplr_precisions(s, 1e-6):
        a = g.standard_normal(64)
        assert hg.afl_encode(a, ui)[3] == afl.encode(a, ui).data


@pytest.mark.parametrize("name", ["exp2d", "laplace", "matern"])
def test_native_construction_matches_oracle(name):
    if name == "exp2d":
        p = synth.exp2d_problem(2048)
    elif name == "laplace":
        p = synth.laplace_problem(3000)
    else:
        p = synth.matern_problem(2500, 101)
    Hp = hg.build_kernel_hmatrix(p.points, p.kind, 1e-6, scale=p.params.get("scale", 1.0), diag=p.params["diag"])
    Ho = ohm.build_hmatrix(p, 1e-6, method="aca")
    assert np.array_equal(Hp.perm, Ho.perm)
    st = Hp.structure()
    so = np.array([(b.row0, b.nrows, b.col0, b.ncols, b.kind) for b in Ho.blocks])
    assert np.array_equal(st[:, :5], so)
    ro = np.array([b.rank for b in Ho.blocks])
    # ACA pivots may differ by rounding; ranks after recompression agree up to one
    assert np.max(np.abs(st[:, 5] - ro)) <= 1
    worst = 0.0
    for i in np.flatnonzero(st[:, 4] == 1):
        b = Hp.block(i)
        if b["S"].size == 0:
            continue
        M = p.entries(Hp.perm[b["row0"]:b["row0"] + b["nrows"]], Hp.perm[b["col0"]:b["col0"] + b["ncols"]])
        worst = max(worst, np.linalg.norm(M - (b["W"] * b["S"]) @ b["X"].T, 2) / np.linalg.norm(M, 2))
        assert np.allclose(b["W"].T @ b["W"], np.eye(b["S"].size), atol=1e-10)
    assert worst <= 3e-6
    for i in np.flatnonzero(st[:, 4] == 0)[:50]:
        b = Hp.block(i)
        M = p.entries(Hp.perm[b["row0"]:b["row0"] + b["nrows"]], Hp.perm[b["col0"]:b["col0"] + b["ncols"]])
        np.testing.assert_allclose(b["D"], M, rtol=1e-13, atol=0)


def _tiny_blocks():
    g = np.random.default_rng(0)
    D = lambda r, c: g.standard_normal((r, c))
    return [
        {"row0": 0, "nrows": 3, "col0": 0, "ncols": 3, "kind": 0, "D": D(3, 3)},
        {"row0": 0, "nrows": 3, "col0": 3, "ncols": 2, "kind": 0, "D": D(3, 2)},
        {"row0": 3, "nrows": 2, "col0": 0, "ncols": 5, "kind": 0, "D": D(2, 5)},
    ]


def test_upload_rejects_invalid_descriptors():
    bl = _tiny_blocks()
    bad_cover = [dict(b) for b in bl[:2]]
    with pytest.raises(hg.HlrError, match="cover"):
        hg.upload(5, None, bad_cover, 1e-6)
    overlap = [dict(b) for b in bl] + [dict(bl[0])]
    with pytest.raises(hg.HlrError, match="cover"):
        hg.upload(5, None, overlap, 1e-6)
    with pytest.raises(hg.HlrError, match="permutation"):
        hg.upload(5, [0, 1, 2, 3, 3], bl, 1e-6)
    nan = [dict(b) for b in bl]
    nan[0]["D"] = nan[0]["D"].copy()
    nan[0]["D"][1, 1] = np.nan
    with pytest.raises(hg.HlrError, match="NaN"):
        hg.upload(5, None, nan, 1e-6)
    with pytest.raises(hg.HlrError, match="eps"):
        hg.upload(5, None, bl, 0.0)
    lr = [dict(b) for b in bl]
    lr[2] = {"row0": 3, "nrows": 2, "col0": 0, "ncols": 5, "kind": 1, "W": np.ones((2, 1)),
             "S": np.array([-1.0]), "X": np.ones((5, 1))}
    with pytest.raises(hg.HlrError, match="sigma"):
        hg.upload(5, None, lr, 1e-6)
    oob = [dict(b) for b in bl]
    oob[1] = dict(oob[1], ncols=3)
    with pytest.raises(hg.HlrError, match="out of range"):
        hg.upload(5, None, oob, 1e-6)


def test_host_errors_have_messages():
    with pytest.raises(hg.HlrError) as ei:
        hg.afl_encode(np.array([1.0, np.inf]), 1e-3)
    assert "non-finite" in str(ei.value)
    with pytest.raises(hg.HlrError):
        hg.build_kernel_hmatrix(np.zeros((4, 2)), "exp2d", 0.0, scale=1.0)


def test_tuning_codes_and_rejection():
    """HLR_TUNING of the header and its Python mirror agree; bad layouts are refused before any
    device work."""
    hdr = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "hlr.h")).read()
    assert "#define HLR_TUNING(sub_log2, leaf_log2, piece_kb) ((sub_log2) | ((leaf_log2) << 4) | ((piece_kb) << 8))" in hdr
    assert hg.tuning_code() == 0
    assert hg.tuning_code(32, 64, 16) == 5 | (6 << 4) | (16 << 8)
    assert hg.tuning_code(128, 32, 8) == 7 | (5 << 4) | (8 << 8)
    assert "#define HLR_CTAS_PER_SM(k) ((k) << 20)" in hdr
    assert "#define HLR_ENCODE_DEVICE (1 << 17)" in hdr and hg.HLR_ENCODE_DEVICE == 1 << 17
    assert hg.tuning_code(ctas_per_sm=3) == 3 << 20
    assert hg.tuning_code(32, 64, 16, 2) == 5 | (6 << 4) | (16 << 8) | (2 << 20)
    with pytest.raises(hg.HlrError):
        hg.tuning_code(16, 64, 16)
    with pytest.raises(hg.HlrError):
        hg.tuning_code(ctas_per_sm=9)
    bl = _tiny_blocks()
    for bad in [3 | (6 << 4) | (16 << 8), 6 | (7 << 4) | (16 << 8), 6 | (6 << 4) | (2 << 8), 6 | (6 << 4) | (17 << 8),
                -1, 1 << 18, 1 << 19, 9 << 20, 1 << 24]:
        with pytest.raises(hg.HlrError, match="tuning"):
            hg.upload(5, None, bl, 1e-6, tuning=bad)
    with pytest.raises(hg.HlrError, match="tuning"):
        hg.upload(5, None, bl, 1e-6, fmt="fp64", tuning=hg.tuning_code(32, 64, 16))


def test_autotuner_rank_classes():
    from paper_2308_10960_gb300 import tune
    assert tune.rank_class({"rank_sum": 1000, "nlowrank": 90}, 8) == (8, 8)
    assert tune.rank_class({"rank_sum": 0, "nlowrank": 0}, 1) == (1, 1)
    t = tune.Autotuner()
    assert t.lookup({"rank_sum": 100, "nlowrank": 10}) is None
    t.table[(8, 1)] = (32, 64, 16)
    assert t.lookup({"rank_sum": 100, "nlowrank": 10}) == hg.tuning_code(32, 64, 16)


@pytest.mark.parametrize("fmt", ["afl", "aflp", "bfl", "dfl"])
@pytest.mark.parametrize("u", [0.5, 1e-2, 2.0 ** -9, 1e-6, 1e-9, 2.0 ** -60])
def test_host_encoder_all_formats_byte_exact(fmt, u):
    """hlr_encode writes exactly the oracle's stream for AFL and its aligned variants."""
    g = np.random.default_rng(21)
    for a in (g.standard_normal(333) * np.exp(g.uniform(-12, 12, 333)), np.zeros(7),
              np.array([0.0, -1.5, 3.0, -0.0, 1e-30])):
        ref = afl.encode(a, u, fmt)
        mm, e, m, data = hg.encode(a, u, fmt)
        assert (e, m) == (ref.e, ref.m) and mm == ref.m_min, (fmt, u)
        assert data == ref.data, (fmt, u)


@pytest.mark.parametrize("u", [0.5, 2.0 ** -11, 1e-4, 2.0 ** -24, 1e-9, 0.0])
def test_host_encoder_mp_byte_exact(u):
    """MP units (Section 3.3): hlr_encode picks the oracle's IEEE format for u and writes the same
    round-to-nearest-even patterns, through FP16 subnormals, ties and the largest finite half."""
    g = np.random.default_rng(22)
    t = 2.0 ** -11
    special = np.array([0.0, -0.0, 1.0 + t, 1.0 + 3 * t, -(1.0 + t), 2.0 ** -24, 2.0 ** -25, 3 * 2.0 ** -26,
                        2.0 ** -14 - 2.0 ** -26, 6.1e-5, 65504.0, 65519.99, -65519.99, 1e-30, 2049.0, 2051.0])
    for a in (g.standard_normal(333) * np.exp(g.uniform(-20, 9, 333)), special, np.zeros(3)):
        if u == 0.0:   # the encoder's "FP64" precision: the oracle selects by name
            ref = afl.encode_mp(a, u, "mp64")
            mm, e, m, data = hg.encode(a, 2.0 ** -60, "mp")
        else:
            ref = afl.encode(a, u, "mp")
            mm, e, m, data = hg.encode(a, u, "mp")
        assert (e, m, mm) == (ref.e, ref.m, 1.0) and data == ref.data, u


def test_host_encoder_mp_rejects_overflow():
    with pytest.raises(hg.HlrError):
        hg.encode(np.array([65520.0]), 0.5, "mp")
    with pytest.raises(hg.HlrError):
        hg.encode(np.array([1e39]), 1e-5, "mp")
    with pytest.raises(ValueError):
        afl.encode(np.array([65520.0]), 0.5, "mp")
    assert hg.encode(np.array([1e39]), 1e-9, "mp")[1] == 11


def test_host_encoder_rejects_values_outside_bfl():
    with pytest.raises(hg.HlrError):
        hg.encode(np.array([1e300]), 1e-6, "bfl")
    with pytest.raises(hg.HlrError):
        hg.encode(np.array([1.0]), 1e-6, 9)


@pytest.mark.parametrize("fmt", ["afl", "mp"])
def test_unit_arrays_follow_the_oracle_unit_order(fmt, exp2d_case):
    """unit_arrays lists the units as upload and the oracle's compress do (dense column-major;
    lowrank W columns then X columns) with the same precisions."""
    p, H, _ = exp2d_case
    C = ohm.compress(H, fmt=fmt)
    vals, off, prec = hg.unit_arrays(oracle_blocks(H), H.eps, fmt)
    units = [u for cb in C.blocks for u in cb.units]
    assert len(units) == prec.size == off.size - 1
    for k in range(0, len(units), 97):
        a = vals[off[k]:off[k + 1]]
        assert afl.encode(a, prec[k], fmt).data == units[k].data


def test_unit_list_precisions_sizes_and_errors(exp2d_case):
    """hlr_unit_list: every lowrank column's precision is the oracle's APLR precision
    eps sigma_0 / sigma_i (Section 3.3), dense leaves get eps (FP64 for MP); NULL outputs give
    the sizes; short outputs and bad sigma are refused."""
    import ctypes as C
    from paper_2308_10960_gb300 import _binding as B
    p, H, _ = exp2d_case
    blocks = oracle_blocks(H)
    vals, off, prec = hg.unit_arrays(blocks, H.eps, "afl")
    expect = []
    for b in H.blocks:
        if b.kind == ohm.DENSE:
            expect.append(H.eps)
        elif b.rank:
            us = afl.aplr_precisions(b.S, H.eps)
            expect += list(us) + list(us)
    assert np.array_equal(prec, np.array(expect))
    assert off[-1] == vals.size == sum(b["D"].size if b["kind"] == ohm.DENSE else
                                       b["S"].size * (b["nrows"] + b["ncols"]) for b in blocks)
    _, _, prec_mp = hg.unit_arrays(blocks, H.eps, "mp")
    dense = np.array([u for b in H.blocks for u in ([1] if b.kind == ohm.DENSE else [0] * (2 * b.rank))], bool)
    assert np.all(prec_mp[dense] == 2.0 ** -60) and np.array_equal(prec_mp[~dense], prec[~dense])
    db = hg._DescBuilder(p.n, None, blocks, H.eps, B.HLR_FMT_AFL_APLR)
    nu, nv = C.c_int64(0), C.c_int64(0)
    assert B.lib.hlr_unit_list(C.byref(db.desc), None, None, None, 0, 0, C.byref(nu), C.byref(nv)) == 0
    assert nu.value == prec.size and nv.value == vals.size
    small = np.zeros(nu.value, dtype=np.int64)
    rc = B.lib.hlr_unit_list(C.byref(db.desc), small.ctypes.data, None, None, nu.value, 0, C.byref(nu), C.byref(nv))
    assert rc == B.HLR_ERR_OOM
    lr = next(i for i, b in enumerate(blocks) if b["kind"] != ohm.DENSE and b["S"].size > 1)
    bad = [dict(b) for b in blocks]
    bad[lr]["S"] = bad[lr]["S"][::-1].copy()          # not led by its maximum
    with pytest.raises(hg.HlrError):
        hg.unit_arrays(bad, H.eps, "afl")
    with pytest.raises(hg.HlrError):
        hg.unit_arrays(blocks, 0.0, "afl")


def test_host_hmatrix_unit_arrays_match_block_copies():
    p = synth.laplace_problem(2048)
    Hh = hg.build_kernel_hmatrix(p.points, "laplace", 1e-6, diag=p.params["diag"])
    try:
        blocks = [Hh.block(i) for i in range(Hh.structure().shape[0])]
        for fmt in ("afl", "mp"):
            a = Hh.unit_arrays(fmt)
            b = hg.unit_arrays(blocks, Hh.eps, fmt)
            for x, y in zip(a, b):
                assert np.array_equal(x, y)
    finally:
        Hh.free()


def test_host_checkpoint_round_trip_and_corruption(tmp_path):
    """hlr_host_save / hlr_host_load: the loaded matrix has the same permutation, eps, block
    structure and bits; a flipped byte, a truncated file, another magic or version are refused."""
    p = synth.laplace_problem(1500)
    Hh = hg.build_kernel_hmatrix(p.points, "laplace", 1e-6, diag=p.params["diag"])
    path = str(tmp_path / "m.hlr")
    try:
        Hh.save(path)
        G = hg.load_host_hmatrix(path)
        try:
            assert G.n == Hh.n and G.eps == Hh.eps and np.array_equal(G.perm, Hh.perm)
            assert np.array_equal(G.structure(), Hh.structure())
            for i in range(Hh.structure().shape[0]):
                a, b = Hh.block(i), G.block(i)
                for k in ("D", "W", "S", "X"):
                    if k in a:
                        assert np.array_equal(np.asarray(a[k]).view(np.int64), np.asarray(b[k]).view(np.int64))
            va, oa, ua = Hh.unit_arrays()
            vb, ob, ub = G.unit_arrays()
            assert np.array_equal(va, vb) and np.array_equal(oa, ob) and np.array_equal(ua, ub)
        finally:
            G.free()
    finally:
        Hh.free()
    raw = open(path, "rb").read()
    bad = []
    flipped = bytearray(raw)
    flipped[len(raw) // 2] ^= 0x10
    bad.append(bytes(flipped))
    bad.append(raw[:-100])
    bad.append(b"XXXXXXXX" + raw[8:])
    for k, data in enumerate(bad):
        q = str(tmp_path / f"bad{k}.hlr")
        open(q, "wb").write(data)
        with pytest.raises(hg.HlrError):
            hg.load_host_hmatrix(q)

    def fnv1a(b):                      # the file's trailer: FNV-1a 64 of every byte before it
        h = 1469598103934665603
        for c in b:
            h = ((h ^ c) * 1099511628211) & (2 ** 64 - 1)
        return h.to_bytes(8, "little")

    body = bytearray(raw[:-8])
    assert fnv1a(bytes(body)) == raw[-8:]
    ver = bytearray(body)
    ver[8] = 2                          # another version, with a valid hash
    q = str(tmp_path / "ver.hlr")
    open(q, "wb").write(bytes(ver) + fnv1a(bytes(ver)))
    with pytest.raises(hg.HlrError, match="unsupported version"):
        hg.load_host_hmatrix(q)
    bad_blk = bytearray(body)
    off = 8 + 4 + 4 + 8 + 8 + 8 + 8 * 1500   # first block: row0
    bad_blk[off:off + 8] = (1500).to_bytes(8, "little", signed=True)   # rows past n
    q = str(tmp_path / "blk.hlr")
    open(q, "wb").write(bytes(bad_blk) + fnv1a(bytes(bad_blk)))
    with pytest.raises(hg.HlrError, match="malformed"):
        hg.load_host_hmatrix(q)
    # a failed save (unwritable directory) leaves no partial file and raises
    with pytest.raises(hg.HlrError):
        Hh2 = hg.build_kernel_hmatrix(p.points[:200], "laplace", 1e-6, diag=p.params["diag"])
        try:
            Hh2.save(str(tmp_path / "missing_dir" / "m.hlr"))
        finally:
            Hh2.free()
    with pytest.raises(hg.HlrError):
        hg.load_host_hmatrix(str(tmp_path / "missing.hlr"))
