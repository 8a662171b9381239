"""Multi-RHS and batched products (hlr_matvec_batched) against the oracle.

The reference is the oracle's decoded matrix A~ (assembled densely at n <= 4096, Section 5.4)
applied to every right-hand side: Y_out = Y_in + A~ X. Multi-RHS requests with FP32
accumulation run passes of up to 32 columns (a value decoded once, used for every column);
single columns, FP64 accumulation and plain FP64 storage run the single-RHS kernels, many
products per persistent launch. Also checked: a request gives the same bits alone and mixed
with others, the same handle may appear twice, and a batch replays from a captured CUDA graph.
"""
import numpy as np
import pytest

import synth
from oracle import hmatrix as ohm
from tests._util import oracle_blocks

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
hg = pytest.importorskip("paper_2308_10960_gb300")

TOL = {"fp64": 1e-12, "fp32": 1e-6}


@pytest.fixture(scope="module")
def dense_refs(exp2d_case, matern_small_case):
    out = {}
    for name, (p, H, C) in (("exp2d", exp2d_case), ("matern", matern_small_case)):
        out[name] = (H, C, ohm.to_dense(C))
    return out


@pytest.fixture(scope="module")
def uploaded(dense_refs):
    mats = {}
    for name, (H, C, Ad) in dense_refs.items():
        mats[name] = hg.upload(H.n, H.perm, oracle_blocks(H), H.eps)
        mats[name + "_fp64"] = hg.upload(H.n, H.perm, oracle_blocks(H), H.eps, fmt="fp64")
    yield mats
    for A in mats.values():
        A.free()


def _rhs(n, r, seed):
    g = np.random.default_rng(seed)
    return g.standard_normal((r, n)), g.standard_normal((r, n))   # X, Y0 as (r, n): column-major n x r


def _check(Ad, X, Y0, got, acc):
    ref = Y0 + (Ad @ X.T).T
    absprod = (np.abs(Ad) @ np.abs(X.T)).T + np.abs(Y0)
    for j in range(X.shape[0]):
        rel = np.linalg.norm(got[j] - ref[j]) / np.linalg.norm(ref[j])
        assert rel <= TOL[acc], (acc, j, rel)
        comp = np.max(np.abs(got[j] - ref[j]) / np.maximum(absprod[j], 1e-300))
        assert comp <= 10 * TOL[acc], (acc, j, comp)


def _batched(mats, Xs, Y0s, acc="fp32"):
    Xd = [torch.from_numpy(np.ascontiguousarray(X)).cuda() for X in Xs]
    Yd = [torch.from_numpy(np.ascontiguousarray(Y)).cuda() for Y in Y0s]
    hg.matvec_batched(mats, Xd, Yd, acc=acc)
    for A in set(mats):
        A.check()
    torch.cuda.synchronize()
    return [Y.cpu().numpy() for Y in Yd]


@pytest.mark.parametrize("r", [2, 8, 13, 32, 45])
@pytest.mark.parametrize("case", ["exp2d", "matern"])
def test_multi_rhs_matches_oracle(case, r, dense_refs, uploaded):
    H, C, Ad = dense_refs[case]
    A = uploaded[case]
    X, Y0 = _rhs(H.n, r, 10 + r)
    got = _batched([A], [X], [Y0])[0]
    _check(Ad, X, Y0, got, "fp32")


@pytest.mark.parametrize("acc", ["fp64", "fp32"])
def test_batched_mixed_requests_match_oracle_and_alone(acc, dense_refs, uploaded):
    reqs = [("exp2d", 1), ("matern", 8), ("exp2d_fp64", 3), ("matern", 1), ("exp2d", 32), ("matern_fp64", 1),
            ("exp2d", 5)]
    mats, Xs, Y0s = [], [], []
    for i, (name, r) in enumerate(reqs):
        A = uploaded[name]
        X, Y0 = _rhs(A.n, r, 100 + i)
        mats.append(A)
        Xs.append(X)
        Y0s.append(Y0)
    mixed = _batched(mats, Xs, Y0s, acc=acc)
    for i, (name, r) in enumerate(reqs):
        Ad = dense_refs[name.replace("_fp64", "")][2]
        tol = "fp64" if (acc == "fp64" or name.endswith("_fp64")) else "fp32"
        if name.endswith("_fp64"):
            # plain storage holds the uncompressed factors: compare with its own dense matrix
            H = dense_refs[name.replace("_fp64", "")][0]
            Ad = ohm.to_dense(H, decoded=False)
        _check(Ad, Xs[i], Y0s[i], mixed[i], tol)
        alone = _batched([mats[i]], [Xs[i]], [Y0s[i]], acc=acc)[0]
        assert np.array_equal(alone.view(np.int64), mixed[i].view(np.int64)), (name, r)


def test_single_rhs_batched_equals_matvec_bits(dense_refs, uploaded):
    A = uploaded["matern"]
    X, Y0 = _rhs(A.n, 1, 7)
    got = _batched([A, A], [X, X], [Y0, Y0])
    xd = torch.from_numpy(X[0].copy()).cuda()
    yd = torch.from_numpy(Y0[0].copy()).cuda()
    A.matvec(xd, yd, acc="fp32")
    ref = yd.cpu().numpy()
    for g in got:
        assert np.array_equal(g[0].view(np.int64), ref.view(np.int64))


def test_batched_graph_replay(dense_refs, uploaded):
    mats = [uploaded["exp2d"], uploaded["matern"], uploaded["exp2d"]]
    rs = [1, 8, 16]
    Xs = [torch.from_numpy(_rhs(A.n, r, 50 + i)[0]).cuda() for i, (A, r) in enumerate(zip(mats, rs))]
    Ys = [torch.zeros((r, A.n), dtype=torch.float64, device="cuda") for A, r in zip(mats, rs)]
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        hg.matvec_batched(mats, Xs, Ys, stream=s)       # eager call: allocates the pass scratch
    torch.cuda.synchronize()
    eager = [Y.clone() for Y in Ys]
    g = torch.cuda.CUDAGraph()
    for Y in Ys:
        Y.zero_()
    torch.cuda.synchronize()
    with torch.cuda.graph(g):
        hg.matvec_batched(mats, Xs, Ys)
    for Y in Ys:
        Y.zero_()
    g.replay()
    torch.cuda.synchronize()
    for Y, E in zip(Ys, eager):
        assert torch.equal(Y, E)
    g.replay()
    torch.cuda.synchronize()
    for Y, E in zip(Ys, eager):
        assert torch.equal(Y, 2 * E)
    for A in set(mats):
        A.check()


def test_batched_validation(uploaded):
    A = uploaded["exp2d"]
    X = torch.zeros(A.n - 1, dtype=torch.float64, device="cuda")
    Y = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    with pytest.raises(hg.HlrError):
        hg.matvec_batched([A], [X], [Y])


def test_multi_columns_are_matvec_bits(dense_refs, uploaded):
    """Under HLR_MULTI every column is a product of its own: its bits are those of matvec for
    that column, in any batch (one request of 40 columns, or 13 + 7 columns, or alone)."""
    H, C, Ad = dense_refs["matern"]
    A = uploaded["matern"]
    X, Y0 = _rhs(H.n, 40, 77)

    def run(mats, Xs, Ys):
        Xd = [torch.from_numpy(np.ascontiguousarray(v)).cuda() for v in Xs]
        Yd = [torch.from_numpy(np.ascontiguousarray(v)).cuda() for v in Ys]
        hg.matvec_batched(mats, Xd, Yd, acc="fp32", multi=True)
        A.check()
        torch.cuda.synchronize()
        return [v.cpu().numpy() for v in Yd]

    wide = run([A], [X], [Y0])[0]
    _check(Ad, X, Y0, wide, "fp32")
    for j in (0, 12, 33, 39):
        yd = torch.from_numpy(Y0[j].copy()).cuda()
        A.matvec(torch.from_numpy(X[j].copy()).cuda(), yd, acc="fp32")
        assert np.array_equal(yd.cpu().numpy().view(np.int64), wide[j].view(np.int64)), j
    mid = run([A, A], [X[:13], X[33:]], [Y0[:13], Y0[33:]])
    assert np.array_equal(mid[0].view(np.int64), wide[:13].view(np.int64))
    assert np.array_equal(mid[1].view(np.int64), wide[33:].view(np.int64))


def test_narrow_and_wide_passes_match_oracle_and_repeat(dense_refs, uploaded):
    """A 40-column request (a wide 32-column pass and a narrow 8-column pass) and the same
    columns as 13- and 7-column requests all match the oracle; every request repeats bit for
    bit (the passes are deterministic)."""
    H, C, Ad = dense_refs["matern"]
    A = uploaded["matern"]
    X, Y0 = _rhs(H.n, 40, 78)
    big = _batched([A], [X], [Y0])[0]
    _check(Ad, X, Y0, big, "fp32")
    parts = _batched([A, A], [X[:13], X[33:]], [Y0[:13], Y0[33:]])
    _check(Ad, X[:13], Y0[:13], parts[0], "fp32")
    _check(Ad, X[33:], Y0[33:], parts[1], "fp32")
    again = _batched([A], [X], [Y0])[0]
    assert np.array_equal(again.view(np.int64), big.view(np.int64))
