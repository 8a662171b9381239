"""Host logic of the serving loop (admission against the HBM budget, LRU eviction, continuous
batching, one operation per matrix at a time, percentiles), with a host-only backend that
computes with numpy and completes products after a simulated device time."""
import threading
import time

import numpy as np
import pytest

from paper_2308_10960_gb300.serve import Request, Server, percentile, poisson_arrivals


class FakeBackend:
    def __init__(self, mats, product_s=2e-3):
        self.mats = mats                      # name -> (dense matrix, device bytes)
        self.product_s = product_s
        self.resident = set()
        self.active = {"mv": set(), "cg": set()}
        self.lock = threading.Lock()
        self.max_used = 0
        self.loads = []
        self.overlap = False

    def device_bytes(self, name):
        return self.mats[name][1]

    def product_bytes(self, name, r):
        return 8.0 * self.mats[name][0].size + 24.0 * r * self.mats[name][0].shape[0]

    def load(self, name):
        self.resident.add(name)
        self.loads.append(name)
        self.max_used = max(self.max_used, sum(self.mats[m][1] for m in self.resident))

    def unload(self, name):
        assert name not in self.active["mv"] and name not in self.active["cg"]
        self.resident.remove(name)

    def _enter(self, name, kind):
        with self.lock:
            assert name in self.resident
            if name in self.active[kind]:
                self.overlap = True
            self.active[kind].add(name)

    def _leave(self, name, kind):
        with self.lock:
            self.active[kind].discard(name)

    def launch_matvecs(self, groups):
        for name, reqs in groups:
            self._enter(name, "mv")
            A = self.mats[name][0]
            for r in reqs:
                r.y = A @ r.x                 # per column: independent of the batch
        return (time.perf_counter() + self.product_s, [name for name, _ in groups])

    def poll(self, tok):
        if time.perf_counter() >= tok[0]:
            for name in tok[1]:
                self._leave(name, "mv")
            return True
        return False

    def solve(self, name, r):
        self._enter(name, "cg")
        try:
            A = self.mats[name][0]
            r.y = np.linalg.solve(A, r.x)
            r.iters = 7
            time.sleep(self.product_s * 3)
        finally:
            self._leave(name, "cg")

    def drain(self):
        pass


def _mats(sizes, nbytes):
    g = np.random.default_rng(0)
    out = {}
    for i, (n, b) in enumerate(zip(sizes, nbytes)):
        M = g.standard_normal((n, n))
        out[f"m{i}"] = (M @ M.T + n * np.eye(n), b)
    return out


def _requests(mats, count, seed, rate=2000.0, solve_frac=0.3):
    g = np.random.default_rng(seed)
    names = sorted(mats)
    arr = poisson_arrivals(count, rate, seed)
    reqs = []
    for i in range(count):
        m = names[g.integers(len(names))]
        kind = "solve" if g.random() < solve_frac else "matvec"
        reqs.append(Request(i, kind, m, g.standard_normal(mats[m][0].shape[0]), arrival=arr[i]))
    return reqs


def test_percentile_nearest_rank():
    v = list(range(1, 101))
    assert percentile(v, 50) == 50 and percentile(v, 99) == 99 and percentile(v, 100) == 100
    assert percentile([3.0], 99) == 3.0


def test_all_requests_served_correctly_within_budget():
    mats = _mats([30, 40, 50, 60], [300, 400, 500, 600])
    be = FakeBackend(mats)
    reqs = _requests(mats, 120, 1)
    st = Server(be, budget_bytes=1000, cg_workers=2, max_rhs=4).run(reqs)
    assert st.completed == 120 and st.failed == 0
    assert be.max_used <= 1000 and st.peak_resident_bytes <= 1000
    assert st.evictions > 0 and not be.overlap
    for r in reqs:
        A = mats[r.matrix][0]
        ref = A @ r.x if r.kind == "matvec" else np.linalg.solve(A, r.x)
        assert np.allclose(r.y, ref, rtol=1e-10, atol=1e-10)
        assert r.finish >= r.start >= r.arrival
    assert all(c <= 4 for c in st.batch_columns)
    for k in ("matvec", "solve"):
        lat = st.latency[k]
        assert lat["count"] > 0 and 0 <= lat["p50"] <= lat["p99"]


def test_burst_is_batched_into_few_launches():
    mats = _mats([20, 20], [10, 10])
    be = FakeBackend(mats, product_s=5e-3)
    g = np.random.default_rng(2)
    reqs = [Request(i, "matvec", f"m{i % 2}", g.standard_normal(20)) for i in range(64)]
    st = Server(be, budget_bytes=100, max_rhs=32).run(reqs, realtime=False)
    assert st.completed == 64
    assert st.batches == 1 and sorted(st.batch_columns) == [32, 32]


def test_oversized_matrix_fails_its_requests_only():
    mats = _mats([10, 10], [50, 500])
    be = FakeBackend(mats)
    g = np.random.default_rng(3)
    reqs = [Request(0, "matvec", "m0", g.standard_normal(10)), Request(1, "matvec", "m1", g.standard_normal(10))]
    st = Server(be, budget_bytes=100).run(reqs, realtime=False)
    assert st.completed == 1 and st.failed == 1
    assert reqs[1].error and reqs[0].error is None


def test_mix_equals_alone():
    mats = _mats([25, 35], [10, 10])
    reqs = _requests(mats, 40, 4, solve_frac=0.25)
    Server(FakeBackend(mats), budget_bytes=100, max_rhs=8).run(reqs)
    for r in reqs:
        alone = Request(0, r.kind, r.matrix, r.x)
        Server(FakeBackend(mats), budget_bytes=100).run([alone], realtime=False)
        assert np.array_equal(alone.y, r.y)


def test_preload_admits_within_budget_and_run_keeps_them():
    mats = _mats([10, 10, 10], [40, 40, 40])
    be = FakeBackend(mats)
    srv = Server(be, budget_bytes=100)
    assert srv.preload(["m0", "m1", "m2"]) == ["m0", "m1"]
    g = np.random.default_rng(5)
    reqs = [Request(i, "matvec", f"m{i % 2}", g.standard_normal(10)) for i in range(6)]
    st = srv.run(reqs, realtime=False)
    assert st.completed == 6 and st.loads == 0 and be.loads == ["m0", "m1"]
