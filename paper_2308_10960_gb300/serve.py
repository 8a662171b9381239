"""Serving loop for compressed H-matrices: continuous batching of matrix-vector products and CG
solves against several matrices kept resident on one GPU.

* Admission: a matrix is uploaded when a request for it is due and its device bytes fit in the
  HBM budget next to the resident ones; otherwise idle resident matrices are evicted, least
  recently used first. A request waits while its matrix cannot be admitted.
* Batching: whenever the GPU finishes a batch, all queued products of every resident idle matrix
  (up to ``max_rhs`` per matrix) go into ONE ``hlr_matvec_batched`` call. With ``HLR_MULTI``
  every column is a product of its own (many per launch) on a scratch set of its own, so a
  request gets the bits of ``matvec`` alone and in the mix, and a batch never shares scratch
  with a solve of the same matrix.
* Solves: unpreconditioned CG (``hlr_solve_cg``) runs in worker threads on their own streams,
  overlapping the product batches; the library call releases the interpreter lock. Its
  product kernels take a share of the CTA slots (``HLR_SM_SHARE``, half by default) and it
  reads its residual from the host only every few iterations, so product batches find room on
  the SMs while solves run.
* A matrix runs at most one product batch and at most one solve at a time: the batches use the
  per-column scratch sets of its handle, the solves the handle's own scratch and the CG
  workspace, so one of each may overlap.

Latency = finish - arrival per request; the run reports p50/p99 per request kind, throughput
and the algorithmic bytes moved. The backend is pluggable: ``GpuBackend`` drives the library,
tests may substitute a host-only backend with the same methods.
"""
from __future__ import annotations

import collections
import math
import threading
import time
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field
from typing import Any


@dataclass
class Request:
    rid: int
    kind: str                 # "matvec" (y = A~ x) or "solve" (A~ y = x by CG)
    matrix: str
    x: Any                    # right-hand side: device vector of length n
    arrival: float = 0.0      # seconds after the start of the run
    rtol: float = 1e-8
    maxit: int = 10000
    y: Any = None             # result; a device vector of length n given here receives it
    ready: Any = None         # CUDA event after the client's writes of x (None: x is complete)
    iters: int = 0
    relres: float = 0.0
    start: float | None = None
    finish: float | None = None
    error: str | None = None

    @property
    def latency(self) -> float:
        return self.finish - self.arrival


def percentile(values, q: float) -> float:
    """Nearest-rank percentile (q in [0, 100]) of a non-empty sequence."""
    v = sorted(values)
    k = max(0, min(len(v) - 1, int(math.ceil(q / 100.0 * len(v))) - 1))
    return float(v[k])


@dataclass
class Stats:
    makespan: float = 0.0
    completed: int = 0
    failed: int = 0
    latency: dict = field(default_factory=dict)     # kind -> {"p50", "p99", "mean", "count"} (ms)
    batches: int = 0
    batch_columns: list = field(default_factory=list)
    bytes_moved: float = 0.0
    loads: int = 0
    evictions: int = 0
    peak_resident_bytes: int = 0

    def as_dict(self) -> dict:
        return {"makespan_s": self.makespan, "completed": self.completed, "failed": self.failed,
                "requests_per_s": self.completed / self.makespan if self.makespan > 0 else 0.0,
                "GB/s": self.bytes_moved / self.makespan / 1e9 if self.makespan > 0 else 0.0,
                "latency_ms": self.latency, "batches": self.batches,
                "mean_batch_columns": (sum(self.batch_columns) / len(self.batch_columns)) if self.batch_columns else 0,
                "loads": self.loads, "evictions": self.evictions, "peak_resident_bytes": self.peak_resident_bytes}


class Server:
    def __init__(self, backend, budget_bytes: int, cg_workers: int = 2, max_rhs: int = 32, poll_s: float = 2e-4):
        self.backend = backend
        self.budget = int(budget_bytes)
        self.cg_workers = int(cg_workers)
        self.max_rhs = int(max_rhs)
        self.poll_s = poll_s
        self._preloaded: collections.OrderedDict[str, int] = collections.OrderedDict()

    def preload(self, names) -> list[str]:
        """Admit matrices before any request arrives, in the given order, while they fit the
        budget (a run starts with them resident). Returns the names loaded."""
        loaded = []
        used = sum(self._preloaded.values())
        for m in names:
            need = self.backend.device_bytes(m)
            if m in self._preloaded or used + need > self.budget:
                continue
            self.backend.load(m)
            self._preloaded[m] = need
            used += need
            loaded.append(m)
        return loaded

    def run(self, requests: list[Request], realtime: bool = True) -> Stats:
        """Serve `requests` (arrival times in seconds from the start). With realtime=False every
        request is due at once (arrival 0)."""
        be = self.backend
        st = Stats()
        todo = sorted(requests, key=lambda r: (r.arrival, r.rid))
        if not realtime:
            for r in todo:
                r.arrival = 0.0
        q_mv: dict[str, collections.deque] = collections.defaultdict(collections.deque)
        q_cg: dict[str, collections.deque] = collections.defaultdict(collections.deque)
        resident: collections.OrderedDict[str, int] = collections.OrderedDict(self._preloaded)   # LRU order
        used = sum(resident.values())
        st.peak_resident_bytes = used
        busy_mv: set[str] = set()      # matrices with a product batch in flight
        busy_cg: set[str] = set()      # matrices with a solve in flight
        inflight_mv: list = []          # (token, names, requests)
        inflight_cg: dict = {}          # future -> (name, request)
        done = 0
        nxt = 0
        pool = ThreadPoolExecutor(max_workers=max(1, self.cg_workers))
        t0 = time.perf_counter()
        now = lambda: time.perf_counter() - t0  # noqa: E731

        def finish(r: Request, err: str | None = None):
            nonlocal done
            r.finish = now()
            r.error = err
            done += 1

        try:
            while done < len(todo):
                progressed = False
                t = now()
                while nxt < len(todo) and todo[nxt].arrival <= t:
                    r = todo[nxt]
                    (q_mv if r.kind == "matvec" else q_cg)[r.matrix].append(r)
                    nxt += 1
                    progressed = True
                # completions
                still = []
                for tok, names, reqs in inflight_mv:
                    if be.poll(tok):
                        for r in reqs:
                            finish(r)
                        busy_mv.difference_update(names)
                        progressed = True
                    else:
                        still.append((tok, names, reqs))
                inflight_mv = still
                for fut in [f for f in inflight_cg if f.done()]:
                    name, r = inflight_cg.pop(fut)
                    exc = fut.exception()
                    finish(r, None if exc is None else str(exc))
                    busy_cg.discard(name)
                    progressed = True
                # admission: matrices with queued work, in order of their oldest request
                wanting = [m for m in set(q_mv) | set(q_cg) if (q_mv[m] or q_cg[m]) and m not in resident]
                wanting.sort(key=lambda m: min([r.arrival for r in list(q_mv[m]) + list(q_cg[m])]))
                for m in wanting:
                    need = be.device_bytes(m)
                    if need > self.budget:
                        for r in list(q_mv[m]) + list(q_cg[m]):
                            finish(r, "matrix larger than the HBM budget")
                        q_mv[m].clear()
                        q_cg[m].clear()
                        continue
                    for victim in list(resident):
                        if used + need <= self.budget:
                            break
                        if victim in busy_mv or victim in busy_cg or q_mv[victim] or q_cg[victim]:
                            continue
                        be.unload(victim)
                        used -= resident.pop(victim)
                        st.evictions += 1
                    if used + need <= self.budget:
                        be.load(m)
                        resident[m] = need
                        used += need
                        st.loads += 1
                        st.peak_resident_bytes = max(st.peak_resident_bytes, used)
                        progressed = True
                # products: one batched call over every resident idle matrix with queued products
                groups = []
                for m in list(resident):
                    if m in busy_mv or not q_mv[m]:
                        continue
                    take = [q_mv[m].popleft() for _ in range(min(self.max_rhs, len(q_mv[m])))]
                    groups.append((m, take))
                if groups:
                    t = now()
                    for m, take in groups:
                        for r in take:
                            r.start = t
                        busy_mv.add(m)
                        resident.move_to_end(m)
                        st.batch_columns.append(len(take))
                    tok = be.launch_matvecs(groups)
                    st.bytes_moved += sum(be.product_bytes(m, len(take)) for m, take in groups)
                    inflight_mv.append((tok, [m for m, _ in groups], [r for _, take in groups for r in take]))
                    st.batches += 1
                    progressed = True
                # solves on free workers
                for m in list(resident):
                    if len(inflight_cg) >= self.cg_workers:
                        break
                    if m in busy_cg or not q_cg[m]:
                        continue
                    r = q_cg[m].popleft()
                    r.start = now()
                    busy_cg.add(m)
                    resident.move_to_end(m)
                    inflight_cg[pool.submit(be.solve, m, r)] = (m, r)
                    progressed = True
                if not progressed:
                    time.sleep(self.poll_s)
        finally:
            pool.shutdown(wait=True)
            be.drain()
        st.makespan = now()
        kinds = collections.defaultdict(list)
        for r in todo:
            if r.error is None:
                kinds[r.kind].append(r.latency * 1e3)
                st.completed += 1
            else:
                st.failed += 1
        for k, lat in kinds.items():
            st.latency[k] = {"p50": percentile(lat, 50), "p99": percentile(lat, 99),
                             "mean": sum(lat) / len(lat), "count": len(lat)}
        # bytes of the solves: one product per iteration
        st.bytes_moved += sum(be.product_bytes(r.matrix, 1) * max(r.iters, 0) for r in todo if r.kind == "solve")
        return st


class GpuBackend:
    """Drives the library. `host_mats` maps names to objects with ``upload(fmt, stream=...)``
    returning a DeviceHMatrix (HostHMatrix, or any adapter); they are uploaded on admission.

    Nothing on the request path allocates device memory, creates CUDA objects or touches the
    legacy default stream: the streams, events and per-matrix staging buffers are made up front
    (at construction and on admission), because those calls can wait for work on other streams
    and stall the serving loop for as long as the solves keep the GPU busy (measured: an event
    recorded on the default stream held a product batch for seconds). A request's x must be
    complete when it is submitted, or carry in ``ready`` an event recorded after its writes. A
    request whose ``y`` is a device vector of length n (the client's output buffer) gets its
    result written there; otherwise one is allocated for it."""

    def __init__(self, host_mats: dict, acc_cg: str = "fp32", solve_share: int = 4, max_rhs: int = 32,
                 cg_workers: int = 4, events: int = 256, tunings: dict | None = None):
        import torch
        from . import matvec_batched
        self.torch = torch
        self._batched = matvec_batched
        self.host = dict(host_mats)
        self.tunings = dict(tunings or {})   # name -> tuning code of its upload (e.g. autotuned)
        self.dev = {}
        self.acc_cg = acc_cg
        self.max_rhs = int(max_rhs)
        # solves run their product kernels on solve_share eighths of the CTA slots
        # (HLR_SM_SHARE), so that product batches find room on every SM while solves run
        self.solve_share = int(solve_share)
        # product batches on a high-priority stream: their CTAs are scheduled ahead of the
        # solves' kernels, so a short product does not queue behind long CG runs
        self.stream = torch.cuda.Stream(priority=-1)
        self._solve_streams = [torch.cuda.Stream() for _ in range(max(1, cg_workers))]
        self._free_streams = list(range(len(self._solve_streams)))
        self._lock = threading.Lock()
        # events, created (first recorded) here: product-batch completion tokens, input order
        # for the product stream and one per solve stream
        self._events = [torch.cuda.Event() for _ in range(events)]
        for e in self._events:
            e.record(self.stream)
        self._free_events = list(range(events))
        self._staging = {}
        self._bytes = {}
        self._alg = {}
        for name, H in self.host.items():     # device footprint and algorithmic bytes, measured once
            A = H.upload("afl")
            self._bytes[name] = int(A.info["device_bytes"])
            self._alg[name] = (float(A.info["algorithmic_bytes"]), int(A.info["n"]))
            A.free()
        torch.cuda.synchronize()

    def device_bytes(self, name: str) -> int:
        return self._bytes[name] + 2 * 8 * self.max_rhs * self._alg[name][1]

    def product_bytes(self, name: str, r: int) -> float:
        alg, n = self._alg[name]
        return alg - 32.0 * n + 8.0 * n + r * 24.0 * n

    def load(self, name: str):
        if name not in self.dev:          # a later run on the same backend finds it resident
            torch = self.torch
            n = self._alg[name][1]
            with torch.cuda.stream(self.stream):
                code = self.tunings.get(name, 0)
                self.dev[name] = (self.host[name].upload("afl", stream=self.stream, tuning=code) if code
                                  else self.host[name].upload("afl", stream=self.stream))
                X, Y = (torch.zeros((self.max_rhs, n), dtype=torch.float64, device="cuda"),
                        torch.zeros((self.max_rhs, n), dtype=torch.float64, device="cuda"))
                self._staging[name] = (X, Y)
                # one full-width batch now, so that the per-column scratch sets exist before any
                # request (the library allocates them on first use)
                self._batched([self.dev[name]], [X], [Y], acc="fp32", stream=self.stream, multi=True)
                Y.zero_()

    def unload(self, name: str):
        if name in self.dev:
            self.dev.pop(name).free()
            self._staging.pop(name, None)

    def launch_matvecs(self, groups):
        torch = self.torch
        mats, Xs, Ys = [], [], []
        with torch.cuda.stream(self.stream):
            for name, reqs in groups:
                X, Y = self._staging[name]
                k = len(reqs)
                for i, r in enumerate(reqs):
                    if r.ready is not None:
                        self.stream.wait_event(r.ready)
                    X[i].copy_(r.x)
                Y[:k].zero_()
                mats.append(self.dev[name])
                Xs.append(X[:k])
                Ys.append(Y[:k])
            self._batched(mats, Xs, Ys, acc="fp32", stream=self.stream, multi=True)
            for (name, reqs), Y in zip(groups, Ys):
                for i, r in enumerate(reqs):
                    if r.y is None:
                        r.y = torch.empty_like(r.x)
                    r.y.copy_(Y[i])
            with self._lock:
                idx = self._free_events.pop() if self._free_events else None
            ev = self._events[idx] if idx is not None else torch.cuda.Event()
            ev.record(self.stream)
        return (ev, idx)

    def poll(self, token) -> bool:
        ev, idx = token
        if not ev.query():
            return False
        if idx is not None:
            with self._lock:
                self._free_events.append(idx)
        return True

    def solve(self, name: str, r: Request):
        torch = self.torch
        with self._lock:                  # a solve holds one of the solve streams while it runs
            if not self._free_streams:    # more concurrent solves than streams made up front
                self._solve_streams.append(torch.cuda.Stream())
                self._free_streams.append(len(self._solve_streams) - 1)
            k = self._free_streams.pop()
        try:
            s = self._solve_streams[k]
            A = self.dev[name]
            if r.ready is not None:
                s.wait_event(r.ready)
            with torch.cuda.stream(s):
                if r.y is None:
                    r.y = torch.zeros_like(r.x)
                else:
                    r.y.zero_()
                r.iters, r.relres = A.solve_cg(r.x, r.y, rtol=r.rtol, maxit=r.maxit, acc=self.acc_cg, stream=s,
                                               raise_noconv=False, sm_share=self.solve_share)
            s.synchronize()
        finally:
            with self._lock:
                self._free_streams.append(k)

    def drain(self):
        self.torch.cuda.synchronize()

    def close(self):
        for name in list(self.dev):
            self.unload(name)


def poisson_arrivals(count: int, rate: float, seed: int) -> list[float]:
    """`count` arrival times of a Poisson process of `rate` requests per second."""
    import numpy as np
    g = np.random.default_rng(seed)
    return list(np.cumsum(g.exponential(1.0 / rate, size=count)))
