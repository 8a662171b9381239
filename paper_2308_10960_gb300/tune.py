"""Autotuner of the work layout and launch shape of the AFL product kernels.

For a matrix, every candidate (rows per lane of an X column, rows of a phase-2 task, piece size,
CTAs per SM the persistent work lists are made for; HLR_TUNING and HLR_CTAS_PER_SM in
include/hlr.h) is uploaded and timed on the GPU with CUDA events for the requested number of
right-hand sides; the fastest wins. Results are kept per rank class (the matrix's mean lowrank
rank, rounded to a power of two, and the column count), so a server can reuse the choice for
new matrices of the same class without timing them.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

from . import HlrError, matvec_batched, tuning_code

# (sub_rows, leaf_rows, piece_kb, ctas_per_sm); ctas_per_sm 0 = as many as the single-column
# kernels keep resident; 3 and 2 balance the work lists for the kernels that keep fewer (the
# 32-column passes, FP64 accumulation)
CANDIDATES = [(64, 64, 16, 0), (32, 64, 16, 0), (128, 64, 16, 0), (64, 32, 16, 0), (32, 32, 16, 0), (64, 64, 8, 0),
              (64, 64, 16, 3), (64, 64, 16, 2)]


@dataclass
class Result:
    best: tuple
    ms: dict = field(default_factory=dict)     # candidate -> ms per product (or pass)
    rank_class: tuple = ()


def rank_class(info: dict, nrhs: int) -> tuple:
    """(power of two of the mean rank of the lowrank blocks, column count)."""
    mean = info["rank_sum"] / max(1, info["nlowrank"])
    return (1 << max(0, round(math.log2(max(1.0, mean)))), int(nrhs))


def _time(A, nrhs: int, reps: int, torch, multi: bool = False) -> float:
    n = A.n
    X = torch.randn((nrhs, n) if nrhs > 1 else (n,), dtype=torch.float64, device="cuda")
    Y = torch.zeros_like(X)
    if nrhs == 1 and not multi:
        run = lambda: A.matvec(X, Y, acc="fp32")  # noqa: E731
    else:
        run = lambda: matvec_batched([A], [X], [Y], multi=multi)  # noqa: E731
    for _ in range(3):
        run()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        run()
    e1.record()
    torch.cuda.synchronize()
    A.check()
    return e0.elapsed_time(e1) / reps


class Autotuner:
    """multi=True times the products as a server runs them (HLR_MULTI: single columns through
    the multi-column pass kernels)."""

    def __init__(self, candidates=None, reps: int = 20, multi: bool = False):
        self.candidates = list(candidates or CANDIDATES)
        self.reps = reps
        self.multi = multi
        self.table: dict[tuple, tuple] = {}

    def lookup(self, info: dict, nrhs: int = 1):
        """Tuning code of the stored choice for this rank class, or None."""
        c = self.table.get(rank_class(info, nrhs))
        return None if c is None else tuning_code(*c)

    def tune(self, host, nrhs: int = 1) -> Result:
        """Time every candidate layout of `host` (an object with upload(fmt, tuning=...)) and
        record the fastest for its rank class."""
        import torch
        ms = {}
        info = None
        for cand in self.candidates:
            try:
                A = host.upload("afl", tuning=tuning_code(*cand))
            except HlrError:
                continue  # a layout this matrix does not fit (e.g. wide codes in small pieces)
            try:
                info = A.info
                ms[cand] = _time(A, nrhs, self.reps, torch, self.multi)
            finally:
                A.free()
        best = min(ms, key=ms.get)
        rc = rank_class(info, nrhs)
        self.table[rc] = best
        return Result(best, ms, rc)

    def choose(self, host, nrhs: int = 1):
        """The tuning code for `host` at `nrhs` columns: the stored choice of its rank class, or
        (first matrix of a class) the result of timing every candidate on it. Returns
        (tuning code, rank class, Result or None when the class was known)."""
        A = host.upload("afl")
        try:
            rc = rank_class(A.info, nrhs)
        finally:
            A.free()
        if rc in self.table:
            return tuning_code(*self.table[rc]), rc, None
        res = self.tune(host, nrhs)
        return tuning_code(*res.best), res.rank_class, res
