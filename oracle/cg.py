"""Unpreconditioned conjugate gradients (oracle; test infrastructure only).

Textbook CG for a symmetric positive definite operator, in FP64 with exactly rounded inner
products; stops when ||r_k|| <= rtol ||b|| (recursive residual) or after maxit iterations.
Used to pin the GPU solver on the decoded operator A~.
"""
from __future__ import annotations

import math

import numpy as np


def _dot(a: np.ndarray, b: np.ndarray) -> float:
    return math.fsum(a * b)


def cg(apply, b: np.ndarray, x0: np.ndarray, rtol: float, maxit: int):
    """Return (x, iterations, recursive relative residual)."""
    x = np.array(x0, dtype=np.float64)
    r = b - apply(x)
    p = r.copy()
    rr = _dot(r, r)
    bnorm = math.sqrt(_dot(b, b))
    if bnorm == 0.0:
        return x, 0, 0.0
    it = 0
    while math.sqrt(rr) > rtol * bnorm and it < maxit:
        Ap = apply(p)
        alpha = rr / _dot(p, Ap)
        x = x + alpha * p
        r = r - alpha * Ap
        rr_new = _dot(r, r)
        p = r + (rr_new / rr) * p
        rr = rr_new
        it += 1
    return x, it, math.sqrt(rr) / bnorm
