"""Seeded synthetic inputs for the compressed H-matrix-vector product.

This module is shared by the CPU oracle (``oracle/``) and by the GPU path's callers
(tests, ``bench.py``). It generates only the *problem*: point sets, kernel functions
evaluated on index sets, the diagonal shift of the sphere problems, and right-hand sides.
It holds none of the method's arithmetic: no cluster or block trees, no lowrank
approximation, no compression, no products.

Workload recipes (synthetic stand-ins for the paper's model problems of Section 5.1; the
paper's BEM and Matern matrices themselves cannot be reproduced here):

* ``exp2d``    : n points uniform in [0,1]^2 (``default_rng(seed)``), K(x,y) = exp(-|x-y|/0.2),
                 plus ``nugget`` on the diagonal (1e-2).
* ``laplace``  : n Fibonacci points on the unit sphere, K(x,y) = 1/(4 pi |x-y|) off the
                 diagonal, the diagonal set to ``diag`` (mean off-diagonal row sum, see
                 :func:`laplace_mean_row_sum`).  Stand-in for the single layer potential, Eq. 3.
* ``matern15`` : n points uniform in the unit cube, Matern covariance with nu = 3/2 and
                 sigma^2 = 1 in closed form, C(d) = (1 + sqrt(3) d / l) exp(-sqrt(3) d / l),
                 l = 0.1, plus a nugget 1e-2 on the diagonal.  Stand-in for Eq. 4 (which the
                 paper evaluates with nu = 1/3).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Problem", "uniform_square", "uniform_cube", "fibonacci_sphere", "laplace_mean_row_sum",
    "rhs", "exp2d_problem", "laplace_problem", "matern_problem", "batch_sizes",
]


def uniform_square(n: int, seed: int = 0) -> np.ndarray:
    """n points uniform in [0,1]^2 from ``numpy.random.default_rng(seed)`` (shape n x 2)."""
    return np.random.default_rng(seed).uniform(size=(n, 2))


def uniform_cube(n: int, seed: int) -> np.ndarray:
    """n points uniform in [0,1]^3 from ``numpy.random.default_rng(seed)`` (shape n x 3)."""
    return np.random.default_rng(seed).uniform(size=(n, 3))


def fibonacci_sphere(n: int) -> np.ndarray:
    """n Fibonacci points on the unit sphere.

    z_i = 1 - (2i+1)/n, r_i = sqrt(1 - z_i^2), phi_i = i * pi * (3 - sqrt 5),
    x_i = (r_i cos phi_i, r_i sin phi_i, z_i).
    """
    i = np.arange(n, dtype=np.float64)
    z = 1.0 - (2.0 * i + 1.0) / n
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    phi = i * (math.pi * (3.0 - math.sqrt(5.0)))
    return np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1)


def rhs(n: int, seed: int, nrhs: int | None = None) -> np.ndarray:
    """Right-hand side(s) x ~ N(0,1) from ``default_rng(seed)``.

    ``nrhs=None`` gives a vector of length n; otherwise an n x nrhs array stored
    column-major (Fortran order), column j being the j-th right-hand side.
    """
    g = np.random.default_rng(seed)
    if nrhs is None:
        return g.standard_normal(n)
    return np.asfortranarray(g.standard_normal((nrhs, n)).T)


def _distances(P: np.ndarray, Q: np.ndarray) -> np.ndarray:
    d = np.zeros((P.shape[0], Q.shape[0]))
    for k in range(P.shape[1]):
        diff = P[:, k][:, None] - Q[:, k][None, :]
        d += diff * diff
    return np.sqrt(d)


@dataclass
class Problem:
    """A kernel matrix K[i, j] = k(p_i, p_j) (+ diagonal term) over a point set.

    ``kind`` is one of ``"exp2d"``, ``"laplace"``, ``"matern15"``; ``params`` holds the
    kernel's scalars (``scale`` for the length, ``diag`` for the diagonal term: the nugget
    added on the diagonal for exp2d/matern15, the diagonal value itself for laplace).
    """
    kind: str
    points: np.ndarray
    params: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return self.points.shape[0]

    def entries(self, I: np.ndarray, J: np.ndarray) -> np.ndarray:
        """K restricted to rows I and columns J (original point indices), FP64."""
        I = np.asarray(I, dtype=np.int64)
        J = np.asarray(J, dtype=np.int64)
        r = _distances(self.points[I], self.points[J])
        same = I[:, None] == J[None, :]
        diag = float(self.params.get("diag", 0.0))
        if self.kind == "exp2d":
            K = np.exp(-r / self.params["scale"])
            return K + np.where(same, diag, 0.0)
        if self.kind == "matern15":
            a = math.sqrt(3.0) * r / self.params["scale"]
            K = (1.0 + a) * np.exp(-a)
            return K + np.where(same, diag, 0.0)
        if self.kind == "laplace":
            with np.errstate(divide="ignore"):
                K = 1.0 / (4.0 * math.pi * r)
            return np.where(same, diag, K)
        raise ValueError(f"unknown kernel {self.kind}")


def laplace_mean_row_sum(points: np.ndarray, sample: int = 1024, seed: int = 7,
                         exact_below: int = 8192) -> float:
    """Diagonal value of the sphere problems: mean over rows of the off-diagonal row sums
    of 1/(4 pi |x-y|).

    Exact (all rows) for n <= ``exact_below``; otherwise the mean over ``sample`` rows
    drawn without replacement by ``default_rng(seed)``, each row summed over all columns.
    """
    n = points.shape[0]
    if n <= exact_below:
        rows = np.arange(n)
    else:
        rows = np.sort(np.random.default_rng(seed).choice(n, size=sample, replace=False))
    total = 0.0
    for c0 in range(0, len(rows), 16):
        I = rows[c0:c0 + 16]
        r = _distances(points[I], points)
        r[np.arange(len(I)), I] = np.inf
        total += float(np.sum(1.0 / (4.0 * math.pi * r)))
    return total / len(rows)


def exp2d_problem(n: int = 4096, seed: int = 0) -> Problem:
    """Small 2D case: uniform points in [0,1]^2, exp(-r/0.2) + 1e-2 I."""
    return Problem("exp2d", uniform_square(n, seed), {"scale": 0.2, "diag": 1e-2})


def laplace_problem(n: int = 262144, diag: float | None = None) -> Problem:
    """Fibonacci sphere, 1/(4 pi r) off the diagonal, diagonal = mean row sum."""
    P = fibonacci_sphere(n)
    if diag is None:
        diag = laplace_mean_row_sum(P)
    return Problem("laplace", P, {"diag": float(diag)})


def matern_problem(n: int, seed: int, scale: float = 0.1, nugget: float = 1e-2) -> Problem:
    """Unit-cube points (``default_rng(seed)``), Matern nu=3/2 with length ``scale`` + nugget."""
    return Problem("matern15", uniform_cube(n, seed), {"scale": scale, "diag": nugget})


def batch_sizes(count: int = 48, lo: int = 8192, hi: int = 131072, seed: int = 3) -> list[int]:
    """Matrix sizes n = round(exp(U(ln lo, ln hi))) from ``default_rng(seed)`` for the batched case."""
    g = np.random.default_rng(seed)
    return [int(round(math.exp(v))) for v in g.uniform(math.log(lo), math.log(hi), size=count)]


def batch_nrhs(count: int = 48, seed: int = 4) -> list[int]:
    """Right-hand-side counts drawn from {1, 8, 32} by ``default_rng(seed)`` for the batched case."""
    g = np.random.default_rng(seed)
    return [int(v) for v in g.choice([1, 8, 32], size=count)]
