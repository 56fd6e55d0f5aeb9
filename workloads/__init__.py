"""Seeded synthetic problem generators shared by the oracle tests, the GPU tests and the bench.

This module draws random problems and nothing else: it holds none of the solver's
arithmetic (no objectives, no dual points, no screening).  Every generator returns the
matrix and data in float32 -- the precision the GPU path stores them in -- so both the
CPU oracle (which reads them as float64) and the CUDA path see bit-identical problems.

Shapes and value distributions follow the experiments of Dantas, Soubies and Fevotte,
"Accelerating Non-Negative and Bounded-Variable Linear Regression Algorithms with Safe
Screening" (Section 5, Tables 1 and 2) and the single-instance / batched workloads built
on them.  All randomness comes from ``numpy.random.default_rng(seed)`` (PCG64).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Problem",
    "nnls_gaussian",
    "nnls_abs_gaussian",
    "bvls_table2",
    "bvls_dirichlet_shared",
    "nnls_shared",
    "bvls_box_shared",
    "mixed_uneven",
    "bvls_gaussian_box",
    "random_tiny",
]


@dataclass
class Problem:
    """One box-constrained least-squares instance  min 1/2||y - A x||^2,  l <= x <= u.

    A is (m, n) float32, C-contiguous in numpy's row-major sense; callers that need the
    column-major layout use ``A.T`` (which is then column-contiguous) or ``np.asfortranarray``.
    y is (m,) float32 for one instance or (B, m) float32 for a batch sharing A.
    l and u are float64 (u may hold +inf).  ``x_true`` is the planted coefficient vector
    (or batch), kept only for reporting.
    """

    name: str
    A: np.ndarray
    y: np.ndarray
    l: np.ndarray
    u: np.ndarray
    x_true: np.ndarray
    meta: dict = field(default_factory=dict)

    @property
    def m(self) -> int:
        return self.A.shape[0]

    @property
    def n(self) -> int:
        return self.A.shape[1]

    @property
    def is_nnls(self) -> bool:
        return bool(np.all(self.l == 0.0) and np.all(np.isinf(self.u)))


def _unit_columns(A: np.ndarray) -> np.ndarray:
    nrm = np.linalg.norm(A, axis=0)
    nrm[nrm == 0.0] = 1.0
    return A / nrm


def _sparse_support(rng, n: int, density: float) -> np.ndarray:
    k = max(1, int(round(density * n)))
    return rng.choice(n, size=k, replace=False)


def nnls_gaussian(m: int, n: int, density: float, noise: float, seed: int,
                  name: str | None = None) -> Problem:
    """NNLS with an iid N(0,1) matrix whose columns are scaled to unit norm.

    x_true has ``density*n`` nonzeros ~ U[0,1] at random positions and
    y = A x_true + N(0, noise^2).  With n >= 2m this family is degenerate (the optimum
    interpolates y), which is the single-instance FP32 workload shape.
    """
    rng = np.random.default_rng(seed)
    A = _unit_columns(rng.standard_normal((m, n)))
    x = np.zeros(n)
    supp = _sparse_support(rng, n, density)
    x[supp] = rng.uniform(0.0, 1.0, size=supp.size)
    y = A @ x + noise * rng.standard_normal(m)
    return Problem(name or f"nnls_gauss_{m}x{n}_s{seed}", A.astype(np.float32),
                   y.astype(np.float32), np.zeros(n), np.full(n, np.inf), x,
                   dict(family="nnls_gaussian", m=m, n=n, density=density, noise=noise, seed=seed))


def nnls_abs_gaussian(m: int, n: int, density: float, noise: float, seed: int,
                      normalize: bool = True, name: str | None = None) -> Problem:
    """NNLS with a_ij = |eta|, eta ~ N(0,1) (the Table 1 family of Section 5).

    x_true has ``density*n`` nonzeros distributed like the entries of A (|N(0,1)|);
    y = A x_true + N(0, noise^2).  ``normalize`` scales the columns to unit norm.
    Nonnegative A has a strictly interior dual direction (t = -1), so the dual
    translation of Section 4.2 applies and screening is effective.
    """
    rng = np.random.default_rng(seed)
    A = np.abs(rng.standard_normal((m, n)))
    if normalize:
        A = _unit_columns(A)
    x = np.zeros(n)
    supp = _sparse_support(rng, n, density)
    x[supp] = np.abs(rng.standard_normal(supp.size))
    y = A @ x + noise * rng.standard_normal(m)
    return Problem(name or f"nnls_abs_{m}x{n}_s{seed}", A.astype(np.float32),
                   y.astype(np.float32), np.zeros(n), np.full(n, np.inf), x,
                   dict(family="nnls_abs_gaussian", m=m, n=n, density=density, noise=noise,
                        seed=seed, normalize=normalize))


def bvls_table2(m: int, n: int, seed: int, density: float = 0.05, noise: float = 1.0,
                normalize: bool = True, name: str | None = None) -> Problem:
    """BVLS with a_ij = |N(0,1)|, box [0,1] (the Table 2 family of Section 5).

    x_true has ``density*n`` nonzeros ~ U(0,1); y = A x_true + N(0, noise^2).
    """
    rng = np.random.default_rng(seed)
    A = np.abs(rng.standard_normal((m, n)))
    if normalize:
        A = _unit_columns(A)
    x = np.zeros(n)
    supp = _sparse_support(rng, n, density)
    x[supp] = rng.uniform(0.0, 1.0, size=supp.size)
    y = A @ x + noise * rng.standard_normal(m)
    return Problem(name or f"bvls_t2_{m}x{n}_s{seed}", A.astype(np.float32),
                   y.astype(np.float32), np.zeros(n), np.ones(n), x,
                   dict(family="bvls_table2", m=m, n=n, density=density, noise=noise,
                        seed=seed, normalize=normalize))


def bvls_gaussian_box(m: int, n: int, box: float, seed: int, name: str | None = None) -> Problem:
    """BVLS with a_ij, y_i ~ N(0,1) and the box b[-1,1] (the saturation-ratio study of Section 5)."""
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((m, n))
    y = rng.standard_normal(m)
    return Problem(name or f"bvls_box{box:g}_{m}x{n}_s{seed}", A.astype(np.float32),
                   y.astype(np.float32), np.full(n, -box), np.full(n, box), np.zeros(n),
                   dict(family="bvls_gaussian_box", m=m, n=n, box=box, seed=seed))


def bvls_dirichlet_shared(m: int, n: int, B: int, k_support: int, noise: float, seed: int,
                          name: str | None = None) -> Problem:
    """Batch of BVLS problems sharing one matrix: A ~ U[0,1] with unit-norm columns, box [0,1].

    Each right-hand side is y_b = A x_b + N(0, noise^2) where x_b puts Dirichlet(1,...,1)
    weights on ``k_support`` random columns (weights already lie in [0,1]).
    Returns y of shape (B, m) and x_true of shape (B, n).
    """
    rng = np.random.default_rng(seed)
    A = _unit_columns(rng.uniform(0.0, 1.0, size=(m, n)))
    X = np.zeros((B, n))
    for b in range(B):
        supp = rng.choice(n, size=k_support, replace=False)
        X[b, supp] = rng.dirichlet(np.ones(k_support))
    Y = X @ A.T + noise * rng.standard_normal((B, m))
    return Problem(name or f"bvls_dir_{m}x{n}_B{B}_s{seed}", A.astype(np.float32),
                   Y.astype(np.float32), np.zeros(n), np.ones(n), X,
                   dict(family="bvls_dirichlet_shared", m=m, n=n, B=B, k_support=k_support,
                        noise=noise, seed=seed))


def nnls_shared(m: int, n: int, B: int, density: float, noise: float, seed: int, abs_matrix: bool = True,
                x_low: float = 0.0, name: str | None = None) -> Problem:
    """Batch of NNLS problems sharing one matrix with unit-norm columns.

    A has entries |N(0,1)| (``abs_matrix``, the Table 1 family) or N(0,1).  Each x_b has
    ``density*n`` nonzeros ~ U[x_low, 1] at random positions and y_b = A x_b + N(0, noise^2).
    Returns y of shape (B, m) and x_true of shape (B, n).
    """
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((m, n))
    A = _unit_columns(np.abs(G) if abs_matrix else G)
    X = np.zeros((B, n))
    for b in range(B):
        supp = _sparse_support(rng, n, density)
        X[b, supp] = rng.uniform(x_low, 1.0, size=supp.size)
    Y = X @ A.T + noise * rng.standard_normal((B, m))
    kind = "abs" if abs_matrix else "gauss"
    return Problem(name or f"nnls_{kind}_shared_{m}x{n}_B{B}_s{seed}", A.astype(np.float32),
                   Y.astype(np.float32), np.zeros(n), np.full(n, np.inf), X,
                   dict(family="nnls_shared", m=m, n=n, B=B, density=density, noise=noise, seed=seed,
                        abs_matrix=abs_matrix, x_low=x_low))


def bvls_box_shared(m: int, n: int, B: int, box: float, seed: int, name: str | None = None) -> Problem:
    """Batch of BVLS problems sharing an N(0,1) matrix, y_b ~ N(0,1), box [-box, box]."""
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((m, n))
    Y = rng.standard_normal((B, m))
    return Problem(name or f"bvls_box{box:g}_shared_{m}x{n}_B{B}_s{seed}", A.astype(np.float32),
                   Y.astype(np.float32), np.full(n, -box), np.full(n, box), np.zeros((B, n)),
                   dict(family="bvls_box_shared", m=m, n=n, B=B, box=box, seed=seed))


def mixed_uneven(B: int, seed: int, m_lo: int = 64, m_hi: int = 1024, abs_matrix: bool = False,
                 noise: float = 0.01, density: float = 0.10) -> list[Problem]:
    """Batch of independent problems of uneven sizes (each with its own matrix).

    m_k ~ U{m_lo..m_hi}, n_k ~ U{2 m_k..8 m_k}; A_k iid N(0,1) (|N(0,1)| with ``abs_matrix``)
    with unit-norm columns; x_k has ``density * n_k`` nonzeros.  Even k: NNLS (l = 0,
    u = +inf), nonzeros ~ U[0,1].  Odd k: BVLS on [-1, 1], nonzeros ~ U[-1,1] of which 20%
    are set to +-1.  y_k = A_k x_k + N(0, noise^2).
    """
    rng = np.random.default_rng(seed)
    out = []
    for k in range(B):
        m = int(rng.integers(m_lo, m_hi + 1))
        n = int(rng.integers(2 * m, 8 * m + 1))
        G = rng.standard_normal((m, n))
        A = _unit_columns(np.abs(G) if abs_matrix else G)
        x = np.zeros(n)
        supp = _sparse_support(rng, n, density)
        if k % 2 == 0:
            x[supp] = rng.uniform(0.0, 1.0, supp.size)
            l, u = np.zeros(n), np.full(n, np.inf)
        else:
            x[supp] = rng.uniform(-1.0, 1.0, supp.size)
            sat = supp[rng.random(supp.size) < 0.2]
            x[sat] = rng.choice([-1.0, 1.0], sat.size)
            l, u = np.full(n, -1.0), np.full(n, 1.0)
        y = A @ x + noise * rng.standard_normal(m)
        out.append(Problem(f"mixed_{k}_{m}x{n}", A.astype(np.float32), y.astype(np.float32), l, u, x,
                           dict(family="mixed_uneven", m=m, n=n, k=k, seed=seed, abs_matrix=abs_matrix,
                                noise=noise)))
    return out


def random_tiny(m: int, n: int, kind: str, seed: int) -> Problem:
    """Small random problems for brute-force comparisons.

    kind: "nnls_abs" (|N| matrix, NNLS), "nnls_gauss" (N(0,1), NNLS),
    "bvls" (N(0,1), box [-1,1]) or "mixed" (N(0,1), half the columns [0,inf), half [-1,1]).
    """
    rng = np.random.default_rng(seed)
    if kind == "nnls_abs":
        A = np.abs(rng.standard_normal((m, n)))
        x = np.abs(rng.standard_normal(n)) * (rng.random(n) < 0.4)
        y = A @ x + rng.standard_normal(m)
        l, u = np.zeros(n), np.full(n, np.inf)
    elif kind == "nnls_gauss":
        A = rng.standard_normal((m, n))
        x = np.abs(rng.standard_normal(n))
        y = A @ x + rng.standard_normal(m)
        l, u = np.zeros(n), np.full(n, np.inf)
    elif kind == "bvls":
        A = rng.standard_normal((m, n))
        x = rng.uniform(-1.5, 1.5, n)
        y = A @ x + 0.5 * rng.standard_normal(m)
        l, u = np.full(n, -1.0), np.full(n, 1.0)
    elif kind == "mixed":
        A = rng.standard_normal((m, n))
        x = rng.uniform(-1.5, 1.5, n)
        y = A @ x + 0.5 * rng.standard_normal(m)
        h = n // 2
        l = np.concatenate([np.zeros(h), np.full(n - h, -1.0)])
        u = np.concatenate([np.full(h, np.inf), np.full(n - h, 1.0)])
    else:
        raise ValueError(kind)
    return Problem(f"tiny_{kind}_{m}x{n}_s{seed}", A.astype(np.float32), y.astype(np.float32),
                   l, u, x, dict(family=f"tiny_{kind}", m=m, n=n, seed=seed))
