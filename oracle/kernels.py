"""Kernel functions k(x, y) of the oracle (plain NumPy, float64).

Test infrastructure: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` leg of ``bench.py`` may import this package.

Kernels (Section 4 of the paper and the synthetic workloads):

* ``gaussian``     exp(-r^2 / l^2)           (Section 4.1, eq. a_gau, with sigma = l^2)
* ``exponential``  exp(-r / l)               (Section 4.2, eq. a_exp, with sigma = l)
* ``matern32``     (1 + sqrt3 r/l) exp(-sqrt3 r/l)
* ``laplace_sl``   1 / (4 pi r)               (Section 4.3, single-layer potential)
* ``poly``         (1 + x.y)^m                (test kernel: a polynomial of degree m
                                               in each variable, reproduced exactly by
                                               Chebyshev interpolation with q > m nodes)
* ``dmatern32_dl`` d/dl of ``matern32`` = (3 r^2 / l^3) exp(-sqrt3 r/l)

The diagonal of the kernel matrix (i == j) is never taken from these formulas
for the singular kernel; see ``diag_value``.
"""
from __future__ import annotations

import math

import numpy as np

KINDS = ("gaussian", "exponential", "matern32", "laplace_sl", "poly", "dmatern32_dl")
SQRT3 = math.sqrt(3.0)


def pairwise_r(X: np.ndarray, Y: np.ndarray) -> np.ndarray:
    """Euclidean distances |x_i - y_j| by explicit differences (no norm expansion)."""
    d = X[:, None, :] - Y[None, :, :]
    return np.sqrt(np.sum(d * d, axis=2))


def kmat(kind: str, X: np.ndarray, Y: np.ndarray, length: float = 1.0,
         degree: int = 2) -> np.ndarray:
    """Matrix of off-diagonal kernel values k(X_i, Y_j)."""
    if kind == "poly":
        return (1.0 + X @ Y.T) ** degree
    r = pairwise_r(X, Y)
    if kind == "gaussian":
        return np.exp(-(r * r) / (length * length))
    if kind == "exponential":
        return np.exp(-r / length)
    if kind == "matern32":
        u = SQRT3 * r / length
        return (1.0 + u) * np.exp(-u)
    if kind == "dmatern32_dl":
        u = SQRT3 * r / length
        return (3.0 * r * r / length ** 3) * np.exp(-u)
    if kind == "laplace_sl":
        with np.errstate(divide="ignore"):
            return 1.0 / (4.0 * math.pi * r)
    raise ValueError(f"unknown kernel {kind!r}")


def self_value(kind: str, X: np.ndarray, length: float = 1.0, degree: int = 2) -> np.ndarray:
    """k(x_i, x_i) for each point (the kernel's value at zero distance)."""
    n = X.shape[0]
    if kind in ("gaussian", "exponential", "matern32"):
        return np.ones(n)
    if kind == "dmatern32_dl":
        return np.zeros(n)
    if kind == "poly":
        return (1.0 + np.sum(X * X, axis=1)) ** degree
    if kind == "laplace_sl":
        return np.full(n, np.inf)   # singular: a diagonal override is required
    raise ValueError(f"unknown kernel {kind!r}")


def diag_value(kind: str, X: np.ndarray, weights, diag, nugget: float, length: float = 1.0,
               degree: int = 2) -> np.ndarray:
    """Diagonal entries A_ii of the kernel matrix.

    A_ii = diag_i + nugget when a per-point override is given (the surface kernel
    of Section 4.3 replaces the singular self-interaction by a geometric value),
    else w_i k(x_i, x_i) + nugget (eqs. a_gau and a_exp: 1 + c).
    """
    if diag is not None:
        return np.asarray(diag, dtype=np.float64) + nugget
    w = np.ones(X.shape[0]) if weights is None else np.asarray(weights, dtype=np.float64)
    return w * self_value(kind, X, length, degree) + nugget


def surface_diag(areas: np.ndarray) -> np.ndarray:
    """Diagonal of the single-layer matrix (Sec. 4.3) in the symmetric scaling
    A_ij = sqrt(a_i a_j) / (4 pi |c_i - c_j|): the panel's self-interaction, taken as
    the potential at the centre of a flat disk of the panel's area a carrying unit
    density, int_disk dA / (4 pi |x - c|) = R / 2 with R = sqrt(a / pi).

    It has the units of the off-diagonal entries (a length). The paper's own choice,
    w_i / (4 pi R_i) with R_i the mean centroid-vertex distance, is about half of it;
    on the perturbed spheres of the surface workload both it and the formula
    a sqrt(a/pi)/2 (an extra factor a) leave the matrix indefinite, while this one
    keeps it positive definite."""
    a = np.asarray(areas, dtype=np.float64)
    return np.sqrt(a / math.pi) / 2.0


def dense_kernel_matrix(kind: str, X: np.ndarray, length: float = 1.0, nugget: float = 0.0,
                        weights=None, diag=None, degree: int = 2) -> np.ndarray:
    """The dense N x N matrix A_ij = sqrt(w_i) k(x_i, x_j) sqrt(w_j), A_ii = diag."""
    K = kmat(kind, X, X, length, degree)
    if weights is not None:
        s = np.sqrt(np.asarray(weights, dtype=np.float64))
        K = s[:, None] * K * s[None, :]
    np.fill_diagonal(K, diag_value(kind, X, weights, diag, nugget, length, degree))
    return K


def kernel_rows(kind: str, X: np.ndarray, rows, length: float = 1.0, nugget: float = 0.0,
                weights=None, diag=None, degree: int = 2, chunk: int = 16) -> np.ndarray:
    """Rows ``rows`` of the dense N x N kernel matrix (A_ij = sqrt(w_i) k(x_i, x_j)
    sqrt(w_j), A_ii = diag), by the formula, ``chunk`` rows at a time: the exact matrix
    that the H2 form approximates, for sampled checks at sizes where the full matrix
    cannot be held."""
    rows = np.asarray(rows, dtype=np.int64)
    X = np.asarray(X, dtype=np.float64)
    w = None if weights is None else np.sqrt(np.asarray(weights, dtype=np.float64))
    dg = diag_value(kind, X[rows], None if weights is None else np.asarray(weights)[rows],
                    None if diag is None else np.asarray(diag)[rows], nugget, length, degree)
    out = np.empty((len(rows), X.shape[0]))
    for a in range(0, len(rows), chunk):
        rr = rows[a:a + chunk]
        with np.errstate(divide="ignore"):
            B = kmat(kind, X[rr], X, length, degree)
        if w is not None:
            B = w[rr][:, None] * B * w[None, :]
        B[np.arange(len(rr)), rr] = dg[a:a + chunk]
        out[a:a + len(rr)] = B
    return out
