"""Seeded synthetic inputs for the H2-MG solver (points, right-hand sides, surfaces).

This module only synthesises inputs. It holds none of the solver's arithmetic: no
kernel evaluation, no tree, no interpolation, no linear algebra of the method. Both
the CPU oracle and the CUDA path take their inputs from here and nowhere else.

Seeds follow one fixed recipe: points use ``default_rng(1000 + k)``, right-hand
sides ``default_rng(2000 + k)`` and the spherical-harmonic coefficients of surface
problem ``j`` use ``default_rng(3000 + j)``, where ``k`` is the workload number
below.

Workloads (shapes and value distributions of the paper's experiments, Section 4,
restated as concrete synthetic problems):

* ``W1``: 4096 points uniform in the unit square; exponential kernel
  exp(-r/0.1) plus 1e-2 on the diagonal; leaf 64; 4x4 Chebyshev nodes; eta 1;
  one N(0,1) right-hand side; relative residual 1e-8.
* ``W2``: 2^20 points uniform in the unit cube; Gaussian kernel
  exp(-r^2/0.05^2) plus 1e-3; leaf 64; 4x4x4 nodes; eta 1; relative residual 1e-10.
* ``W3``: perturbed icospheres (single-layer kernel on panel centroids, weights =
  panel areas); a shared m=57 sphere with 64 right-hand sides and 32 problems of
  log-uniform size in [2^12, 2^16]; leaf 64; 4x4x4 nodes.
* ``W4``: 2^18 points uniform in the unit cube; Matern-3/2 kernel, length 0.1,
  nugget 1e-2 (and the same at 2^12 for dense checks).
* ``W5``: 2^23 points uniform in the unit cube; Gaussian exp(-r^2/0.02^2) plus
  1e-3; leaf 128; 5x5x5 nodes; 16 right-hand sides.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "WORKLOADS",
    "uniform_points",
    "tensor_grid",
    "normal_rhs",
    "perturbed_icosphere",
    "surface_problem_sizes",
    "workload",
]


def uniform_points(n: int, dim: int, k: int) -> np.ndarray:
    """``n`` points i.i.d. uniform in the unit ``dim``-cube, seed ``1000 + k``.

    Returns a C-contiguous float64 array of shape (n, dim).
    """
    rng = np.random.default_rng(1000 + k)
    return np.ascontiguousarray(rng.random((n, dim)))


def tensor_grid(m: int) -> np.ndarray:
    """The uniform m x m tensor grid on the unit square (the paper's 2-D workloads,
    Sec. 4.1-4.2): points (i/(m-1), j/(m-1)), i, j = 0..m-1, the first coordinate
    slowest. Shape (m*m, 2), float64."""
    t = np.arange(m, dtype=np.float64) / max(m - 1, 1)
    X, Y = np.meshgrid(t, t, indexing="ij")
    return np.ascontiguousarray(np.stack([X.ravel(), Y.ravel()], axis=1))


def normal_rhs(n: int, k: int, nrhs: int = 1) -> np.ndarray:
    """Right-hand sides i.i.d. N(0,1), seed ``2000 + k``.

    Shape (n,) for one right-hand side, else (n, nrhs) in column-major order
    (Fortran layout), which is the layout the C library expects for several
    right-hand sides.
    """
    rng = np.random.default_rng(2000 + k)
    if nrhs == 1:
        return rng.standard_normal(n)
    return np.asfortranarray(rng.standard_normal((nrhs, n)).T)


# ---------------------------------------------------------------------------
# Perturbed icosphere (surface workload)
# ---------------------------------------------------------------------------

def _icosahedron():
    t = (1.0 + math.sqrt(5.0)) / 2.0
    v = np.array([
        [-1, t, 0], [1, t, 0], [-1, -t, 0], [1, -t, 0],
        [0, -1, t], [0, 1, t], [0, -1, -t], [0, 1, -t],
        [t, 0, -1], [t, 0, 1], [-t, 0, -1], [-t, 0, 1],
    ], dtype=np.float64)
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    f = np.array([
        [0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
        [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
        [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
        [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1],
    ], dtype=np.int64)
    return v, f


def _real_sph_harm_table(nmax: int, theta: np.ndarray, phi: np.ndarray) -> np.ndarray:
    """Orthonormal real spherical harmonics Y_nm, n <= nmax, |m| <= n.

    theta is the polar angle, phi the azimuth. Returns an array of shape
    ((nmax+1)^2, len(theta)) ordered by (n, m) with m from -n to n. Associated
    Legendre values come from the standard three-term recurrence (no
    Condon-Shortley phase), which is enough for a smooth random perturbation.
    """
    x = np.cos(theta)
    s = np.sqrt(np.maximum(0.0, 1.0 - x * x))
    # P[n][m] for m <= n
    P = [[None] * (nmax + 1) for _ in range(nmax + 1)]
    P[0][0] = np.ones_like(x)
    for m in range(1, nmax + 1):
        P[m][m] = (2 * m - 1) * s * P[m - 1][m - 1]
    for m in range(0, nmax):
        P[m + 1][m] = (2 * m + 1) * x * P[m][m]
    for m in range(0, nmax + 1):
        for n in range(m + 2, nmax + 1):
            P[n][m] = ((2 * n - 1) * x * P[n - 1][m] - (n + m - 1) * P[n - 2][m]) / (n - m)
    out = []
    for n in range(nmax + 1):
        for m in range(-n, n + 1):
            am = abs(m)
            norm = math.sqrt((2 * n + 1) / (4 * math.pi)
                             * math.factorial(n - am) / math.factorial(n + am))
            if m == 0:
                out.append(norm * P[n][0])
            elif m > 0:
                out.append(math.sqrt(2.0) * norm * P[n][am] * np.cos(am * phi))
            else:
                out.append(math.sqrt(2.0) * norm * P[n][am] * np.sin(am * phi))
    return np.array(out)


def perturbed_icosphere(m: int, j: int, amplitude: float = 0.2, degree: int = 8):
    """Triangulated perturbed sphere for surface problem ``j``.

    A geodesic icosahedron of frequency ``m``: every face of the icosahedron is
    split into m^2 triangles and the vertices are projected to the unit sphere,
    giving N = 20 m^2 panels. Each vertex is moved to radius
    1 + amplitude * h(direction), where h is a sum of real spherical harmonics of
    degree <= ``degree`` with N(0,1) coefficients (seed ``3000 + j``), scaled so
    that max |h| over the vertices is 1.

    Returns ``(centroids (N,3), areas (N,), vertices (N,3,3))`` of the perturbed
    panels.
    """
    if m < 1:
        raise ValueError("frequency m must be >= 1")
    v0, faces = _icosahedron()
    # Barycentric lattice on each face: lattice point (a, b) with a + b <= m.
    tri = []
    for (ia, ib, ic) in faces:
        A, B, C = v0[ia], v0[ib], v0[ic]

        def pt(a, b):
            return A + (B - A) * (a / m) + (C - A) * (b / m)

        for a in range(m):
            for b in range(m - a):
                tri.append((pt(a, b), pt(a + 1, b), pt(a, b + 1)))
                if a + b < m - 1:
                    tri.append((pt(a + 1, b), pt(a + 1, b + 1), pt(a, b + 1)))
    verts = np.array(tri, dtype=np.float64)            # (N, 3, 3)
    dirs = verts / np.linalg.norm(verts, axis=2, keepdims=True)
    flat = dirs.reshape(-1, 3)
    theta = np.arccos(np.clip(flat[:, 2], -1.0, 1.0))
    phi = np.arctan2(flat[:, 1], flat[:, 0])
    Y = _real_sph_harm_table(degree, theta, phi)
    rng = np.random.default_rng(3000 + j)
    coef = rng.standard_normal(Y.shape[0])
    h = coef @ Y
    h = h / np.max(np.abs(h))
    radius = 1.0 + amplitude * h
    pv = (flat * radius[:, None]).reshape(verts.shape)
    centroids = pv.mean(axis=1)
    cr = np.cross(pv[:, 1] - pv[:, 0], pv[:, 2] - pv[:, 0])
    areas = 0.5 * np.linalg.norm(cr, axis=1)
    return np.ascontiguousarray(centroids), areas, pv


def surface_problem_sizes(count: int = 32, lo: int = 2 ** 12, hi: int = 2 ** 16):
    """Frequencies m_j of the uneven surface problems of workload W3.

    Target sizes are drawn log-uniform in [lo, hi] (seed 1003); each becomes the
    frequency m = round(sqrt(N/20)) of a geodesic sphere, whose actual size is
    20 m^2.
    """
    rng = np.random.default_rng(1003)
    target = np.exp(rng.uniform(math.log(lo), math.log(hi), size=count))
    return [max(1, int(round(math.sqrt(t / 20.0)))) for t in target]


# ---------------------------------------------------------------------------
# Workload table
# ---------------------------------------------------------------------------

WORKLOADS = {
    1: dict(name="exp2d_n4096", n=4096, dim=2, kernel="exponential", length=0.1,
            nugget=1e-2, leaf=64, q=4, eta=1.0, tol=1e-8, nrhs=1),
    2: dict(name="gauss3d_n1048576", n=2 ** 20, dim=3, kernel="gaussian", length=0.05,
            nugget=1e-3, leaf=64, q=4, eta=1.0, tol=1e-10, nrhs=1),
    3: dict(name="sphere_sl_m57", m=57, dim=3, kernel="laplace_sl", length=1.0,
            nugget=0.0, leaf=64, q=4, eta=1.0, tol=1e-10, nrhs=64, problems=32),
    4: dict(name="matern3d_n262144", n=2 ** 18, dim=3, kernel="matern32", length=0.1,
            nugget=1e-2, leaf=64, q=4, eta=1.0, tol=1e-10, nrhs=1),
    5: dict(name="gauss3d_n8388608", n=2 ** 23, dim=3, kernel="gaussian", length=0.02,
            nugget=1e-3, leaf=128, q=5, eta=1.0, tol=1e-10, nrhs=16),
}


def workload(k: int, n: int | None = None):
    """Points and right-hand side(s) of workload ``k`` (optionally at size ``n``).

    For the point-cloud workloads returns ``dict(points, b, **params)``. For the
    surface workload returns the shared sphere with its areas as ``weights`` and
    the per-panel diagonal inputs (areas) so each side can form its own diagonal.
    """
    p = dict(WORKLOADS[k])
    if k == 3:
        c, a, _ = perturbed_icosphere(p["m"], 0)
        p.update(points=c, weights=a, n=c.shape[0])
        p["b"] = normal_rhs(c.shape[0], k, p["nrhs"])
        return p
    if n is not None:
        p["n"] = int(n)
    p["points"] = uniform_points(p["n"], p["dim"], k)
    p["b"] = normal_rhs(p["n"], k, p["nrhs"] if n is None else 1)
    return p
