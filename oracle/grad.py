"""Gradients of a solve-based loss for the oracle (test infrastructure; see the
package docstring for who may import this module).

L(y, b, theta) = 1/2 y^T A^{-1} y + 1^T A^{-1} b with A the H2 matrix of the
Matern-3/2 kernel (1 + sqrt3 r/l) exp(-sqrt3 r/l) plus nugget s. With a = A^{-1} y,
x = A^{-1} b and w = A^{-1} 1 (A symmetric):
    dL/dy = a,  dL/db = w,  dL/dtheta = -1/2 a^T (dA/dtheta) a - w^T (dA/dtheta) x,
with dA/ds = I and dA/dl the H2 matrix of the derivative kernel (3 r^2/l^3) exp(-sqrt3 r/l).
With Chebyshev bases it is built with the same tree, nodes and orthonormalisation
factors as A: interpolation bases do not depend on theta, so it is the exact derivative of
A's H2 form. Skeleton bases are selected from A's own kernel values and would not
represent the derivative kernel's far field; there dA/dl is the derivative kernel's own
skeleton H2 matrix on A's tree (same tolerance and rank cap), an approximation of the
exact kernel's derivative to that tolerance. The solves here are dense (np.linalg.solve
of the H2 matrix), small N only.
"""
from __future__ import annotations

import copy

import numpy as np

from .h2 import H2Matrix, KernelSpec


def derivative_h2(h: H2Matrix, kspec: KernelSpec) -> H2Matrix:
    """The H2 matrix of kernel ``kspec`` with h's tree and partition: with h's nodes and
    bases (Chebyshev), or with skeletons of its own (skeleton bases)."""
    if h.basis == "skeleton":
        return H2Matrix(h.X, kspec, h.leaf, h.q, h.eta, tree=h.tree, partition=(h.far, h.inadm), basis="skeleton",
                        tol=h.tol, rank_max=h.rank_max)
    d = copy.copy(h)
    d.kspec = kspec
    d._cache = {k: v for k, v in h._cache.items() if k[0] == "off"}
    T = h.tree
    from . import kernels as K
    d.sqrt_w_tree = np.ones(T.n)
    d.diag_tree = K.diag_value(kspec.kind, h.X, None, None, kspec.nugget, kspec.length,
                               kspec.degree)[T.perm]
    d._fill_near()
    if h.tstar is not None:
        d._couplings()
    return d


def matern_loss(points, y, b, length, nugget, leaf=64, q=4, eta=1.0):
    """(L, a, x, A) with dense solves of the oracle's H2 matrix."""
    A = H2Matrix(points, KernelSpec("matern32", length, nugget), leaf, q, eta)
    Ad = A.dense()
    a = np.linalg.solve(Ad, y)
    x = np.linalg.solve(Ad, b)
    return 0.5 * float(y @ a) + float(x.sum()), a, x, A


def matern_grads(points, y, b, length, nugget, leaf=64, q=4, eta=1.0):
    """Closed-form gradients (dL/dy, dL/db, dL/dl, dL/ds) of ``matern_loss``."""
    L, a, x, A = matern_loss(points, y, b, length, nugget, leaf, q, eta)
    Ad = A.dense()
    w = np.linalg.solve(Ad, np.ones_like(b))
    dA = derivative_h2(A, KernelSpec("dmatern32_dl", length, 0.0))
    dl = -0.5 * float(a @ dA.apply(a)) - float(w @ dA.apply(x))
    ds = -0.5 * float(a @ a) - float(w @ x)
    return L, a, w, dl, ds
