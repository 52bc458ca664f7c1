"""Nested cluster bases by recursive skeletonization (interpolative decompositions),
the tolerance-driven construction of the oracle's H2 matrices.

Test infrastructure: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` leg of ``bench.py`` may import this package.

The paper builds its H2 matrices with an external algebraic method to a relative
accuracy eps = 1e-9 with adaptive ranks (Sec. 4.1: "matrices constructed with
relative accuracy"; Sec. 4.2 likewise). This module is the oracle's reading of such
a construction. Every cluster gets a *skeleton*: a subset of its points such that
the cluster's far-field rows are interpolated from the skeleton's rows,

    A(X_tau, F_tau) ~= T_tau A(skel_tau, F_tau),    T_tau[skel_tau, :] = I,

and the skeletons are nested: a leaf chooses among its own points, a parent among
the union of its children's skeletons (its *candidates*). This gives the same three
ingredients as Chebyshev interpolation, with skeleton points in place of nodes:
the leaf basis U = T_leaf, the transfer E_c = the rows of T_parent that belong to
child c's skeleton, and the coupling S_tau,sigma = A(skel_tau, skel_sigma). The
orthonormalisation chain of Sec. 3.3 then runs unchanged on these factors.

Steps for a cluster tau at tree level ell (levels L down to t*):

1. candidates: the leaf's points in tree order (ell = L), else the skeleton of the
   first child followed by the skeleton of the second;
2. far-field sample F_tau, in this order: the candidates of every far partner sigma
   of tau at level ell (partners in increasing index), then, for every far partner
   sigma' of tau's parent at level ell - 1 (increasing index), the candidates of
   sigma's two children concatenated and thinned to every s-th entry from the
   first, s = ceil(count / 128);
3. W = A(F_tau, candidates)  (|F| x |cand|, A_ij = sqrt(w_i) k(x_i, x_j) sqrt(w_j));
   R0 = the R factor of a QR factorisation of W (column geometry of W preserved);
4. greedy column-pivoted Householder QR of R0: at step j the column of largest
   remaining norm is taken (columns within a relative 1e-10 of the largest in
   squared norm count as tied, and the lowest index wins); stop once j = rank_max,
   j = min(rows, |cand|), or the taken column's norm <= tol * (the first pivot's
   norm); r = number of pivots taken (at least one);
5. skeleton = candidates at the first r pivots (in pivot order); with R11, R12 the
   leading blocks of the pivoted R, T[pivot a] = e_a for a < r and, for the other
   candidates (in pivot order), T[pivot r + b] = (R11^{-1} R12)[:, b].

A cluster whose sample is empty (nothing far from it or its parent) keeps its first
min(|cand|, rank_max) candidates with T = [I; 0]; nothing multiplies its basis then.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg as sla

from . import kernels as K

SAMPLE_CAP = 128      # points kept per far partner of the parent (step 2)
TIE = 1e-10           # relative tie band of the pivot choice (step 4)


def pivoted_qr_id(R0: np.ndarray, tol: float, rank_max: int):
    """Steps 4-5 on the small square-or-wide factor R0 (rows x ncand).

    Returns (piv, r, T): the pivot order (all ncand columns), the rank and the
    interpolation matrix T (ncand x r) in the original column order."""
    A = np.array(R0, dtype=np.float64, copy=True)
    m, nc = A.shape
    piv = np.arange(nc)
    kmax = min(rank_max, m, nc)
    r = 0
    first = 0.0
    for j in range(kmax):
        norms = np.sum(A[j:, j:] ** 2, axis=0)
        big = norms.max()
        if j == 0:
            first = math.sqrt(big)
            if first == 0.0:
                break
        elif math.sqrt(big) <= tol * first:
            break
        p = j + int(np.flatnonzero(norms >= big * (1.0 - TIE))[0])
        if p != j:
            A[:, [j, p]] = A[:, [p, j]]
            piv[[j, p]] = piv[[p, j]]
        # Householder reflector on A[j:, j]
        x = A[j:, j].copy()
        alpha = x[0]
        sigma = float(x[1:] @ x[1:])
        if sigma > 0.0:
            beta = -math.copysign(math.sqrt(alpha * alpha + sigma), alpha)
            v = x / (alpha - beta)
            v[0] = 1.0
            tau = (beta - alpha) / beta
            A[j:, j + 1:] -= tau * np.outer(v, v @ A[j:, j + 1:])
            A[j, j] = beta
            A[j + 1:, j] = 0.0
        r = j + 1
    r = max(r, 1)
    T = np.zeros((nc, r))
    T[piv[:r], np.arange(r)] = 1.0
    if r < nc and A[0, 0] != 0.0:
        X = sla.solve_triangular(A[:r, :r], A[:r, r:])      # R11^{-1} R12, r x (nc - r)
        T[piv[r:], :] = X.T
    return piv, r, T


def far_partners(far_pairs) -> dict:
    """tau -> sorted list of its far partners sigma (both orders of every pair)."""
    out: dict = {}
    for (t, s) in far_pairs:
        out.setdefault(int(t), []).append(int(s))
    for v in out.values():
        v.sort()
    return out


class Skeletons:
    """Skeletons and interpolation matrices of every cluster at levels t*..L."""

    def __init__(self, tree, far, tstar: int, kspec, sqrt_w_tree: np.ndarray, tol: float,
                 rank_max: int):
        self.tree = tree
        self.tol, self.rank_max = float(tol), int(rank_max)
        Xt = tree.points_tree
        L = tree.L
        self.skel = {}       # (ell, j) -> tree positions of the skeleton, pivot order
        self.T = {}          # (ell, j) -> |cand| x r interpolation matrix
        self.cand = {}       # (ell, j) -> tree positions of the candidates
        self.sampled = {}    # (ell, j) -> False when the far-field sample was empty
        part = {ell: far_partners(far[ell]) for ell in range(tstar, L + 1)}

        def amat(rows, cols):
            B = K.kmat(kspec.kind, Xt[rows], Xt[cols], kspec.length, kspec.degree)
            return sqrt_w_tree[rows][:, None] * B * sqrt_w_tree[cols][None, :]

        for ell in range(L, tstar - 1, -1):
            for j in range(1 << ell):
                if ell == L:
                    c = np.arange(tree.offsets[L][j], tree.offsets[L][j + 1])
                else:
                    c = np.concatenate([self.skel[(ell + 1, 2 * j)], self.skel[(ell + 1, 2 * j + 1)]])
                self.cand[(ell, j)] = c.astype(np.int64)
            for j in range(1 << ell):
                c = self.cand[(ell, j)]
                cols = [self.cand[(ell, s)] for s in part[ell].get(j, [])]
                if ell - 1 >= tstar:
                    for s in part[ell - 1].get(j // 2, []):
                        pts = np.concatenate([self.cand[(ell, 2 * s)], self.cand[(ell, 2 * s + 1)]])
                        step = max(1, -(-len(pts) // SAMPLE_CAP))
                        cols.append(pts[::step])
                F = np.concatenate(cols) if cols else np.zeros(0, np.int64)
                self.sampled[(ell, j)] = len(F) > 0 and len(c) > 0
                if len(F) == 0 or len(c) == 0:
                    r = min(len(c), self.rank_max)
                    T = np.zeros((len(c), r))
                    T[np.arange(r), np.arange(r)] = 1.0
                    self.skel[(ell, j)] = c[:r]
                    self.T[(ell, j)] = T
                    continue
                W = amat(F, c)                                   # |F| x |cand|
                R0 = np.linalg.qr(W, mode="r")
                piv, r, T = pivoted_qr_id(R0, self.tol, self.rank_max)
                self.skel[(ell, j)] = c[piv[:r]]
                self.T[(ell, j)] = T

    def rank(self, ell: int, j: int) -> int:
        return int(self.skel[(ell, j)].shape[0])

    def leaf_basis(self, j: int) -> np.ndarray:
        """U^skel of leaf j: its interpolation matrix (rows = the leaf's points)."""
        return self.T[(self.tree.L, j)]

    def transfer(self, ell: int, c: int) -> np.ndarray:
        """E_c (r_c x r_parent): the rows of the parent's T that belong to child c."""
        p = c // 2
        Tp = self.T[(ell - 1, p)]
        r1 = self.rank(ell, 2 * p)
        return Tp[:r1] if c % 2 == 0 else Tp[r1:]
