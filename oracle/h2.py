"""H2 matrix of the oracle: cluster tree, block partition, Chebyshev nested bases,
orthonormalisation, matrix-vector product and the Galerkin coarse operators.

Test infrastructure: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` leg of ``bench.py`` may import this package. It is a plain, slow,
float64 restatement of the paper; it shares no code with the CUDA library.

Notation (Section 3.1 of the paper). The matrix is A = D + U_1 S_1 V_1 (eq. h20 and
the line after it), and recursively S_1 = D_2 + U_2 S_2 V_2 (eq. s1), giving the
H2 form A = D + U_1 (D_2 + U_2 (... (D_l + U_l S_l V_l) ...) V_2) V_1 (eq. h2).
For a symmetric kernel V_i = U_i^T. Tree levels are counted from the root
(ell = 0) to the leaves (ell = L). Multigrid level i = 1 is the point level; for
i >= 2 the level-i space X_i is the coefficient space of tree level
m(i) = L - i + 2, so X_2 holds the leaf coefficients x_1 = V_1 x.

Readings where the paper leaves the construction open (it uses an external
algebraic H2 builder):

* tree: recursive bisection of every cluster above depth L = ceil(log2(N/leaf))
  along the axis of largest tight-box extent (ties: lowest axis); the cluster's
  points are ordered by (coordinate, original index) and the first ceil(n/2) go
  to the left child;
* block partition (Section 3.1, close/far blocks): a pair of clusters is far
  (admissible) when the boxes are apart (dist > 0) and
  max(diam_tau, diam_sigma) <= eta * dist; pairs are refined from (root, root)
  until far or both are leaves (close);
* bases: tensor Chebyshev interpolation with q first-kind nodes per dimension on
  each tight box (half-width floored at 1e-12 of the root extent); leaf basis
  U^cheb[i, a] = sqrt(w_i) L_a(x_i), transfer E_c[a, b] = L^P_b(xi^c_a), coupling
  S^cheb = k(xi_tau, xi_sigma);
* orthonormal bases (the restriction argument of Section 3.3 uses orthogonal U):
  QR of the leaf bases and of the stacked [R_c1 E_c1; R_c2 E_c2] of each parent,
  with diag(R) >= 0; couplings become R_tau S^cheb R_sigma^T. This changes the
  basis, not the matrix. Ranks are r = min(k, rows), never truncated.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import kernels as K


# ---------------------------------------------------------------------------
# Cluster tree
# ---------------------------------------------------------------------------

class ClusterTree:
    """Complete binary cluster tree of uniform depth L (see the module docstring).

    Attributes
    ----------
    perm : perm[p] = original index of the point at tree position p
    offsets[ell] : start offsets (length 2^ell + 1) of the clusters of level ell
    lo[ell], hi[ell] : tight boxes of the clusters of level ell, shape (2^ell, dim)
    """

    def __init__(self, points: np.ndarray, leaf: int):
        X = np.asarray(points, dtype=np.float64)
        n, dim = X.shape
        if n < 1 or leaf < 1:
            raise ValueError("need n >= 1 and leaf >= 1")
        L = 0 if n <= leaf else int(math.ceil(math.log2(n / leaf)))
        # guard against floating round-off in log2
        while (n + (1 << L) - 1) >> L > leaf:
            L += 1
        while L > 0 and (n + (1 << (L - 1)) - 1) >> (L - 1) <= leaf:
            L -= 1
        self.n, self.dim, self.L, self.leaf = n, dim, L, leaf
        order = np.arange(n)
        offsets = [np.array([0, n], dtype=np.int64)]
        self.split_axis = []
        for ell in range(L):
            off = offsets[ell]
            nxt = [0]
            axes = np.zeros(1 << ell, dtype=np.int64)
            for j in range(1 << ell):
                a, b = off[j], off[j + 1]
                seg = order[a:b]
                P = X[seg]
                ext = P.max(axis=0) - P.min(axis=0)
                axis = int(np.argmax(ext))           # first maximum = lowest axis on ties
                axes[j] = axis
                idx = np.lexsort((seg, P[:, axis]))  # primary: coordinate, then original index
                order[a:b] = seg[idx]
                nl = (b - a + 1) // 2
                nxt += [a + nl, b]
            offsets.append(np.array(nxt, dtype=np.int64))
            self.split_axis.append(axes)
        self.perm = order
        self.offsets = offsets
        self.lo, self.hi = [], []
        Xt = X[order]
        for ell in range(L + 1):
            off = offsets[ell]
            lo = np.empty((1 << ell, dim))
            hi = np.empty((1 << ell, dim))
            for j in range(1 << ell):
                P = Xt[off[j]:off[j + 1]]
                lo[j] = P.min(axis=0)
                hi[j] = P.max(axis=0)
            self.lo.append(lo)
            self.hi.append(hi)
        self.points_tree = Xt

    def size(self, ell: int, j: int) -> int:
        return int(self.offsets[ell][j + 1] - self.offsets[ell][j])

    def rows(self, ell: int, j: int) -> slice:
        return slice(int(self.offsets[ell][j]), int(self.offsets[ell][j + 1]))


def admissible(lo_t, hi_t, lo_s, hi_s, eta: float) -> np.ndarray:
    """Far-field test for arrays of box pairs: dist > 0 and max(diam) <= eta * dist."""
    diam_t = np.sqrt(np.sum((hi_t - lo_t) ** 2, axis=-1))
    diam_s = np.sqrt(np.sum((hi_s - lo_s) ** 2, axis=-1))
    gap = np.maximum(0.0, np.maximum(lo_s - hi_t, lo_t - hi_s))
    dist = np.sqrt(np.sum(gap * gap, axis=-1))
    return (dist > 0.0) & (np.maximum(diam_t, diam_s) <= eta * dist)


def block_partition(tree: ClusterTree, eta: float):
    """Dual traversal from (root, root) (Section 3.1: close and far blocks).

    Returns ``(far, inadm)``: per tree level, int64 arrays of pairs (tau, sigma)
    sorted by (tau, sigma). ``far[ell]`` are the admissible pairs met at level ell;
    ``inadm[ell]`` the pairs refined further (at ell = L: the close leaf pairs).
    """
    far, inadm = [], []
    cand = np.zeros((1, 2), dtype=np.int64)
    for ell in range(tree.L + 1):
        lo, hi = tree.lo[ell], tree.hi[ell]
        t, s = cand[:, 0], cand[:, 1]
        adm = admissible(lo[t], hi[t], lo[s], hi[s], eta)
        f = cand[adm]
        c = cand[~adm]
        f = f[np.lexsort((f[:, 1], f[:, 0]))]
        c = c[np.lexsort((c[:, 1], c[:, 0]))]
        far.append(f)
        inadm.append(c)
        if ell < tree.L:
            kids = []
            for dt in (0, 1):
                for ds in (0, 1):
                    kids.append(np.stack([2 * c[:, 0] + dt, 2 * c[:, 1] + ds], axis=1))
            cand = np.concatenate(kids, axis=0) if kids else np.zeros((0, 2), np.int64)
    return far, inadm


# ---------------------------------------------------------------------------
# Chebyshev interpolation
# ---------------------------------------------------------------------------

def cheb_nodes_1d(q: int) -> np.ndarray:
    """First-kind Chebyshev nodes t_a = cos((2a+1) pi / (2q)), a = 0..q-1."""
    a = np.arange(q)
    return np.cos((2 * a + 1) * math.pi / (2 * q))


def lagrange_1d(t: np.ndarray, nodes: np.ndarray) -> np.ndarray:
    """Values l_b(t) of the Lagrange polynomials on ``nodes``: shape (len(t), q)."""
    q = nodes.shape[0]
    out = np.ones((t.shape[0], q))
    for b in range(q):
        for c in range(q):
            if c != b:
                out[:, b] *= (t - nodes[c]) / (nodes[b] - nodes[c])
    return out


def multi_index(q: int, dim: int) -> np.ndarray:
    """Rows a -> (a_0, ..., a_{d-1}) with a = sum_d a_d q^d (dimension 0 fastest)."""
    k = q ** dim
    a = np.arange(k)
    return np.stack([(a // q ** d) % q for d in range(dim)], axis=1)


class Chebyshev:
    """Tensor Chebyshev interpolation on the tight boxes of a cluster tree."""

    def __init__(self, tree: ClusterTree, q: int):
        self.q, self.dim = q, tree.dim
        self.k = q ** tree.dim
        self.t = cheb_nodes_1d(q)
        self.mi = multi_index(q, tree.dim)
        ext = float(np.max(tree.hi[0][0] - tree.lo[0][0])) if tree.n > 0 else 1.0
        self.floor = 1e-12 * max(ext, 1e-300)
        self.tree = tree

    def center_half(self, ell: int, j: int):
        lo, hi = self.tree.lo[ell][j], self.tree.hi[ell][j]
        return 0.5 * (lo + hi), np.maximum(0.5 * (hi - lo), self.floor)

    def nodes(self, ell: int, j: int) -> np.ndarray:
        """The k = q^d interpolation nodes xi_a of cluster j at level ell."""
        c, h = self.center_half(ell, j)
        return c[None, :] + h[None, :] * self.t[self.mi]

    def lagrange(self, ell: int, j: int, Y: np.ndarray) -> np.ndarray:
        """L_a(y) for the cluster's tensor Lagrange basis: shape (len(Y), k)."""
        c, h = self.center_half(ell, j)
        T = (Y - c[None, :]) / h[None, :]
        out = np.ones((Y.shape[0], self.k))
        for d in range(self.dim):
            out *= lagrange_1d(T[:, d], self.t)[:, self.mi[:, d]]
        return out


def qr_nonneg(M: np.ndarray):
    """Householder QR (LAPACK) with diag(R) >= 0; reduced when rows > cols."""
    Q, R = np.linalg.qr(M, mode="reduced")
    s = np.sign(np.diag(R)).copy()
    s[s == 0] = 1.0
    return Q * s[None, :], R * s[:, None]


class BlockOp:
    """y += sum over blocks (t, s): B_ts x_s, for a list of dense blocks.

    ``rows``/``cols`` are the offsets of the row and column segments; every block
    B_ts has shape (rows[t+1]-rows[t], cols[s+1]-cols[s]). The products are
    batched with zero padding to a common shape (exact: padded entries are zero)
    and summed into y by ``np.add.at``; this changes only the rounding order.
    """

    def __init__(self, rows, cols, pairs, blocks):
        self.rows = np.asarray(rows, np.int64)
        self.cols = np.asarray(cols, np.int64)
        self.pairs = np.asarray(pairs, np.int64).reshape(-1, 2)
        nb = self.pairs.shape[0]
        self.nout = int(self.rows[-1])
        self.nin = int(self.cols[-1])
        if nb == 0:
            self.stack = None
            return
        rt = self.rows[self.pairs[:, 0] + 1] - self.rows[self.pairs[:, 0]]
        cs = self.cols[self.pairs[:, 1] + 1] - self.cols[self.pairs[:, 1]]
        R, C = int(rt.max()), int(cs.max())
        dtype = np.result_type(*[b.dtype for b in blocks[:1]])
        st = np.zeros((nb, R, C), dtype=dtype)
        for k, b in enumerate(blocks):
            st[k, :b.shape[0], :b.shape[1]] = b
        self.stack = st
        ar, ac = np.arange(R), np.arange(C)
        ri = self.rows[self.pairs[:, 0]][:, None] + ar[None, :]
        ci = self.cols[self.pairs[:, 1]][:, None] + ac[None, :]
        self.ri = np.where(ar[None, :] < rt[:, None], ri, self.nout)   # padded rows -> dummy
        self.ci = np.where(ac[None, :] < cs[:, None], ci, self.nin)    # padded cols -> zero

    def matvec(self, x: np.ndarray, out: np.ndarray | None = None) -> np.ndarray:
        tail = x.shape[1:]
        y = np.zeros((self.nout + 1,) + tail, dtype=x.dtype)
        if self.stack is not None:
            xe = np.concatenate([x, np.zeros((1,) + tail, dtype=x.dtype)], axis=0)
            g = xe[self.ci]                                   # (nb, C, ...)
            st = self.stack.astype(x.dtype, copy=False)
            if tail:
                prod = np.matmul(st, g)                       # (nb, R, ncols)
                np.add.at(y, self.ri.reshape(-1), prod.reshape(-1, *tail))
            else:
                prod = np.matmul(st, g[..., None])[..., 0]    # (nb, R)
                np.add.at(y, self.ri.reshape(-1), prod.reshape(-1))
        y = y[:self.nout]
        if out is not None:
            out += y
            return out
        return y


# ---------------------------------------------------------------------------
# The H2 matrix
# ---------------------------------------------------------------------------

@dataclass
class KernelSpec:
    kind: str
    length: float = 1.0
    nugget: float = 0.0
    degree: int = 2
    weights: np.ndarray | None = None    # per point, original order
    diag: np.ndarray | None = None       # per point, original order (override)


class H2Matrix:
    """The H2 approximation of a kernel matrix with orthonormal nested bases.

    Parameters mirror the paper's problem statement: points, kernel, leaf size,
    interpolation order q (rank k = q^d) and admissibility parameter eta.

    ``basis`` selects how the nested bases are made before orthonormalisation:
    ``"chebyshev"`` (tensor interpolation with q nodes per axis, rank q^d), or
    ``"skeleton"`` (recursive skeletonization to the relative tolerance ``tol`` with
    ranks of at most ``rank_max``, see ``oracle.skeleton``; the paper's matrices are
    built by such a tolerance-driven method, Sec. 4.1). Both yield the same
    ingredients -- leaf basis, child-to-parent transfers, coupling points -- and
    the same orthonormalisation and couplings S = R_tau S^0 R_sigma^T follow.
    """

    def __init__(self, points, kspec: KernelSpec, leaf: int, q: int, eta: float,
                 tree: ClusterTree | None = None, partition=None, basis: str = "chebyshev",
                 tol: float = 1e-9, rank_max: int = 64):
        self.X = np.ascontiguousarray(points, dtype=np.float64)
        self.kspec = kspec
        self.leaf, self.q, self.eta = leaf, q, eta
        if basis not in ("chebyshev", "skeleton"):
            raise ValueError(f"unknown basis {basis!r}")
        self.basis, self.tol, self.rank_max = basis, float(tol), int(rank_max)
        self._cache = {}
        self.tree = tree if tree is not None else ClusterTree(self.X, leaf)
        T = self.tree
        self.L = T.L
        far, inadm = partition if partition is not None else block_partition(T, eta)
        self.far, self.inadm = far, inadm
        self.near = inadm[T.L]
        levels_with_far = [ell for ell in range(T.L + 1) if far[ell].shape[0] > 0]
        self.tstar = levels_with_far[0] if levels_with_far else None
        self.cheb = Chebyshev(T, q)
        n = T.n
        w = np.ones(n) if kspec.weights is None else np.asarray(kspec.weights, np.float64)
        self.sqrt_w_tree = np.sqrt(w[T.perm])
        self.diag_tree = K.diag_value(kspec.kind, self.X, kspec.weights, kspec.diag,
                                      kspec.nugget, kspec.length, kspec.degree)[T.perm]
        self._fill_near()
        self.skeletons = None
        if self.tstar is not None:
            if basis == "skeleton":
                from .skeleton import Skeletons
                self.skeletons = Skeletons(T, far, self.tstar, kspec, self.sqrt_w_tree, tol, rank_max)
            self._bases()
            self._couplings()

    # -- kernel helpers -------------------------------------------------------
    def _k(self, A, B):
        s = self.kspec
        return K.kmat(s.kind, A, B, s.length, s.degree)

    # -- close blocks D ---------------------------------------------------------
    def _fill_near(self):
        """D_tau,sigma[i, j] = sqrt(w_i) k(x_i, x_j) sqrt(w_j), A_ii on the diagonal."""
        T = self.tree
        Xt, sw = T.points_tree, self.sqrt_w_tree
        self.D = []
        for (t, s) in self.near:
            rt, rs = T.rows(T.L, t), T.rows(T.L, s)
            with np.errstate(divide="ignore"):
                B = self._k(Xt[rt], Xt[rs])
            B = sw[rt][:, None] * B * sw[rs][None, :]
            if t == s:
                np.fill_diagonal(B, self.diag_tree[rt])
            self.D.append(B)

    # -- nested orthonormal bases ----------------------------------------------
    def _bases(self):
        """Leaf bases U_tau, transfers E'_c and factors R_tau (levels t*..L)."""
        T, C = self.tree, self.cheb
        L, ts = T.L, self.tstar
        self.U = {}        # leaf j -> (n_j x r_j) orthonormal
        self.Et = {}       # (ell, c) -> (r_c x r_parent) orthonormal transfer, ell > t*
        self.R = {}        # (ell, j) -> (r_j x k)
        self.rank = {}     # (ell, j) -> r_j
        Xt, sw = T.points_tree, self.sqrt_w_tree
        Sk = self.skeletons
        for j in range(1 << L):
            rj = T.rows(L, j)
            if Sk is None:
                Uc = sw[rj][:, None] * C.lagrange(L, j, Xt[rj])
            else:
                Uc = Sk.leaf_basis(j)        # the weights are inside the sampled rows
            Q, R = qr_nonneg(Uc)
            self.U[j] = Q
            self.R[(L, j)] = R
            self.rank[(L, j)] = Q.shape[1]
        for ell in range(L - 1, ts - 1, -1):
            for p in range(1 << ell):
                blocks = []
                for c in (2 * p, 2 * p + 1):
                    if Sk is None:
                        E = C.lagrange(ell, p, C.nodes(ell + 1, c))   # E_c[a, b] = L^P_b(xi^c_a)
                    else:
                        E = Sk.transfer(ell + 1, c)                  # rows of T_parent for c's skeleton
                    blocks.append(self.R[(ell + 1, c)] @ E)
                M = np.vstack(blocks)
                Q, R = qr_nonneg(M)
                r1 = blocks[0].shape[0]
                self.Et[(ell + 1, 2 * p)] = Q[:r1]
                self.Et[(ell + 1, 2 * p + 1)] = Q[r1:]
                self.R[(ell, p)] = R
                self.rank[(ell, p)] = Q.shape[1]

    def coupling_points(self, ell: int, j: int):
        """(points, weights) whose kernel matrix is the coupling factor S^0 of cluster j:
        the Chebyshev nodes with unit weights, or the skeleton points with sqrt(w)."""
        if self.skeletons is None:
            C = self.cheb
            return C.nodes(ell, j), np.ones(C.k)
        idx = self.skeletons.skel[(ell, j)]
        return self.tree.points_tree[idx], self.sqrt_w_tree[idx]

    def _couplings(self):
        """S_tau,sigma = R_tau S^0_tau,sigma R_sigma^T for every far pair, with
        S^0 = k(xi_tau, xi_sigma) on the Chebyshev nodes, or the matrix entries
        A(skel_tau, skel_sigma) on the skeletons."""
        self.S = {}
        for ell in range(self.tstar, self.L + 1):
            lst = []
            for (t, s) in self.far[ell]:
                Pt, wt = self.coupling_points(ell, t)
                Ps, ws = self.coupling_points(ell, s)
                Sc = wt[:, None] * self._k(Pt, Ps) * ws[None, :]
                lst.append(self.R[(ell, t)] @ Sc @ self.R[(ell, s)].T)
            self.S[ell] = lst

    # -- coefficient-space layout -------------------------------------------------
    def coef_offsets(self, ell: int) -> np.ndarray:
        """Offsets of the cluster coefficient blocks of tree level ell (concatenated)."""
        key = ("off", ell)
        if key not in self._cache:
            r = [self.rank[(ell, j)] for j in range(1 << ell)]
            self._cache[key] = np.concatenate([[0], np.cumsum(r)]).astype(np.int64)
        return self._cache[key]

    def _op(self, key, make):
        if key not in self._cache:
            self._cache[key] = make()
        return self._cache[key]

    def near_op(self) -> BlockOp:
        """The close part D (block sparse over the close leaf pairs)."""
        off = self.tree.offsets[self.L]
        return self._op("D", lambda: BlockOp(off, off, self.near, self.D))

    def coupling_op(self, ell: int) -> BlockOp:
        """The far blocks S_tau,sigma of tree level ell."""
        off = self.coef_offsets(ell)
        return self._op(("S", ell), lambda: BlockOp(off, off, self.far[ell], self.S[ell]))

    def up_op(self, ell: int) -> BlockOp:
        """x_P = sum_c E'_c^T x_c: level ell+1 coefficients -> level ell."""
        def make():
            kids = np.arange(1 << (ell + 1))
            pairs = np.stack([kids // 2, kids], axis=1)
            blocks = [self.Et[(ell + 1, int(c))].T for c in kids]
            return BlockOp(self.coef_offsets(ell), self.coef_offsets(ell + 1), pairs, blocks)
        return self._op(("up", ell), make)

    def down_op(self, ell: int) -> BlockOp:
        """y_c += E'_c y_P: level ell-1 coefficients -> level ell."""
        def make():
            kids = np.arange(1 << ell)
            pairs = np.stack([kids, kids // 2], axis=1)
            blocks = [self.Et[(ell, int(c))] for c in kids]
            return BlockOp(self.coef_offsets(ell), self.coef_offsets(ell - 1), pairs, blocks)
        return self._op(("down", ell), make)

    def leaf_ops(self):
        """(U_1^T, U_1): leaf coefficients <-> points in tree order."""
        def make():
            L = self.L
            leaves = np.arange(1 << L)
            pairs = np.stack([leaves, leaves], axis=1)
            offc, offp = self.coef_offsets(L), self.tree.offsets[L]
            return (BlockOp(offc, offp, pairs, [self.U[int(j)].T for j in leaves]),
                    BlockOp(offp, offc, pairs, [self.U[int(j)] for j in leaves]))
        return self._op("leaf", make)

    # -- H2 matrix-vector product (Section 3.1, x_i = V_i x_{i-1}, y_{i-1} = D_i x_{i-1} + U_i y_i)
    def _up(self, xh: dict, top: int, bottom: int):
        """x_P = sum_c E'_c^T x_c from level ``bottom`` up to level ``top``."""
        for ell in range(bottom - 1, top - 1, -1):
            xh[ell] = self.up_op(ell).matvec(xh[ell + 1])

    def _couple(self, xh: dict, yh: dict, top: int, bottom: int):
        """y_tau = sum_sigma S_tau,sigma x_sigma at every level ell in [top, bottom]."""
        for ell in range(top, bottom + 1):
            yh[ell] = self.coupling_op(ell).matvec(xh[ell])

    def _down(self, yh: dict, top: int, bottom: int):
        """y_c += E'_c y_parent from level top+1 down to ``bottom``."""
        for ell in range(top + 1, bottom + 1):
            self.down_op(ell).matvec(yh[ell - 1], out=yh[ell])

    def leaf_restrict(self, v_tree: np.ndarray) -> np.ndarray:
        """U_1^T v: leaf coefficients of a point vector in tree order."""
        return self.leaf_ops()[0].matvec(v_tree)

    def leaf_prolong(self, e: np.ndarray) -> np.ndarray:
        """U_1 e: point vector (tree order) from leaf coefficients."""
        return self.leaf_ops()[1].matvec(e)

    def apply_tree(self, xt: np.ndarray) -> np.ndarray:
        """y = A x with x, y in tree order (any number of columns)."""
        y = self.near_op().matvec(xt)
        if self.tstar is None:
            return y
        L = self.L
        xh = {L: self.leaf_restrict(xt)}
        self._up(xh, self.tstar, L)
        yh = {}
        self._couple(xh, yh, self.tstar, L)
        self._down(yh, self.tstar, L)
        return y + self.leaf_prolong(yh[L])

    def apply(self, x: np.ndarray) -> np.ndarray:
        """y = A x with x, y in the user's point order."""
        x = np.asarray(x)
        perm = self.tree.perm
        y = np.empty_like(x)
        y[perm] = self.apply_tree(x[perm])
        return y

    def dense(self) -> np.ndarray:
        """The represented matrix as a dense array (user order; small N only)."""
        return self.apply(np.eye(self.tree.n))

    def expanded_basis(self, ell: int, j: int) -> np.ndarray:
        """U_tau of cluster j at level ell expanded to its points (tree order):
        the leaf basis for ell = L, else blockdiag(children's bases) [E'_c1; E'_c2]."""
        if ell == self.L:
            return self.U[j]
        B1 = self.expanded_basis(ell + 1, 2 * j)
        B2 = self.expanded_basis(ell + 1, 2 * j + 1)
        return np.vstack([B1 @ self.Et[(ell + 1, 2 * j)], B2 @ self.Et[(ell + 1, 2 * j + 1)]])

    def dense_blocks(self) -> np.ndarray:
        """The represented matrix assembled block by block (tree order): the close
        blocks D and, for every far pair, U_tau S U_sigma^T with expanded bases. A
        second route to the same matrix as ``apply`` (eq. h2 written out blockwise)."""
        T = self.tree
        A = np.zeros((T.n, T.n))
        for (t, s), B in zip(self.near, self.D):
            A[T.rows(T.L, t), T.rows(T.L, s)] = B
        if self.tstar is None:
            return A
        for ell in range(self.tstar, self.L + 1):
            Bx = {j: self.expanded_basis(ell, j) for j in range(1 << ell)}
            for (t, s), S in zip(self.far[ell], self.S[ell]):
                A[T.rows(ell, t), T.rows(ell, s)] = Bx[t] @ S @ Bx[s].T
        return A

    def astype(self, dtype) -> "H2Matrix":
        """A shallow copy whose stored blocks are rounded to ``dtype``."""
        import copy
        o = copy.copy(self)
        o._cache = {k: v for k, v in self._cache.items() if k[0] == "off"}
        o.D = [b.astype(dtype) for b in self.D]
        if self.tstar is not None:
            o.U = {k: v.astype(dtype) for k, v in self.U.items()}
            o.Et = {k: v.astype(dtype) for k, v in self.Et.items()}
            o.S = {ell: [b.astype(dtype) for b in lst] for ell, lst in self.S.items()}
        return o


def dense_partition_check(h: H2Matrix) -> np.ndarray:
    """Coverage matrix of the block partition: every (i, j) must be covered exactly
    once by a close block or a far block of some level (Section 3.1: A = D + F)."""
    T = h.tree
    cov = np.zeros((T.n, T.n), dtype=np.int64)
    for (t, s) in h.near:
        cov[T.rows(T.L, t), T.rows(T.L, s)] += 1
    for ell in range(T.L + 1):
        for (t, s) in h.far[ell]:
            cov[T.rows(ell, t), T.rows(ell, s)] += 1
    return cov
