"""Pins of the CPU oracle against what the paper and the mathematics fix.

None of these compares the oracle with itself: each checks a closed form, an
identity the paper states, a textbook special case or a brute-force computation.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import H2MG, H2Matrix, KernelSpec, SolveOpts, cg, dense_kernel_matrix, solve
from oracle.h2 import (ClusterTree, admissible, block_partition, cheb_nodes_1d,
                       dense_partition_check, lagrange_1d)
from oracle.mg import solve_mixed, vcycle


def pts(n, dim, seed=7):
    return np.random.default_rng(seed).random((n, dim))


# --------------------------------------------------------------------------- tree
@pytest.mark.parametrize("n,leaf", [(1, 4), (5, 4), (100, 8), (1000, 64), (777, 16)])
def test_tree_structure(n, leaf):
    X = pts(n, 2)
    T = ClusterTree(X, leaf)
    assert sorted(T.perm.tolist()) == list(range(n))
    assert T.L == (0 if n <= leaf else math.ceil(math.log2(n / leaf)))
    for ell in range(T.L + 1):
        sz = np.diff(T.offsets[ell])
        assert sz.min() >= n // (1 << ell) and sz.max() <= -(-n // (1 << ell))
    assert np.diff(T.offsets[T.L]).max() <= leaf
    # brute-force split rule at every internal cluster
    Xt = X[T.perm]
    for ell in range(T.L):
        for j in range(1 << ell):
            seg = T.rows(ell, j)
            P = Xt[seg]
            ext = P.max(0) - P.min(0)
            axis = int(np.argmax(ext))
            assert T.split_axis[ell][j] == axis
            left = T.rows(ell + 1, 2 * j)
            right = T.rows(ell + 1, 2 * j + 1)
            nl = left.stop - left.start
            assert nl == -(-(seg.stop - seg.start) // 2)
            if right.stop > right.start:
                kl = [(Xt[i, axis], T.perm[i]) for i in range(left.start, left.stop)]
                kr = [(Xt[i, axis], T.perm[i]) for i in range(right.start, right.stop)]
                assert max(kl) < min(kr)
    # tight boxes
    for ell in range(T.L + 1):
        for j in range(1 << ell):
            P = Xt[T.rows(ell, j)]
            assert np.array_equal(T.lo[ell][j], P.min(0)) and np.array_equal(T.hi[ell][j], P.max(0))


def test_tree_tie_break_by_original_index():
    # all points share the split coordinate: the order must follow original indices
    X = np.zeros((8, 2))
    X[:, 1] = [3, 3, 3, 3, 1, 1, 1, 1]   # longest extent along axis 1
    T = ClusterTree(X, 2)
    left = T.perm[T.rows(1, 0)]
    assert sorted(left.tolist()) == [4, 5, 6, 7]


# --------------------------------------------------------------------------- partition
def test_admissibility_brute_force():
    lo_t, hi_t = np.array([0.0, 0.0]), np.array([1.0, 1.0])
    # touching boxes: dist = 0 -> never admissible
    assert not admissible(lo_t, hi_t, np.array([1.0, 0.0]), np.array([2.0, 1.0]), 10.0)
    # dist = 2 along x, diam = sqrt(2): admissible for eta >= sqrt(2)/2
    lo_s, hi_s = np.array([3.0, 0.0]), np.array([4.0, 1.0])
    assert admissible(lo_t, hi_t, lo_s, hi_s, math.sqrt(2) / 2)
    assert not admissible(lo_t, hi_t, lo_s, hi_s, math.sqrt(2) / 2 * 0.999)
    # diagonal gap: dist = sqrt(2*0.5^2)
    lo_s, hi_s = np.array([1.5, 1.5]), np.array([2.0, 2.5])
    d = math.sqrt(0.5)
    diam = max(math.sqrt(2), math.sqrt(0.25 + 1.0))
    assert admissible(lo_t, hi_t, lo_s, hi_s, diam / d)
    assert not admissible(lo_t, hi_t, lo_s, hi_s, diam / d * 0.999)


@pytest.mark.parametrize("dim,eta", [(1, 1.0), (2, 1.0), (3, 1.0), (2, 0.5), (2, 0.0)])
def test_partition_covers_matrix_once(dim, eta):
    X = pts(600, dim)
    T = ClusterTree(X, 16)
    far, inadm = block_partition(T, eta)
    h = H2Matrix.__new__(H2Matrix)
    h.tree, h.near, h.far = T, inadm[T.L], far
    cov = dense_partition_check(h)
    assert (cov == 1).all()          # A = D + F with disjoint close / far blocks (eq. h20)
    for ell in range(T.L + 1):
        for (t, s) in far[ell]:
            assert admissible(T.lo[ell][t], T.hi[ell][t], T.lo[ell][s], T.hi[ell][s], eta)
            # parent pair was inadmissible (refinement stops at the first far level)
            if ell > 0:
                assert any((inadm[ell - 1] == [t // 2, s // 2]).all(1))
        pairs = {tuple(p) for p in far[ell].tolist()}
        assert all((s, t) in pairs for (t, s) in pairs)    # symmetric partition
    if eta == 0.0:
        assert sum(len(f) for f in far) == 0


# --------------------------------------------------------------------------- Chebyshev
@pytest.mark.parametrize("q", [1, 2, 3, 4, 5, 7])
def test_chebyshev_nodes_and_lagrange(q):
    t = cheb_nodes_1d(q)
    # first-kind nodes are the roots of T_q(t) = cos(q arccos t)
    assert np.allclose(np.cos(q * np.arccos(t)), 0.0, atol=1e-14)
    Lg = lagrange_1d(t, t)
    assert np.allclose(Lg, np.eye(q), atol=1e-14)
    # interpolation reproduces polynomials of degree <= q-1
    s = np.linspace(-1, 1, 17)
    c = np.random.default_rng(q).standard_normal(q)
    poly = lambda z: np.polyval(c, z)
    assert np.allclose(lagrange_1d(s, t) @ poly(t), poly(s), atol=1e-12)


# --------------------------------------------------------------------------- H2 matvec
@pytest.mark.parametrize("dim,q,deg", [(1, 3, 2), (2, 3, 2), (2, 4, 3), (3, 3, 2)])
def test_polynomial_kernel_is_exact(dim, q, deg):
    """With ranks never truncated, Chebyshev interpolation of degree q-1 reproduces
    a kernel that is a polynomial of degree <= q-1 in each variable, so the H2
    matvec equals the dense matvec up to rounding."""
    X = pts(700, dim)
    ks = KernelSpec("poly", nugget=0.5, degree=deg)
    h = H2Matrix(X, ks, 16, q, 1.0)
    assert h.tstar is not None
    x = np.random.default_rng(1).standard_normal(700)
    Kd = dense_kernel_matrix("poly", X, nugget=0.5, degree=deg)
    y, yd = h.apply(x), Kd @ x
    assert np.linalg.norm(y - yd) / np.linalg.norm(yd) < 1e-13


def test_polynomial_kernel_degree_too_high_is_not_exact():
    X = pts(700, 2)
    h = H2Matrix(X, KernelSpec("poly", nugget=0.5, degree=4), 16, 3, 1.0)
    x = np.random.default_rng(1).standard_normal(700)
    Kd = dense_kernel_matrix("poly", X, nugget=0.5, degree=4)
    assert np.linalg.norm(h.apply(x) - Kd @ x) / np.linalg.norm(Kd @ x) > 1e-10


def test_weights_and_diagonal_override():
    X = pts(500, 3)
    w = 0.5 + np.random.default_rng(3).random(500)
    dg = 2.0 + np.random.default_rng(4).random(500)
    ks = KernelSpec("poly", nugget=0.1, degree=1, weights=w, diag=dg)
    h = H2Matrix(X, ks, 16, 2, 1.0)
    Kd = dense_kernel_matrix("poly", X, nugget=0.1, degree=1, weights=w, diag=dg)
    assert np.allclose(np.diag(Kd), dg + 0.1)
    x = np.random.default_rng(5).standard_normal(500)
    assert np.linalg.norm(h.apply(x) - Kd @ x) / np.linalg.norm(Kd @ x) < 1e-13


def test_eta_zero_is_dense():
    X = pts(300, 2)
    ks = KernelSpec("exponential", 0.1, 1e-2)
    h = H2Matrix(X, ks, 32, 3, 0.0)
    assert h.tstar is None
    Kd = dense_kernel_matrix("exponential", X, 0.1, 1e-2)
    assert np.abs(h.dense() - Kd).max() < 1e-15


@pytest.mark.parametrize("kind,length,dim", [("gaussian", 0.3, 2), ("exponential", 0.3, 2),
                                              ("matern32", 0.3, 3)])
def test_interpolation_error_decays_in_q(kind, length, dim):
    X = pts(1024, dim)
    Kd = dense_kernel_matrix(kind, X, length, 1e-2)
    x = np.random.default_rng(2).standard_normal(1024)
    errs = []
    for q in (2, 3, 4, 5):
        h = H2Matrix(X, KernelSpec(kind, length, 1e-2), 32, q, 1.0)
        errs.append(np.linalg.norm(h.apply(x) - Kd @ x) / np.linalg.norm(Kd @ x))
    assert all(b < a for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < errs[0] / 30.0, errs


def test_symmetry_and_orthonormal_bases():
    X = pts(1500, 2)
    h = H2Matrix(X, KernelSpec("gaussian", 0.2, 1e-3), 32, 4, 1.0)
    rng = np.random.default_rng(3)
    x, y = rng.standard_normal(1500), rng.standard_normal(1500)
    a, b = y @ h.apply(x), x @ h.apply(y)
    assert abs(a - b) <= 1e-14 * np.linalg.norm(x) * np.linalg.norm(y) * 10
    for j, U in h.U.items():
        assert np.abs(U.T @ U - np.eye(U.shape[1])).max() < 1e-13
    for ell in range(h.tstar, h.L):
        for p in range(1 << ell):
            Q = np.vstack([h.Et[(ell + 1, 2 * p)], h.Et[(ell + 1, 2 * p + 1)]])
            assert np.abs(Q.T @ Q - np.eye(Q.shape[1])).max() < 1e-13
    # S_sigma,tau = S_tau,sigma^T
    for ell in range(h.tstar, h.L + 1):
        idx = {tuple(p): k for k, p in enumerate(h.far[ell].tolist())}
        for (t, s), k in idx.items():
            assert np.abs(h.S[ell][k] - h.S[ell][idx[(s, t)]].T).max() < 1e-12


def test_orthonormalisation_keeps_the_matrix():
    """U^cheb S^cheb U^cheb^T = U S U^T: compare with the Chebyshev (non-orthogonal)
    form of one far block, evaluated directly from the interpolation formulas."""
    X = pts(1024, 2)
    ks = KernelSpec("exponential", 0.2, 0.0)
    h = H2Matrix(X, ks, 32, 3, 1.0)
    T, C = h.tree, h.cheb
    ell = h.L
    t, s = h.far[ell][0]
    Ut = C.lagrange(ell, t, T.points_tree[T.rows(ell, t)])
    Us = C.lagrange(ell, s, T.points_tree[T.rows(ell, s)])
    from oracle.kernels import kmat
    Sc = kmat("exponential", C.nodes(ell, t), C.nodes(ell, s), 0.2)
    blk = Ut @ Sc @ Us.T
    A = h.dense()
    got = A[np.ix_(T.perm[T.rows(ell, t)], T.perm[T.rows(ell, s)])]
    assert np.abs(got - blk).max() < 1e-13 * np.abs(blk).max()


# --------------------------------------------------------------------------- multigrid
def small_mg(n=2048, dim=2, kind="exponential", length=0.1, nugget=1e-2, leaf=32, q=3,
             coarse_level=-1):
    X = pts(n, dim, seed=11)
    h = H2Matrix(X, KernelSpec(kind, length, nugget), leaf, q, 1.0)
    return h, H2MG(h, coarse_level)


def test_galerkin_coarse_operators():
    """A_{i+1} = U_i^T A_i U_i (eq. a2_str with orthogonal bases), at every level."""
    h, mg = small_mg()
    assert mg.l >= 3
    Ai = h.dense()
    for i in range(1, mg.l):
        ni1 = mg.size(i + 1)
        Ui = mg.prolong(i, np.eye(ni1))
        assert np.abs(Ui.T @ Ui - np.eye(ni1)).max() < 1e-13
        Ag = Ui.T @ Ai @ Ui
        Anext = mg.apply(i + 1, np.eye(ni1)) if i + 1 < mg.l else mg.Al
        assert np.abs(Anext - Ag).max() <= 1e-13 * np.abs(Ag).max()
        # restriction is the transpose of the prolongation
        v = np.random.default_rng(i).standard_normal(mg.size(i))
        assert np.allclose(mg.restrict(i, v), Ui.T @ v, atol=1e-13)
        Ai = Anext


def test_level_sizes_and_coarsest_level():
    h, mg = small_mg()
    assert mg.l == h.L - h.tstar + 1
    assert mg.m(mg.l) == h.tstar + 1
    for i in range(2, mg.l + 1):
        assert mg.size(i) == sum(h.rank[(mg.m(i), j)] for j in range(1 << mg.m(i)))


def test_cg_exact_after_n_iterations():
    rng = np.random.default_rng(0)
    M = rng.standard_normal((30, 30))
    A = M @ M.T + 30 * np.eye(30)
    f = rng.standard_normal(30)
    x, r = cg(lambda v: A @ v, f, None, 30)
    xe = np.linalg.solve(A, f)
    assert np.linalg.norm(x - xe) <= 1e-10 * np.linalg.norm(xe)
    # from an initial guess
    x0 = rng.standard_normal(30)
    x, r = cg(lambda v: A @ v, f, x0, 30)
    assert np.linalg.norm(x - xe) <= 1e-10 * np.linalg.norm(xe)
    # one step from zero is the steepest-descent step alpha = f.f / f.Af
    x1, r1 = cg(lambda v: A @ v, f, None, 1)
    assert np.allclose(x1, (f @ f) / (f @ A @ f) * f, rtol=1e-14)
    assert np.allclose(r1, f - A @ x1, atol=1e-13)


def test_cg_zero_rhs_and_breakdown_guard():
    A = np.diag([1.0, 2.0, 3.0])
    x, r = cg(lambda v: A @ v, np.zeros(3), None, 5)
    assert not x.any()
    # indefinite operator: p^T A p <= 0 stops before the update
    B = np.diag([1.0, -1.0])
    x, r = cg(lambda v: B @ v, np.array([1.0, 1.0]), None, 3)
    assert not x.any()


def test_coarse_cholesky_solves_dense_coarse_system():
    h, mg = small_mg()
    r = np.random.default_rng(3).standard_normal(mg.size(mg.l))
    e = mg.dir_sol(r)
    assert np.linalg.norm(mg.Al @ e - r) <= 1e-10 * np.linalg.norm(r)
    L = np.linalg.cholesky(mg.Al)
    assert np.abs(L @ L.T - mg.Al).max() < 1e-12 * np.abs(mg.Al).max()


def test_vcycle_is_a_contraction_in_energy_norm():
    """CG minimises the energy error over a Krylov space from its start and the
    Galerkin correction is an energy projection, so a V-cycle never increases
    the A-norm of the error (Section 3.3 with orthogonal bases)."""
    h, mg = small_mg()
    A = h.dense()
    b = np.random.default_rng(5).standard_normal(A.shape[0])
    xs = np.linalg.solve(A, b)
    x = np.zeros_like(b)
    prev = math.sqrt(xs @ A @ xs)
    for _ in range(4):
        x = vcycle(mg, x, b - h.apply(x), SolveOpts(n_f=1, n_c=10))
        e = x - xs
        cur = math.sqrt(e @ A @ e)
        assert cur <= prev * (1 + 1e-9)
        prev = cur
    assert prev < 0.8 * math.sqrt(xs @ A @ xs)


def test_coarse_level_one_is_one_direct_solve():
    h, mg = small_mg(coarse_level=1)
    b = np.random.default_rng(6).standard_normal(h.tree.n)
    x, info = solve(mg, b, SolveOpts(tol=1e-11, max_cycles=3))
    assert info.cycles == 1 and info.converged


def test_solve_matches_dense_solution():
    h, mg = small_mg(n=1024, leaf=32, q=3, nugget=1e-1)
    A = h.dense()
    b = np.random.default_rng(8).standard_normal(1024)
    x, info = solve(mg, b, SolveOpts(tol=1e-10, max_cycles=200))
    assert info.converged
    xd = np.linalg.solve(A, b)
    kappa = np.linalg.cond(A)
    assert np.linalg.norm(x - xd) <= kappa * 1e-10 * np.linalg.norm(xd)
    assert np.linalg.norm(b - A @ x) <= 1e-10 * np.linalg.norm(b) * 1.0000001


def test_mixed_precision_refinement_reaches_float64_tolerance():
    h, mg = small_mg(n=1024, leaf=32, q=3, nugget=1e-1)
    b = np.random.default_rng(9).standard_normal(1024)
    x, info = solve_mixed(mg, b, SolveOpts(tol=1e-10, max_cycles=200))
    assert info.converged
    A = h.dense()
    assert np.linalg.norm(b - A @ x) <= 1e-10 * np.linalg.norm(b) * 1.0000001


# --------------------------------------------------------------------------- inputs
def test_icosphere_geometry():
    c, a, v = W.perturbed_icosphere(4, 0, amplitude=0.0)
    assert c.shape == (20 * 16, 3)
    # unperturbed: vertices on the unit sphere, total area below 4 pi and close to it
    assert np.allclose(np.linalg.norm(v, axis=2), 1.0)
    assert 0.9 * 4 * math.pi < a.sum() < 4 * math.pi
    c, a, v = W.perturbed_icosphere(6, 1)
    r = np.linalg.norm(v, axis=2)
    assert r.min() >= 0.8 - 1e-12 and r.max() <= 1.2 + 1e-12
    assert abs(abs(r - 1).max() - 0.2) < 1e-12


def test_surface_self_interaction_is_the_disk_potential():
    """The single-layer diagonal (Sec. 4.3, symmetric scaling) is the potential at the
    centre of a flat unit-density disk of the panel's area, checked by adaptive
    Cartesian quadrature of 1 / (4 pi |y|) over the quarter disk (times four)."""
    from scipy.integrate import dblquad

    from oracle import surface_diag
    for area in (1e-3, 0.05, 2.0):
        R = math.sqrt(area / math.pi)
        q, _ = dblquad(lambda y, x: 1.0 / (4 * math.pi * math.hypot(x, y)), 0.0, R,
                       0.0, lambda x: math.sqrt(max(R * R - x * x, 0.0)), epsabs=1e-14, epsrel=1e-10)
        val = 4 * q
        assert abs(surface_diag(np.array([area]))[0] - val) <= 1e-7 * val, (area, val)
    # scaling: a length, like the off-diagonal sqrt(a a) / (4 pi r)
    assert math.isclose(surface_diag(np.array([4.0]))[0], 2 * surface_diag(np.array([1.0]))[0])


def test_surface_matrix_is_positive_definite():
    """With the disk self-interaction the dense single-layer matrix of a perturbed
    sphere is positive definite (and reasonably conditioned); the formula with an extra
    factor of the area on the diagonal is not."""
    from oracle import surface_diag
    c, a, _ = W.perturbed_icosphere(8, 1)
    A = dense_kernel_matrix("laplace_sl", c, 1.0, 0.0, weights=a, diag=surface_diag(a))
    ev = np.linalg.eigvalsh(A)
    assert ev[0] > 0 and ev[-1] / ev[0] < 1e3
    B = A.copy()
    np.fill_diagonal(B, a * np.sqrt(a / math.pi) / 2)
    assert np.linalg.eigvalsh(B)[0] < 0


def test_skip_square_levels():
    """Option skip_square_levels: a level whose restriction is square (as many basis
    columns as rows in every cluster) gets no smoothing. Where no level is square it
    changes nothing; where one is, the cycle still contracts the energy norm of the
    error and the solve still reaches the dense solution."""
    from oracle.mg import vcycle
    # 2-D, 4 x 4 nodes < 64 points per leaf: no square level
    X2 = W.uniform_points(2048, 2, 3)
    mg2 = H2MG(H2Matrix(X2, KernelSpec("exponential", 0.1, 1e-2), 64, 4, 1.0))
    assert all(mg2.size(i) < mg2.size(i - 1) for i in range(2, mg2.l + 1))
    r = np.random.default_rng(5).standard_normal(2048)
    a = vcycle(mg2, np.zeros(2048), r, SolveOpts(n_f=1, n_c=5))
    b = vcycle(mg2, np.zeros(2048), r, SolveOpts(n_f=1, n_c=5, skip_square_levels=True))
    assert np.array_equal(a, b)
    # 3-D, 2 x 2 x 2 nodes and leaves of 8 points: U_1 is square
    X3 = W.uniform_points(1024, 3, 3)
    h3 = H2Matrix(X3, KernelSpec("gaussian", 0.2, 1e-1), 8, 2, 1.0)
    mg3 = H2MG(h3)
    assert mg3.size(2) == mg3.size(1)
    o = SolveOpts(tol=1e-10, max_cycles=200, n_f=1, n_c=10, skip_square_levels=True)
    Ad = h3.dense()
    xt = np.random.default_rng(6).standard_normal(1024)
    bb = Ad @ xt
    x1 = vcycle(mg3, np.zeros(1024), bb, o)
    e0, e1 = xt, xt - x1
    assert e1 @ Ad @ e1 < e0 @ Ad @ e0
    x, info = solve(mg3, bb, o)
    assert info.converged
    assert np.linalg.norm(x - np.linalg.solve(Ad, bb)) <= np.linalg.cond(Ad) * 1e-10 * np.linalg.norm(xt)
