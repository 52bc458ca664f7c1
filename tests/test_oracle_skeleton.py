"""Pins of the oracle's skeleton (interpolative-decomposition) bases.

The construction is the oracle's reading of the tolerance-driven H2 builder the
paper uses (Sec. 4.1: matrices of relative accuracy 1e-9 with adaptive ranks). Each
pin checks it against something other than itself: LAPACK's column-pivoted QR, the
defining property of an interpolative decomposition, the exact rank of a polynomial
kernel, the dense kernel matrix and its eigenvalues.
"""
import math

import numpy as np
import pytest
import scipy.linalg as sla

import workloads as W
from oracle import H2MG, H2Matrix, KernelSpec, SolveOpts, dense_kernel_matrix, solve, solve_fcg
from oracle.skeleton import SAMPLE_CAP, pivoted_qr_id


def user_dense(h):
    """The represented matrix in user order, by the block assembly."""
    A = h.dense_blocks()
    p = h.tree.perm
    out = np.empty_like(A)
    out[np.ix_(p, p)] = A
    return out


# --------------------------------------------------------------------------- the pivoted QR
def test_pivoted_qr_matches_lapack_on_a_generic_matrix():
    """Greedy largest-remaining-norm pivoting is LAPACK's dgeqp3 rule: on a matrix
    without ties both give the same pivots and the same R11^{-1} R12."""
    rng = np.random.default_rng(1)
    B = rng.standard_normal((40, 30)) @ np.diag(np.logspace(0, -6, 30)) @ rng.standard_normal((30, 30))
    piv, r, T = pivoted_qr_id(B, 0.0, 30)
    Q, R, p = sla.qr(B, mode="economic", pivoting=True)
    assert r == 30
    assert list(piv) == list(p)
    piv, r, T = pivoted_qr_id(B, 1e-3, 30)
    k = int(np.sum(np.abs(np.diag(R)) > 1e-3 * abs(R[0, 0])))
    assert r == k
    X = sla.solve_triangular(R[:k, :k], R[:k, k:])
    np.testing.assert_allclose(T[p[k:], :], X.T, rtol=1e-9, atol=1e-12)
    np.testing.assert_array_equal(T[p[:k], :], np.eye(k))


def test_pivoted_qr_exact_low_rank_and_caps():
    """A rank-5 matrix: rank 5 found at a small tolerance, and the skeleton columns
    interpolate every column exactly; rank_max caps the rank."""
    rng = np.random.default_rng(2)
    B = rng.standard_normal((30, 5)) @ rng.standard_normal((5, 20))
    piv, r, T = pivoted_qr_id(B, 1e-10, 64)
    assert r == 5
    np.testing.assert_allclose(B[:, piv[:r]] @ T.T, B, atol=1e-10 * np.abs(B).max())
    piv, r, T = pivoted_qr_id(B, 0.0, 3)
    assert r == 3
    piv, r, T = pivoted_qr_id(np.zeros((4, 6)), 1e-9, 64)   # nothing to interpolate
    assert r == 1


def test_pivoted_qr_ties_take_the_lowest_index():
    """Columns of equal norm: the lowest index wins, whatever rounding would say."""
    B = np.eye(6)
    piv, r, T = pivoted_qr_id(B, 1e-12, 6)
    assert list(piv[:r]) == list(range(6))


# --------------------------------------------------------------------------- the ID property
def test_every_cluster_interpolates_its_sampled_far_field():
    """A(F_tau, cand) ~= A(F_tau, skel) T^T within a small multiple of tol, for every
    cluster (the defining property of the interpolative decomposition, step 3-5),
    and T is the identity on the skeleton."""
    X = W.uniform_points(2048, 2, 1)
    tol = 1e-7
    h = H2Matrix(X, KernelSpec("exponential", 0.1, 1e-2), 32, 4, 1.0, basis="skeleton", tol=tol)
    Sk = h.skeletons
    Xt = h.tree.points_tree
    from oracle.skeleton import far_partners
    checked = 0
    for ell in range(h.tstar, h.L + 1):
        part = far_partners(h.far[ell])
        partp = far_partners(h.far[ell - 1]) if ell - 1 >= h.tstar else {}
        for j in range(1 << ell):
            c = Sk.cand[(ell, j)]
            cols = [Sk.cand[(ell, s)] for s in part.get(j, [])]
            for s in partp.get(j // 2, []):
                pts_ = np.concatenate([Sk.cand[(ell, 2 * s)], Sk.cand[(ell, 2 * s + 1)]])
                cols.append(pts_[::max(1, math.ceil(len(pts_) / SAMPLE_CAP))])
            if not cols:
                continue
            F = np.concatenate(cols)
            A = dense_kernel_matrix("exponential", Xt[np.r_[F, c]], 0.1, 0.0)[: len(F), len(F):]
            T = Sk.T[(ell, j)]
            pos = {int(v): i for i, v in enumerate(c)}
            sk = [pos[int(v)] for v in Sk.skel[(ell, j)]]
            np.testing.assert_array_equal(T[sk, :], np.eye(len(sk)))
            err = np.linalg.norm(A - A[:, sk] @ T.T) / np.linalg.norm(A)
            assert err <= 30 * tol, (ell, j, err)
            checked += 1
    assert checked > 20


# --------------------------------------------------------------------------- exactness
@pytest.mark.parametrize("dim,deg", [(2, 2), (3, 1), (2, 3)])
def test_polynomial_kernel_has_its_exact_rank(dim, deg):
    """(1 + x.y)^m has rank C(m + d, d) on any point set: every cluster with enough
    candidates stops at exactly that rank, and the H2 product equals the dense one."""
    X = W.uniform_points(1500, dim, 3)
    kr = math.comb(deg + dim, dim)
    h = H2Matrix(X, KernelSpec("poly", degree=deg, nugget=1.0), 32, 4, 0.8, basis="skeleton", tol=1e-11)
    seen = 0
    for (ell, j), sk in h.skeletons.skel.items():
        nc = len(h.skeletons.cand[(ell, j)])
        if nc >= kr and h.skeletons.sampled[(ell, j)]:
            assert len(sk) == kr, (ell, j, len(sk), kr)
            seen += 1
        elif not h.skeletons.sampled[(ell, j)]:          # nothing far: all candidates kept
            assert len(sk) == min(nc, 64)
    assert seen > 10
    K = dense_kernel_matrix("poly", X, degree=deg, nugget=1.0)
    x = np.random.default_rng(0).standard_normal(1500)
    assert np.linalg.norm(h.apply(x) - K @ x) / np.linalg.norm(K @ x) < 1e-12


def test_block_assembly_equals_the_product():
    """Two routes to the represented matrix: the level-by-level product (Sec. 3.1)
    and the block-by-block assembly of eq. h2 with expanded bases."""
    X = W.uniform_points(1200, 3, 4)
    h = H2Matrix(X, KernelSpec("gaussian", 0.2, 1e-3), 32, 4, 1.0, basis="skeleton", tol=1e-8)
    x = np.random.default_rng(1).standard_normal((1200, 3))
    np.testing.assert_allclose(h.apply(x), user_dense(h) @ x, rtol=0, atol=1e-13 * np.abs(h.apply(x)).max())


@pytest.mark.parametrize("tol", [1e-4, 1e-6, 1e-8])
def test_error_follows_the_tolerance(tol):
    """Relative error of the represented matrix against the dense kernel matrix stays
    within a small multiple of the tolerance (the paper's relative accuracy)."""
    X = W.uniform_points(2048, 2, 5)
    K = dense_kernel_matrix("exponential", X, 0.1, 1e-2)
    h = H2Matrix(X, KernelSpec("exponential", 0.1, 1e-2), 64, 4, 1.0, basis="skeleton", tol=tol)
    err = np.linalg.norm(user_dense(h) - K, 2) / np.linalg.norm(K, 2)
    assert err <= 10 * tol, err
    assert err >= 1e-3 * tol or tol == 1e-8   # it is a truncation, not an exact copy


def test_weights_enter_the_sampled_rows():
    """Surface kernel with panel areas as weights and the disk diagonal: the skeleton
    H2 matrix is within 1e-7 of the dense weighted matrix."""
    c, a, _ = W.perturbed_icosphere(9, 0)
    from oracle.kernels import surface_diag
    ks = KernelSpec("laplace_sl", weights=a, diag=surface_diag(a))
    h = H2Matrix(c, ks, 32, 4, 1.0, basis="skeleton", tol=1e-9)
    K = dense_kernel_matrix("laplace_sl", c, weights=a, diag=surface_diag(a))
    err = np.linalg.norm(user_dense(h) - K, 2) / np.linalg.norm(K, 2)
    assert err < 1e-7, err


# --------------------------------------------------------------------------- structure kept
def test_symmetry_orthonormality_and_galerkin():
    """The orthonormalisation chain runs unchanged on skeleton factors: orthonormal
    expanded bases, S_st = S_ts^T (symmetric matrix), and A_{i+1} = U_i^T A_i U_i at
    every level (eq. a2_str)."""
    X = W.uniform_points(1024, 2, 6)
    h = H2Matrix(X, KernelSpec("gaussian", 0.15, 1e-3), 16, 4, 1.0, basis="skeleton", tol=1e-9)
    A = user_dense(h)
    assert np.abs(A - A.T).max() <= 1e-14 * np.abs(A).max()
    for ell in range(h.tstar, h.L + 1):
        for j in range(1 << ell):
            B = h.expanded_basis(ell, j)
            np.testing.assert_allclose(B.T @ B, np.eye(B.shape[1]), atol=1e-12)
    mg = H2MG(h)
    for i in range(1, mg.l):
        n_i, n_c = mg.size(i), mg.size(i + 1)
        Ai = np.stack([mg.apply(i, e) for e in np.eye(n_i)], axis=1)
        U = np.stack([mg.prolong(i, e) for e in np.eye(n_c)], axis=1)
        Ac = np.stack([mg.apply(i + 1, e) for e in np.eye(n_c)], axis=1)
        np.testing.assert_allclose(Ac, U.T @ Ai @ U, atol=1e-12 * np.abs(Ai).max())


# --------------------------------------------------------------------------- definiteness
def test_dense_gaussian_at_the_full_size_density_is_kept_positive_definite():
    """4096 points at the density of 2^20 points in the unit cube (a cube of side
    (2^-8)^(1/3)), Gaussian exp(-r^2/0.05^2) + 1e-3 I, leaf 64, eta 1: the 4x4x4
    Chebyshev H2 matrix is indefinite (its interpolation error exceeds the nugget),
    while the skeleton H2 matrix with rank <= 64 at tol 1e-9 keeps lambda_min within
    1% of the nugget, the dense kernel matrix's own bound."""
    n = 4096
    X = W.uniform_points(n, 3, 2) * (n / 2.0 ** 20) ** (1 / 3)
    ks = KernelSpec("gaussian", 0.05, 1e-3)
    hc = H2Matrix(X, ks, 64, 4, 1.0)
    hs = H2Matrix(X, ks, 64, 4, 1.0, basis="skeleton", tol=1e-9, rank_max=64)
    lc = np.linalg.eigvalsh(hc.dense_blocks())[0]
    ls = np.linalg.eigvalsh(hs.dense_blocks())[0]
    lk = np.linalg.eigvalsh(dense_kernel_matrix("gaussian", X, 0.05, 1e-3))[0]
    assert lc < -1e-3, lc
    assert ls > 0.99e-3 and abs(ls - lk) < 1e-5, (ls, lk)
    assert max(hs.rank.values()) <= 64


def test_skeleton_solve_converges_like_the_dense_system():
    """H2-MG on the skeleton H2 matrix of the exponential workload: repeated V-cycles
    reach 1e-8 and flexible CG 1e-10, and both solutions are the dense Cholesky
    solution of the represented matrix within kappa * tol."""
    p = W.workload(1, n=2048)
    h = H2Matrix(p["points"], KernelSpec("exponential", 0.1, 1e-2), 64, 4, 1.0, basis="skeleton", tol=1e-10)
    mg = H2MG(h)
    A = user_dense(h)
    xd = sla.cho_solve(sla.cho_factor(A), p["b"])
    kappa = np.linalg.cond(A)
    x, info = solve(mg, p["b"], SolveOpts(tol=1e-8, max_cycles=200))
    assert info.converged, info.history[-3:]
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) < 1e-8 * kappa
    x, info = solve_fcg(mg, p["b"], SolveOpts(tol=1e-10, max_cycles=200))
    assert info.converged, info.history[-3:]
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) < 1e-10 * kappa


def test_kernel_rows_are_rows_of_the_dense_matrix():
    """Sampled rows by the formula equal the rows of the dense matrix (both routes of
    kernels.py), with weights and a diagonal override, and the nugget on the diagonal."""
    from oracle.kernels import kernel_rows
    c, a, _ = W.perturbed_icosphere(6, 0)
    from oracle.kernels import surface_diag
    K = dense_kernel_matrix("laplace_sl", c, weights=a, diag=surface_diag(a), nugget=0.1)
    rows = [0, 5, 17, len(a) - 1]
    np.testing.assert_array_equal(kernel_rows("laplace_sl", c, rows, weights=a, diag=surface_diag(a), nugget=0.1),
                                  K[rows])
    X = W.uniform_points(500, 3, 1)
    K = dense_kernel_matrix("gaussian", X, 0.1, 1e-3)
    np.testing.assert_allclose(kernel_rows("gaussian", X, [3, 499], 0.1, 1e-3), K[[3, 499]], rtol=1e-15, atol=0)
