"""Pins of the oracle's outer loops and cycles against closed forms and textbook
iterations written densely here.

* flexible CG with an exact preconditioner converges in one step, and with the
  identity it is textbook CG (Hestenes-Stiefel, written out on the dense matrix);
* the plain CG outer loop is that same textbook CG;
* a two-level V-cycle (Algorithm 1 with l = 2) is x0 + U_1 A_2^{-1} U_1^T r without
  smoothing and, with one CG step on level 1, the three dense steps written out;
* the recursive cycle with one coarse visit is Algorithm 1; without smoothing a
  W- or F-cycle equals the V-cycle (the Galerkin coarse correction is a projection);
  with smoothing they equal the textbook recursions written densely here;
* the paper's 2-D tensor-grid workloads (Sec. 4.1, 4.2) with its A-norm stopping
  rule converge in a few cycles, roughly flat in N, and in far fewer cycles than
  unpreconditioned CG needs iterations.
"""
import numpy as np
import pytest
import scipy.linalg as sla

import workloads as W
from oracle import H2MG, H2Matrix, KernelSpec, SolveOpts, cycle, solve, solve_cg, solve_fcg, vcycle


def dense_levels(mg):
    """Dense A_i (i = 1..l) and U_i (i = 1..l-1) of an oracle hierarchy."""
    As, Us = {}, {}
    for i in range(1, mg.l + 1):
        n = mg.size(i)
        As[i] = np.stack([mg.apply(i, e) for e in np.eye(n)], axis=1)
    for i in range(1, mg.l):
        nc = mg.size(i + 1)
        Us[i] = np.stack([mg.prolong(i, e) for e in np.eye(nc)], axis=1)
    return As, Us


def textbook_cg(A, f, x0, n):
    """n Hestenes-Stiefel CG steps on the dense A (rho'/rho form)."""
    x = np.zeros_like(f) if x0 is None else x0.copy()
    r = f - A @ x
    p = r.copy()
    rho = r @ r
    for _ in range(n):
        q = A @ p
        if not (p @ q) > 0:
            break
        al = rho / (p @ q)
        x = x + al * p
        r = r - al * q
        rn = r @ r
        if rn <= (1e-30 * np.linalg.norm(f)) ** 2:
            break
        p = r + (rn / rho) * p
        rho = rn
    return x, r


@pytest.fixture(scope="module")
def small():
    p = W.workload(1, n=1024)
    h = H2Matrix(p["points"], KernelSpec("exponential", 0.1, 1e-2), 32, 3, 1.0)
    return h, p["b"]


def test_fcg_exact_preconditioner_one_step(small):
    h, b = small
    mg = H2MG(h)
    A = h.dense()
    F = sla.cho_factor(A)
    x, info = solve_fcg(mg, b, SolveOpts(tol=1e-12, max_cycles=5), precond=lambda r: sla.cho_solve(F, r))
    assert info.converged and info.cycles == 1, info.history


def test_fcg_identity_preconditioner_is_textbook_cg(small):
    h, b = small
    mg = H2MG(h)
    A = h.dense()
    hist = [1.0]
    x = np.zeros_like(b)
    for k in range(1, 13):
        x, _ = textbook_cg(A, b, None, k)
        hist.append(np.linalg.norm(b - A @ x) / np.linalg.norm(b))
    _, info = solve_fcg(mg, b, SolveOpts(tol=0.0, max_cycles=12), precond=lambda r: r.copy())
    np.testing.assert_allclose(info.history, hist, rtol=1e-8)
    _, icg = solve_cg(mg, b, SolveOpts(tol=0.0, max_cycles=12))
    # the plain CG loop reports the recurrence residual: equal to the explicit one here
    np.testing.assert_allclose(icg.history, hist, rtol=1e-8)


def test_cg_outer_loop_counts_products(small):
    """CG to 1e-8: converged, its explicit residual within a factor of the recurrence
    one, and no more iterations than the matrix dimension."""
    h, b = small
    x, info = solve_cg(H2MG(h), b, SolveOpts(tol=1e-8, max_cycles=2000))
    assert info.converged and 0 < info.cycles <= len(b)
    assert info.relres <= 1e-7


@pytest.fixture(scope="module")
def two_level():
    X = W.uniform_points(600, 2, 3)
    h = H2Matrix(X, KernelSpec("gaussian", 0.2, 1e-2), 16, 3, 1.0, basis="skeleton", tol=1e-8, rank_max=12)
    mg = H2MG(h, coarse_level=2)
    As, Us = dense_levels(mg)
    b = W.normal_rhs(600, 3)
    return mg, As, Us, b


def test_two_level_vcycle_without_smoothing(two_level):
    mg, As, Us, b = two_level
    x0 = 0.3 * W.normal_rhs(600, 4)
    r = b - As[1] @ x0
    want = x0 + Us[1] @ np.linalg.solve(As[2], Us[1].T @ r)
    got = vcycle(mg, x0, r, SolveOpts(n_f=0, n_c=0))
    # the coarse solve by Cholesky against a dense LU solve: rounding of order eps * cond
    tol = 1e-14 * np.linalg.cond(As[2])
    assert np.linalg.norm(got - want) <= tol * np.linalg.norm(want)


def test_two_level_vcycle_with_one_cg_step(two_level):
    """e~ = one CG step from 0; r_2 = U^T(r - A e~); e~ += U A_2^{-1} r_2; one CG step
    from e~ -- written out densely."""
    mg, As, Us, b = two_level
    A, U = As[1], Us[1]
    x0 = np.zeros_like(b)
    r = b.copy()
    al = (r @ r) / (r @ (A @ r))
    et = al * r
    r2 = U.T @ (r - A @ et)
    et = et + U @ np.linalg.solve(As[2], r2)
    rr = r - A @ et
    e = et + ((rr @ rr) / (rr @ (A @ rr))) * rr
    got = vcycle(mg, x0, r, SolveOpts(n_f=1, n_c=0))
    tol = 1e-14 * np.linalg.cond(As[2])
    assert np.linalg.norm(got - e) <= tol * np.linalg.norm(e)
    for kind in ("W", "F"):   # a second visit of an exactly solved level changes nothing
        w = cycle(mg, x0, r, SolveOpts(n_f=1, n_c=0), kind)
        assert np.linalg.norm(w - e) <= tol * np.linalg.norm(e), kind


@pytest.fixture(scope="module")
def deep():
    X = W.uniform_points(1500, 2, 5)
    h = H2Matrix(X, KernelSpec("exponential", 0.2, 1e-2), 16, 3, 1.0, basis="skeleton", tol=1e-8, rank_max=12)
    mg = H2MG(h)
    assert mg.l >= 4
    As, Us = dense_levels(mg)
    return mg, As, Us, W.normal_rhs(1500, 5)


def test_recursive_v_cycle_is_algorithm_1(deep):
    mg, As, Us, b = deep
    o = SolveOpts(n_f=1, n_c=3)
    x0 = np.zeros_like(b)
    np.testing.assert_allclose(cycle(mg, x0, b, o, "V"), vcycle(mg, x0, b, o), rtol=0, atol=1e-14 * 10)


def test_w_and_f_equal_v_without_smoothing(deep):
    """With no smoothing every cycle is P r with P the nested Galerkin coarse
    correction, a projection in the A_i inner products: repeating it changes nothing."""
    mg, As, Us, b = deep
    o = SolveOpts(n_f=0, n_c=0)
    v = vcycle(mg, np.zeros_like(b), b, o)
    for kind in ("W", "F"):
        w = cycle(mg, np.zeros_like(b), b, o, kind)
        assert np.linalg.norm(w - v) <= 1e-10 * np.linalg.norm(v), kind


def dense_cycle(As, Us, l, f, g, kind, n_f, n_c, i=1):
    """The textbook gamma-cycle on dense matrices (pre-smooth from g, restrict the
    residual, visit the coarser level once (V), twice (W) or F-then-V (F), prolong,
    post-smooth); the coarsest level is solved exactly."""
    if i == l:
        return np.linalg.solve(As[l], f)
    n = n_f if i == 1 else n_c
    et, _ = textbook_cg(As[i], f, g, n)
    rc = Us[i].T @ (f - As[i] @ et)
    e = None
    for k in {"V": ("V",), "W": ("W", "W"), "F": ("F", "V")}[kind]:
        e = dense_cycle(As, Us, l, rc, e, k, n_f, n_c, i + 1)
    et = et + Us[i] @ e
    e, _ = textbook_cg(As[i], f, et, n)
    return e


@pytest.mark.parametrize("kind", ["V", "W", "F"])
def test_cycles_match_the_dense_recursion(deep, kind):
    mg, As, Us, b = deep
    o = SolveOpts(n_f=1, n_c=2, explicit_restrict_residual=True)
    want = dense_cycle(As, Us, mg.l, b, None, kind, 1, 2)
    got = cycle(mg, np.zeros_like(b), b, o, kind)
    assert np.linalg.norm(got - want) <= 1e-14 * np.linalg.cond(As[mg.l]) * 10 * np.linalg.norm(want)


# --------------------------------------------------------------------------- the paper's trend
@pytest.mark.parametrize("kernel,sigma,limit", [("gaussian", 0.1, 6), ("exponential", 0.1, 30)])
def test_tensor_grid_cycle_counts_stay_small_and_flat(kernel, sigma, limit):
    """Sec. 4.1 / 4.2: uniform tensor grids on the unit square, exp(-d^2/sigma) and
    exp(-d/sigma) with c = 1e-3, matrices built to relative accuracy 1e-9 (here the
    skeleton bases), b = A x_true, stop at (e^T A e)^{1/2}/|b| < 1e-9, n_f = 1,
    n_c = 40. The paper's Tables report 2 and 14-18 V-cycles at N = 1e4..4e4; here at
    N = 32^2 and 64^2 the counts stay within a few of those, do not grow with N, and
    unpreconditioned CG needs several times more iterations."""
    length = np.sqrt(sigma) if kernel == "gaussian" else sigma
    counts, cgs = [], []
    for m in (32, 64):
        X = W.tensor_grid(m)
        h = H2Matrix(X, KernelSpec(kernel, length, 1e-3), 64, 4, 1.0, basis="skeleton", tol=1e-9)
        mg = H2MG(h)
        xt = W.normal_rhs(m * m, 7)
        b = h.apply(xt)
        _, info = solve(mg, b, SolveOpts(tol=1e-9, max_cycles=limit + 5), x_true=xt)
        assert info.converged, info.history[-3:]
        counts.append(info.cycles)
        _, icg = solve_cg(mg, b, SolveOpts(tol=1e-9, max_cycles=5000), x_true=xt)
        cgs.append(icg.cycles)
    assert max(counts) <= limit, counts
    assert counts[1] <= counts[0] + 2, counts
    assert all(c >= 4 * v for c, v in zip(cgs, counts)), (counts, cgs)
