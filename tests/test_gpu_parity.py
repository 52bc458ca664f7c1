"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Every expected value comes from ``oracle/``; every input from ``workloads``.
Tolerance: 1e-12 relative (2-norm) for the linear operators (matvec, level
operators, coarse solve), as the H2 matvec target states; short CG runs are
compared at 1e-10; full solves (CG smoothers with tens of iterations are
sensitive to rounding order, so iterates are not comparable bit for bit) by the
final float64 residual and the V-cycle count within 25% (at least +-2): on the
4096-point exponential workload the oracle's own count moves over 113..123 cycles
(repeated V-cycles, tol 1e-8) and 86..97 (flexible CG, tol 1e-9) when b is
perturbed by 1e-15 to 1e-12 relative, and six GPU solves of the same system take
85..101 flexible-CG cycles, so a tighter band would test rounding order, not the
method.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import H2MG, H2Matrix, KernelSpec, SolveOpts, dense_kernel_matrix, solve, solve_fcg, surface_diag

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2501_17656_gb300 as pkg  # noqa: E402

pkg.load_library(build_if_missing=True)


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def build_pair(X, kind, length=1.0, nugget=0.0, leaf=64, q=4, eta=1.0, weights=None, diag=None,
               degree=2, storage="f64", with_f32=False, coarse_level=-1):
    A = pkg.H2Matrix(cuda(X), kind, length=length, nugget=nugget, degree=degree,
                     weights=None if weights is None else cuda(weights),
                     diag=None if diag is None else cuda(diag), leaf=leaf, q=q, eta=eta,
                     storage=storage, with_f32=with_f32, coarse_level=coarse_level)
    h = H2Matrix(X, KernelSpec(kind, length, nugget, degree, weights, diag), leaf, q, eta)
    return A, h


CASES = {
    "w1_exp2d": lambda: (W.workload(1)["points"], dict(kind="exponential", length=0.1, nugget=1e-2, leaf=64, q=4)),
    "gauss3d_8k": lambda: (W.uniform_points(8192, 3, 2), dict(kind="gaussian", length=0.05, nugget=1e-3, leaf=64, q=4)),
    "gauss3d_wide": lambda: (W.uniform_points(8192, 3, 2), dict(kind="gaussian", length=0.3, nugget=1e-3, leaf=64, q=3)),
    "matern3d_ragged": lambda: (W.uniform_points(5000, 3, 4), dict(kind="matern32", length=0.1, nugget=1e-2, leaf=32, q=3)),
    "exp1d_ragged": lambda: (W.uniform_points(3001, 1, 9), dict(kind="exponential", length=0.05, nugget=1e-2, leaf=16, q=6)),
    "exp2d_leaf16": lambda: (W.uniform_points(4000, 2, 5), dict(kind="exponential", length=0.1, nugget=1e-2, leaf=16, q=2)),
}


@pytest.fixture(scope="module", params=sorted(CASES))
def pair(request):
    X, kw = CASES[request.param]()
    A, h = build_pair(X, **kw)
    yield request.param, X, A, h
    A.close()


def test_structure_matches_oracle(pair):
    name, X, A, h = pair
    T = h.tree
    assert A.query("L") == T.L
    assert A.query("TSTAR") == (-1 if h.tstar is None else h.tstar)
    # leaves as point sets
    perm = A.export("PERM")
    off = A.export("LEAF_OFFSETS")
    assert np.array_equal(off, T.offsets[T.L])
    for j in range(1 << T.L):
        assert set(perm[off[j]:off[j + 1]].tolist()) == set(T.perm[T.rows(T.L, j)].tolist())
    near = A.export("NEAR").reshape(-1, 2)
    on = h.near[h.near[:, 1] >= h.near[:, 0]]
    assert np.array_equal(near, on)
    for ell in range(T.L + 1):
        far = A.export("FAR", ell).reshape(-1, 2)
        of = h.far[ell][h.far[ell][:, 1] > h.far[ell][:, 0]]
        assert np.array_equal(far, of), ell
        boxes = A.export("BOXES", ell).reshape(-1, 2, X.shape[1])
        assert np.array_equal(boxes[:, 0], T.lo[ell]) and np.array_equal(boxes[:, 1], T.hi[ell])


def test_matvec_matches_oracle(pair):
    name, X, A, h = pair
    rng = np.random.default_rng(11)
    for _ in range(2):
        x = rng.standard_normal(X.shape[0])
        y = A.apply(cuda(x)).cpu().numpy()
        assert rel(y, h.apply(x)) < 1e-12, name


def test_matvec_host_buffers(pair):
    name, X, A, h = pair
    x = np.random.default_rng(12).standard_normal(X.shape[0])
    y = A.apply(x)                      # NumPy in, NumPy out: staged by the library
    assert rel(y, h.apply(x)) < 1e-12


def _pad(mg, i, v, KC):
    """oracle level-i coefficients (ragged ranks) -> padded GPU layout"""
    h = mg.h
    m = mg.m(i)
    off = h.coef_offsets(m)
    out = np.zeros((1 << m) * KC)
    for j in range(1 << m):
        out[j * KC: j * KC + off[j + 1] - off[j]] = v[off[j]:off[j + 1]]
    return out


def _unpad(mg, i, v, KC):
    h = mg.h
    m = mg.m(i)
    off = h.coef_offsets(m)
    return np.concatenate([v[j * KC: j * KC + off[j + 1] - off[j]] for j in range(1 << m)])


def test_level_operators_match_oracle(pair):
    name, X, A, h = pair
    if h.tstar is None:
        pytest.skip("no far field")
    mg = H2MG(h)
    assert A.levels == mg.l
    KC = A.query("KC")
    rng = np.random.default_rng(13)
    for i in range(2, mg.l + 1):
        v = rng.standard_normal(mg.size(i))
        y = A.apply_level(i, cuda(_pad(mg, i, v, KC))).cpu().numpy()
        assert rel(_unpad(mg, i, y, KC), mg.apply(i, v)) < 1e-12, (name, i)


def test_coarse_solve_matches_oracle(pair):
    name, X, A, h = pair
    mg = H2MG(h)
    l = mg.l
    r = np.random.default_rng(14).standard_normal(mg.size(l))
    if l == 1:
        e = A.coarse_solve(cuda(r)).cpu().numpy()
        assert rel(e, mg.dir_sol(r)) < 1e-10
        return
    KC = A.query("KC")
    if mg.chol is None:
        # the interpolation error exceeds the smallest eigenvalue: both sides must
        # find the coarse operator indefinite
        with pytest.raises(pkg.H2MGError) as err:
            A.coarse_solve(cuda(_pad(mg, l, r, KC)))
        assert err.value.name == "NOT_SPD"
        return
    e = A.coarse_solve(cuda(_pad(mg, l, r, KC))).cpu().numpy()
    ref = mg.dir_sol(r)
    kappa = np.linalg.cond(mg.Al)
    assert rel(_unpad(mg, l, e, KC), ref) < max(1e-12, 1e-15 * kappa), (name, kappa)


@pytest.mark.parametrize("n_it", [1, 3])
def test_smoother_matches_oracle(pair, n_it):
    name, X, A, h = pair
    mg = H2MG(h)
    from oracle import cg
    rng = np.random.default_rng(15)
    f = rng.standard_normal(X.shape[0])
    x, r = A.smooth(1, cuda(f), None, n_it)
    xo, ro = cg(lambda v: mg.apply(1, v), f, None, n_it)
    assert rel(x.cpu().numpy(), xo) < 1e-10 and rel(r.cpu().numpy(), ro) < 1e-10
    if mg.l >= 3:
        KC = A.query("KC")
        f2 = rng.standard_normal(mg.size(2))
        x0 = rng.standard_normal(mg.size(2))
        x, r = A.smooth(2, cuda(_pad(mg, 2, f2, KC)), cuda(_pad(mg, 2, x0, KC)), n_it)
        xo, ro = cg(lambda v: mg.apply(2, v), f2, x0, n_it)
        assert rel(_unpad(mg, 2, x.cpu().numpy(), KC), xo) < 1e-10


def test_vcycle_matches_oracle_short_smoothing(pair):
    """With short smoothers the V-cycle is a smooth function of its input, so the
    GPU and the oracle agree to rounding."""
    name, X, A, h = pair
    mg = H2MG(h)
    if mg.chol is None:
        pytest.skip("indefinite H2 approximation")
    from oracle.mg import vcycle
    b = np.random.default_rng(16).standard_normal(X.shape[0])
    o = SolveOpts(n_f=1, n_c=2)
    x0 = np.zeros_like(b)
    xg = A.vcycle(cuda(x0), cuda(b), n_f=1, n_c=2).cpu().numpy()
    xo = vcycle(mg, x0, b, o)
    assert rel(xg, xo) < 1e-9, name
    # no smoothing where the restriction is square (the GPU decides per cluster, the
    # oracle by level sizes)
    o2 = SolveOpts(n_f=1, n_c=2, skip_square_levels=True)
    xg2 = A.vcycle(cuda(x0), cuda(b), n_f=1, n_c=2, skip_square_levels=True).cpu().numpy()
    xo2 = vcycle(mg, x0, b, o2)
    assert rel(xg2, xo2) < 1e-9, name
    square = any(mg.size(i) == mg.size(i - 1) for i in range(2, mg.l))
    assert (rel(xo2, xo) > 1e-6) == square, name


def test_solve_cycles_match_oracle():
    p = W.workload(1)
    A, h = build_pair(p["points"], "exponential", 0.1, 1e-2, 64, 4)
    mg = H2MG(h)
    tol = 1e-8
    xg, info = A.solve(cuda(p["b"]), tol=tol, max_cycles=300)
    xo, io = solve(mg, p["b"], SolveOpts(tol=tol, max_cycles=300))
    assert info.converged and io.converged
    assert abs(info.cycles - io.cycles) <= max(2, 0.25 * io.cycles), (info.cycles, io.cycles)
    xg = xg.cpu().numpy()
    r = p["b"] - h.apply(xg)
    assert np.linalg.norm(r) / np.linalg.norm(p["b"]) <= tol * 1.0001
    # against the dense Cholesky solution of the H2 matrix (kappa * tol)
    Ad = h.dense()
    xd = np.linalg.solve(Ad, p["b"])
    assert rel(xg, xd) < np.linalg.cond(Ad) * tol


@pytest.mark.parametrize("storage", ["df64"])
def test_double_float_storage_matvec(storage):
    X = W.uniform_points(8192, 3, 2)
    A, h = build_pair(X, "gaussian", 0.05, 1e-3, 64, 4, storage=storage)
    x = np.random.default_rng(3).standard_normal(8192)
    assert rel(A.apply(cuda(x)).cpu().numpy(), h.apply(x)) < 1e-12
    mg = H2MG(h)
    KC = A.query("KC")
    for i in range(2, mg.l + 1):
        v = np.random.default_rng(i).standard_normal(mg.size(i))
        y = A.apply_level(i, cuda(_pad(mg, i, v, KC))).cpu().numpy()
        assert rel(_unpad(mg, i, y, KC), mg.apply(i, v)) < 1e-12, i


def test_polynomial_kernel_full_size_rows():
    """At any size the H2 matvec of a low-degree polynomial kernel equals the dense
    matvec (interpolation is exact); sampled rows are checked by brute force."""
    n = 1 << 17
    X = W.uniform_points(n, 3, 7)
    A = pkg.H2Matrix(cuda(X), "poly", nugget=0.5, degree=2, leaf=64, q=4, eta=1.0)
    x = np.random.default_rng(5).standard_normal(n)
    y = A.apply(cuda(x)).cpu().numpy()
    rows = np.random.default_rng(6).choice(n, 64, replace=False)
    Kr = (1.0 + X[rows] @ X.T) ** 2
    Kr[np.arange(64), rows] += 0.5
    yr = Kr @ x
    assert rel(y[rows], yr) < 1e-12


def test_surface_kernel_weights_and_diagonal():
    """Single-layer kernel on a perturbed sphere: the library forms the panel
    self-interaction from the areas itself; the oracle from its own formula."""
    c, a, _ = W.perturbed_icosphere(12, 0)
    A = pkg.H2Matrix(cuda(c), "laplace_sl", weights=cuda(a), leaf=64, q=3)
    h = H2Matrix(c, KernelSpec("laplace_sl", 1.0, 0.0, 2, a, surface_diag(a)), 64, 3, 1.0)
    x = np.random.default_rng(8).standard_normal(c.shape[0])
    assert rel(A.apply(cuda(x)).cpu().numpy(), h.apply(x)) < 1e-12
    # an explicit diagonal override is used as given
    dg = np.random.default_rng(9).uniform(0.01, 0.02, c.shape[0])
    A2, h2 = build_pair(c, "laplace_sl", 1.0, 0.0, 64, 3, weights=a, diag=dg)
    assert rel(A2.apply(cuda(x)).cpu().numpy(), h2.apply(x)) < 1e-12
    A.close()
    A2.close()


def test_fp32_product_after_float64_product_on_ragged_leaves():
    """Leaves of about 40 points padded to 64 slots: the FP32 product must not read
    what a float64 product left in the shared point buffer (as floats those bytes can
    be NaN)."""
    c, a, _ = W.perturbed_icosphere(16, 0)
    A = pkg.H2Matrix(cuda(c), "laplace_sl", weights=cuda(a), leaf=64, q=4, with_f32=True)
    x = cuda(np.random.default_rng(2).standard_normal(c.shape[0]))
    for _ in range(2):
        y64 = A.apply_level(1, x, "f64")
        y32 = A.apply_level(1, x, "mixed_f32")
        assert bool(torch.isfinite(y32).all())
        assert float((y32 - y64).norm() / y64.norm()) < 1e-5
        X = torch.stack([x, 2 * x, -x, x]).t()
        A.apply(X)                                   # two-column float64 groups
    A.close()


@pytest.mark.parametrize("m,j", [(20, 1), (16, 0)])
def test_surface_problem_solves_like_oracle(m, j):
    c, a, _ = W.perturbed_icosphere(m, j)
    A = pkg.H2Matrix(cuda(c), "laplace_sl", weights=cuda(a), leaf=64, q=4, with_f32=True)
    h = H2Matrix(c, KernelSpec("laplace_sl", 1.0, 0.0, 2, a, surface_diag(a)), 64, 4, 1.0)
    b = W.normal_rhs(c.shape[0], 3)
    _, io = solve_fcg(H2MG(h), b, SolveOpts(tol=1e-10, max_cycles=50))
    for prec in ("f64", "mixed_f32"):
        x, info = A.solve(cuda(b), tol=1e-10, max_cycles=50, outer="fcg", precision=prec)
        assert info.converged and io.converged
        assert abs(info.cycles - io.cycles) <= 2, (prec, info.cycles, io.cycles)
        r = b - h.apply(x.cpu().numpy())
        assert np.linalg.norm(r) / np.linalg.norm(b) <= 1e-10 * 1.0001
    A.close()


def test_mixed_precision_solve_reaches_float64_tolerance():
    X = W.uniform_points(8192, 3, 2)
    A, h = build_pair(X, "gaussian", 0.05, 1e-3, 64, 4, with_f32=True)
    b = W.normal_rhs(8192, 2)
    x, info = A.solve(cuda(b), tol=1e-10, max_cycles=100, precision="mixed_f32")
    assert info.converged
    r = b - h.apply(x.cpu().numpy())
    assert np.linalg.norm(r) / np.linalg.norm(b) <= 1e-10 * 1.0001


def test_invalid_arguments_rejected_before_launch():
    X = cuda(W.uniform_points(100, 2, 1))
    with pytest.raises(pkg.H2MGError) as e:
        pkg.H2Matrix(X, "gaussian", length=-1.0)
    assert e.value.name == "INVALID_ARG"
    with pytest.raises(pkg.H2MGError):
        pkg.H2Matrix(X, "gaussian", length=1.0, leaf=1)
    bad = W.uniform_points(100, 2, 1)
    bad[3, 1] = np.nan
    with pytest.raises(pkg.H2MGError) as e:
        pkg.H2Matrix(cuda(bad), "gaussian", length=1.0)
    assert e.value.name == "INVALID_ARG"


def test_not_converged_and_nan_statuses():
    p = W.workload(1, n=2048)
    A = pkg.H2Matrix(cuda(p["points"]), "exponential", length=0.1, nugget=1e-2, leaf=64, q=4)
    x, info = A.solve(cuda(p["b"]), tol=1e-16, max_cycles=1, raise_on_fail=False)
    assert info.cycles == 1 and not info.converged
    bad = p["b"].copy()
    bad[0] = np.inf
    with pytest.raises(pkg.H2MGError) as e:
        A.solve(cuda(bad), tol=1e-8, max_cycles=3)
    assert e.value.name == "NAN"


def test_not_spd_reported():
    X = W.uniform_points(600, 2, 3)
    A = pkg.H2Matrix(cuda(X), "exponential", length=0.1, nugget=-5.0, leaf=32, q=3)
    with pytest.raises(pkg.H2MGError) as e:
        A.solve(cuda(np.ones(600)), tol=1e-8, max_cycles=2)
    assert e.value.name == "NOT_SPD"
