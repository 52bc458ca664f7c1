"""GPU parity of the W- and F-cycles and of the unpreconditioned CG outer loop.

The cycles with short smoothers are smooth functions of their input, so on a
Chebyshev hierarchy (operators equal to the oracle's to 1e-12) one GPU cycle agrees
with the oracle's recursion to 1e-9, as the V-cycle does. Full solves on the paper's
2-D tensor-grid exponential workload (Sec. 4.2, skeleton bases to 1e-9) converge in
the oracle's number of V-cycles +-1 (W- and F-cycles +-2); the CG outer loop runs
hundreds of iterations, so
its count is compared within 2% (at least +-2) and its first twenty residuals at 1e-6.
"""
import numpy as np
import pytest

import workloads as W
from oracle import H2MG, H2Matrix, KernelSpec, SolveOpts, cycle, solve, solve_cg, solve_fcg

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


@pytest.fixture(scope="module")
def deep_cheb():
    X = W.uniform_points(3001, 1, 9)
    A = pkg.H2Matrix(cuda(X), "exponential", length=0.05, nugget=1e-2, leaf=16, q=6, eta=1.0)
    h = H2Matrix(X, KernelSpec("exponential", 0.05, 1e-2), 16, 6, 1.0)
    mg = H2MG(h)
    assert mg.l >= 4 and mg.chol is not None
    yield A, h, mg
    A.close()


@pytest.mark.parametrize("kind", ["V", "W", "F"])
def test_one_cycle_matches_the_oracle(deep_cheb, kind):
    A, h, mg = deep_cheb
    b = np.random.default_rng(21).standard_normal(h.tree.n)
    x0 = np.zeros_like(b)
    xg = A.vcycle(cuda(x0), cuda(b), n_f=1, n_c=2, cycle=kind).cpu().numpy()
    xo = cycle(mg, x0, b, SolveOpts(n_f=1, n_c=2), kind)
    assert rel(xg, xo) < 1e-9, kind
    if kind != "V":
        xv = cycle(mg, x0, b, SolveOpts(n_f=1, n_c=2), "V")
        assert rel(xo, xv) > 1e-6       # the cycles really differ


@pytest.fixture(scope="module")
def grid_exp():
    X = W.tensor_grid(64)
    xt = W.normal_rhs(4096, 7)
    A = pkg.H2Matrix(cuda(X), "exponential", length=0.1, nugget=1e-3, leaf=64, eta=1.0, basis="skeleton",
                     basis_tol=1e-9, with_f32=True)
    h = H2Matrix(X, KernelSpec("exponential", 0.1, 1e-3), 64, 4, 1.0, basis="skeleton", tol=1e-9)
    mg = H2MG(h)
    b = h.apply(xt)
    yield A, h, mg, b
    A.close()


@pytest.mark.parametrize("kind", ["V", "W", "F"])
def test_tensor_grid_solves_match_cycle_counts(grid_exp, kind):
    A, h, mg, b = grid_exp
    assert mg.l >= 3
    xo, io = solve(mg, b, SolveOpts(tol=1e-9, max_cycles=60, cycle=kind))
    xg, ig = A.solve(cuda(b), tol=1e-9, max_cycles=60, cycle=kind, use_graph=True)
    assert io.converged and ig.converged
    # a W- or F-cycle visits the coarse levels many times per cycle (2^(i-1) or i), each
    # visit a nonlinear CG smoothing on operators that differ from the oracle's by
    # about eps / tol (skeleton bases): one cycle more or less either way
    band = 1 if kind == "V" else 2
    assert abs(ig.cycles - io.cycles) <= band, (kind, ig.cycles, io.cycles)
    r = b - h.apply(xg.cpu().numpy())
    assert np.linalg.norm(r) / np.linalg.norm(b) <= 1e-9 * 1.0001
    # flexible CG preconditioned by the same cycle, in mixed precision
    xf, jf = A.solve(cuda(b), tol=1e-9, max_cycles=60, cycle=kind, outer="fcg", precision="mixed_f32",
                     use_graph=True)
    assert jf.converged
    r = b - h.apply(xf.cpu().numpy())
    assert np.linalg.norm(r) / np.linalg.norm(b) <= 1e-9 * 1.0001


def test_cg_outer_loop_matches_the_oracle(grid_exp):
    """Unpreconditioned CG, the paper's comparison solver: the GPU's iteration count
    and residual history against the oracle's textbook CG, and far more iterations
    than H2-MG needs cycles (Sec. 4: CG iterations grow, V-cycles do not)."""
    A, h, mg, b = grid_exp
    xo, io = solve_cg(mg, b, SolveOpts(tol=1e-9, max_cycles=3000))
    xg, ig = A.solve(cuda(b), tol=1e-9, max_cycles=3000, outer="cg")
    assert io.converged and ig.converged
    assert abs(ig.cycles - io.cycles) <= max(2, 0.02 * io.cycles), (ig.cycles, io.cycles)
    np.testing.assert_allclose(ig.history()[:20], io.history[:20], rtol=1e-6)
    r = b - h.apply(xg.cpu().numpy())
    assert np.linalg.norm(r) / np.linalg.norm(b) <= 2e-9
    _, iv = solve(mg, b, SolveOpts(tol=1e-9, max_cycles=60))
    assert ig.cycles >= 5 * iv.cycles


def test_unknown_cycle_and_outer_are_rejected(grid_exp):
    A, h, mg, b = grid_exp
    o = pkg.H2Matrix._opts(tol=1e-9)
    o.cycle = 3
    info = pkg.SolveInfo()
    x = torch.zeros(len(b), dtype=torch.float64, device="cuda")
    st = A._lib.h2mg_solve(A._h, pkg._ptr(cuda(b)), pkg._ptr(x), 1, len(b), pkg.ctypes.byref(o),
                           pkg.ctypes.byref(info), pkg._stream())
    assert st == 1
    o.cycle = 0
    o.outer = 7
    st = A._lib.h2mg_solve(A._h, pkg._ptr(cuda(b)), pkg._ptr(x), 1, len(b), pkg.ctypes.byref(o),
                           pkg.ctypes.byref(info), pkg._stream())
    assert st == 1
