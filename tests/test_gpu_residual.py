"""The extended-precision outer residual: the level-1 product with double-double
vectors and sums over the float64 blocks (h2mg_apply_level precision F64_DD; the
solve option residual_dd).

* Exactness: with eta = 0 every pair is a close block, and the kernel (1 + x.y)^0 = 1
  stores every entry exactly, so A x = sum(x) + c x is known exactly (math.fsum). With
  entries of 1e11 and both signs the float64 block product loses digits to rounding;
  the double-double product, including its atomic accumulation of the transposed
  partial sums, must keep the exact value to float64 rounding of the result.
* Consistency: on an ordinary matrix with a far field, the double-double product
  equals the float64 product and the oracle's to 1e-13.
* The floor: on the Gaussian at the density of 2^20 points (|x| about 950 |b|) the
  float64 residual cannot be driven much below 1e-11; with the double-double residual
  the same solve reaches 2e-12.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import H2Matrix, KernelSpec

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2501_17656_gb300 as pkg  # noqa: E402

pkg.load_library(build_if_missing=True)


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_double_double_product_is_exact_where_float64_rounds():
    n, c = 3000, 0.25
    X = W.uniform_points(n, 2, 3)
    A = pkg.H2Matrix(cuda(X), "poly", degree=0, nugget=c, leaf=64, q=2, eta=0.0)
    rng = np.random.default_rng(5)
    # pairs a, -a + d: entries near 1e11 whose sum (a few hundred) cancels almost
    # entirely; every value exact in float64 (at most 53 significant bits), while the
    # running sums of a float64 product need more bits than that
    a = rng.integers(-10 ** 11, 10 ** 11, size=n // 2).astype(np.float64)
    d = rng.integers(-4 << 16, 4 << 16, size=n // 2).astype(np.float64) * 0.5 ** 16
    x = np.empty(n)
    x[0::2] = a
    x[1::2] = -a + d
    x = x[rng.permutation(n)]
    total = math.fsum(x.tolist())
    exact = np.array([math.fsum([total, c * v]) for v in x])
    y64 = A.apply_level(1, cuda(x), "f64").cpu().numpy()
    ydd = A.apply_level(1, cuda(x), "f64_dd").cpu().numpy()
    err64 = np.abs(y64 - exact).max()
    errdd = np.abs(ydd - exact).max()
    scale = np.abs(exact).max()
    assert errdd <= 2 * np.finfo(float).eps * scale, (errdd, scale)
    assert err64 > 10 * max(errdd, np.spacing(scale)), (err64, errdd)
    A.close()


@pytest.mark.parametrize("basis", ["chebyshev", "skeleton"])
def test_double_double_product_matches_float64_and_oracle(basis):
    X = W.uniform_points(5000, 3, 4)
    kw = dict(basis=basis, basis_tol=1e-9) if basis == "skeleton" else {}
    A = pkg.H2Matrix(cuda(X), "matern32", length=0.1, nugget=1e-2, leaf=32, q=3, eta=1.0, **kw)
    h = H2Matrix(X, KernelSpec("matern32", 0.1, 1e-2), 32, 3, 1.0,
                 **(dict(basis="skeleton", tol=1e-9) if basis == "skeleton" else {}))
    x = np.random.default_rng(7).standard_normal(5000)
    ydd = A.apply_level(1, cuda(x), "f64_dd").cpu().numpy()
    y64 = A.apply_level(1, cuda(x), "f64").cpu().numpy()
    yo = h.apply(x)
    assert np.linalg.norm(ydd - y64) <= 1e-13 * np.linalg.norm(y64)
    assert np.linalg.norm(ydd - yo) <= 1e-12 * np.linalg.norm(yo)
    A.close()


def test_double_double_rejects_other_levels_and_storage():
    X = W.uniform_points(2000, 2, 1)
    A = pkg.H2Matrix(cuda(X), "exponential", length=0.1, nugget=1e-2, leaf=32, q=3, storage="df64")
    with pytest.raises(pkg.H2MGError):
        A.apply_level(1, cuda(np.ones(2000)), "f64_dd")
    A.close()
    B = pkg.H2Matrix(cuda(X), "exponential", length=0.1, nugget=1e-2, leaf=32, q=3)
    if B.levels >= 2:
        with pytest.raises(pkg.H2MGError):
            B.apply_level(2, cuda(np.ones(B.level_size(2))), "f64_dd")
    B.close()


def test_double_double_residual_removes_the_float64_floor():
    n = 8192
    X = W.uniform_points(n, 3, 2) * (n / 2.0 ** 20) ** (1 / 3)
    b = cuda(W.normal_rhs(n, 2))
    A = pkg.H2Matrix(cuda(X), "gaussian", length=0.05, nugget=1e-3, leaf=64, eta=1.0, basis="skeleton",
                     basis_tol=1e-9, with_f32=True)
    kw = dict(max_cycles=150, outer="fcg", precision="mixed_f32", use_graph=True, raise_on_fail=False)
    x64, i64 = A.solve(b, tol=2e-12, **kw)
    xdd, idd = A.solve(b, tol=2e-12, residual_dd=True, **kw)
    xau, iau = A.solve(b, tol=2e-12, residual_dd="auto", **kw)
    best64 = min(i64.history())
    assert idd.converged, (idd.cycles, min(idd.history()), best64)
    assert iau.converged, (iau.cycles, min(iau.history()), best64)
    assert float(xdd.norm() / b.norm()) > 100      # the |x| >> |b| regime of the floor
    print(f"best float64-residual relres {best64:.2e}; double-double reached {idd.relres:.2e} in {idd.cycles}")
    A.close()
