"""Pins of the oracle's adjoint gradients (test infrastructure, CPU).

* central finite differences of the oracle's own H2 loss (dense solves);
* dense float64 torch autograd of the exact kernel loss, with 12 x 12 nodes so that
  the H2 form differs from the dense matrix only by the interpolation error
  (< 1e-9 entrywise), which bounds the gradient differences;
* the closed forms dL/db = A^{-1} 1 and dL/ds = -1/2 a^T a - w^T x.
"""
import numpy as np
import pytest

from oracle.grad import derivative_h2, matern_grads, matern_loss
from oracle.h2 import H2Matrix, KernelSpec
from oracle.kernels import dense_kernel_matrix

torch = pytest.importorskip("torch")


def setup(n=600, dim=3, seed=4):
    rng = np.random.default_rng(seed)
    return rng.random((n, dim)), rng.standard_normal(n), rng.standard_normal(n)


def test_derivative_h2_is_the_h2_derivative():
    """dA/dl built on A's bases equals the finite difference of A's H2 form."""
    X, _, _ = setup()
    l, h = 0.3, 1e-6
    A = H2Matrix(X, KernelSpec("matern32", l, 0.1), 32, 3, 1.0)
    dA = derivative_h2(A, KernelSpec("dmatern32_dl", l, 0.0))
    Ap = H2Matrix(X, KernelSpec("matern32", l + h, 0.1), 32, 3, 1.0)
    Am = H2Matrix(X, KernelSpec("matern32", l - h, 0.1), 32, 3, 1.0)
    v = np.random.default_rng(1).standard_normal(600)
    fd = (Ap.apply(v) - Am.apply(v)) / (2 * h)
    assert np.linalg.norm(dA.apply(v) - fd) / np.linalg.norm(fd) < 1e-7


@pytest.mark.parametrize("q", [3, 4])
def test_gradients_match_central_differences(q):
    X, y, b = setup()
    l, s = 0.3, 0.1
    L, a, w, dl, ds = matern_grads(X, y, b, l, s, leaf=32, q=q)
    h = 1e-5
    Lp = matern_loss(X, y, b, l + h * l, s, leaf=32, q=q)[0]
    Lm = matern_loss(X, y, b, l - h * l, s, leaf=32, q=q)[0]
    fd_l = (Lp - Lm) / (2 * h * l)
    Lp = matern_loss(X, y, b, l, s + h, leaf=32, q=q)[0]
    Lm = matern_loss(X, y, b, l, s - h, leaf=32, q=q)[0]
    fd_s = (Lp - Lm) / (2 * h)
    assert abs(dl - fd_l) <= 1e-6 * abs(fd_l)
    assert abs(ds - fd_s) <= 1e-6 * abs(fd_s)
    # dL/db along a random direction
    d = np.random.default_rng(7).standard_normal(600)
    Lp = matern_loss(X, y, b + h * d, l, s, leaf=32, q=q)[0]
    Lm = matern_loss(X, y, b - h * d, l, s, leaf=32, q=q)[0]
    assert abs((Lp - Lm) / (2 * h) - w @ d) <= 1e-6 * abs(w @ d)


def test_gradients_match_dense_autograd():
    X, y, b = setup(n=1024, dim=2)
    l, s = 0.2, 0.05
    A = H2Matrix(X, KernelSpec("matern32", l, s), 16, 12, 1.0)
    assert A.tstar is not None
    Kd = dense_kernel_matrix("matern32", X, l, s)
    assert np.abs(A.dense() - Kd).max() < 1e-9
    L, a, w, dl, ds = matern_grads(X, y, b, l, s, leaf=16, q=12)
    Xt = torch.tensor(X, dtype=torch.float64)
    lt = torch.tensor(l, dtype=torch.float64, requires_grad=True)
    st = torch.tensor(s, dtype=torch.float64, requires_grad=True)
    yt = torch.tensor(y, dtype=torch.float64, requires_grad=True)
    bt = torch.tensor(b, dtype=torch.float64, requires_grad=True)
    r = torch.cdist(Xt, Xt)
    u = np.sqrt(3.0) * r / lt
    K = (1 + u) * torch.exp(-u) + st * torch.eye(1024, dtype=torch.float64)
    Lt = 0.5 * yt @ torch.linalg.solve(K, yt) + torch.linalg.solve(K, bt).sum()
    Lt.backward()
    assert abs(L - Lt.item()) <= 1e-6 * abs(L)
    assert abs(dl - lt.grad.item()) <= 1e-5 * abs(lt.grad.item())
    assert abs(ds - st.grad.item()) <= 1e-5 * abs(st.grad.item())
    assert np.linalg.norm(w - bt.grad.numpy()) <= 1e-6 * np.linalg.norm(w)
    assert np.linalg.norm(a - yt.grad.numpy()) <= 1e-6 * np.linalg.norm(a)


def test_skeleton_derivative_matrix_has_its_own_skeletons():
    """With skeleton bases, dA/dl is the derivative kernel's own skeleton H2 matrix on A's
    tree and partition: within the basis tolerance of the dense derivative kernel
    (3 r^2 / l^3) exp(-sqrt3 r / l) (zero diagonal), with skeletons of its own."""
    rng = np.random.default_rng(8)
    X = rng.random((3000, 3))
    l = 0.1
    A = H2Matrix(X, KernelSpec("matern32", l, 1e-2), 32, 4, 1.0, basis="skeleton", tol=1e-9)
    assert A.tstar is not None
    dA = derivative_h2(A, KernelSpec("dmatern32_dl", l, 0.0))
    assert dA.tree is A.tree and dA.far is A.far
    Kd = dense_kernel_matrix("dmatern32_dl", X, l, 0.0)
    assert np.abs(np.diag(Kd)).max() == 0.0
    v = rng.standard_normal(3000)
    ref = Kd @ v
    # its own skeletons: ~5e-13 here; the matrix's skeletons with derivative couplings
    # would give ~1e-7 (they do not span the derivative kernel's far field)
    assert np.linalg.norm(dA.apply(v) - ref) / np.linalg.norm(ref) < 1e-10
    # the derivative kernel's skeletons differ from the matrix's own somewhere
    diff = [key for key in A.skeletons.skel if not np.array_equal(A.skeletons.skel[key], dA.skeletons.skel[key])]
    assert diff
