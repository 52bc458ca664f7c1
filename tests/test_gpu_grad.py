"""GPU adjoint gradients (the differentiation form) against the oracle, central
differences and dense float64 autograd, on the Matern-3/2 workload at 2^12 points."""
import math

import numpy as np
import pytest

import workloads as W
from oracle.grad import derivative_h2, matern_grads
from oracle.h2 import H2Matrix, KernelSpec

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2501_17656_gb300 as pkg  # noqa: E402

N, L_, S_ = 4096, 0.1, 1e-2


@pytest.fixture(scope="module")
def data():
    X = W.uniform_points(N, 3, 4)
    rng = np.random.default_rng(2004)
    return X, rng.standard_normal(N), rng.standard_normal(N)


def cuda(a, grad=False):
    return torch.tensor(a, dtype=torch.float64, device="cuda", requires_grad=grad)


def gpu_loss_grads(X, y, b, l, s, tol=1e-12):
    yt, bt = cuda(y, True), cuda(b, True)
    lt, st = cuda(l, True), cuda(s, True)
    L = pkg.MaternLoss.apply(torch.from_numpy(X).cuda(), yt, bt, lt, st, tol=tol)
    L.backward()
    return L.item(), yt.grad.cpu().numpy(), bt.grad.cpu().numpy(), lt.grad.item(), st.grad.item()


def test_derivative_sibling_matches_oracle(data):
    X, _, _ = data
    A = pkg.H2Matrix(torch.from_numpy(X).cuda(), "matern32", length=L_, nugget=S_, leaf=64, q=4)
    dA = A.sibling("dmatern32_dl", length=L_)
    h = H2Matrix(X, KernelSpec("matern32", L_, S_), 64, 4, 1.0)
    dh = derivative_h2(h, KernelSpec("dmatern32_dl", L_, 0.0))
    v = np.random.default_rng(3).standard_normal(N)
    got = dA.apply(torch.from_numpy(v).cuda()).cpu().numpy()
    ref = dh.apply(v)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-12
    with pytest.raises(pkg.H2MGError):
        dA.solve(torch.from_numpy(v).cuda())
    dA.close()
    A.close()


def test_skeleton_sibling_has_its_own_skeletons(data):
    """A sibling of a skeleton matrix skeletonizes the derivative kernel itself on the
    same tree: ranks and product equal to the oracle's derivative matrix, and within the
    basis tolerance of the dense derivative kernel."""
    X, _, _ = data
    kw = dict(basis="skeleton", basis_tol=1e-9)
    A = pkg.H2Matrix(torch.from_numpy(X).cuda(), "matern32", length=L_, nugget=S_, leaf=32, q=4, **kw)
    dA = A.sibling("dmatern32_dl", length=L_)
    h = H2Matrix(X, KernelSpec("matern32", L_, S_), 32, 4, 1.0, basis="skeleton", tol=1e-9)
    dh = derivative_h2(h, KernelSpec("dmatern32_dl", L_, 0.0))
    for ell in range(dh.tstar, dh.L + 1):
        assert list(dA.export("RANKS", ell)) == [dh.rank[(ell, j)] for j in range(1 << ell)], ell
    v = np.random.default_rng(5).standard_normal(N)
    got = dA.apply(torch.from_numpy(v).cuda()).cpu().numpy()
    ref = dh.apply(v)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-12
    Xt = torch.from_numpy(X).cuda()
    r = torch.cdist(Xt, Xt)
    Kd = 3.0 * r ** 2 / L_ ** 3 * torch.exp(-math.sqrt(3.0) * r / L_)
    exact = (Kd @ torch.from_numpy(v).cuda()).cpu().numpy()
    assert np.linalg.norm(got - exact) / np.linalg.norm(exact) < 1e-10
    dA.close()
    A.close()


def test_adjoint_gradients_match_oracle(data):
    X, y, b = data
    L, gy, gb, gl, gs = gpu_loss_grads(X, y, b, L_, S_)
    Lo, a, w, dl, ds = matern_grads(X, y, b, L_, S_, leaf=64, q=4)
    assert abs(L - Lo) <= 1e-9 * abs(Lo)
    assert np.linalg.norm(gy - a) <= 1e-8 * np.linalg.norm(a)
    assert np.linalg.norm(gb - w) <= 1e-8 * np.linalg.norm(w)
    assert abs(gl - dl) <= 1e-8 * abs(dl)
    assert abs(gs - ds) <= 1e-8 * abs(ds)


def test_adjoint_gradients_match_central_differences(data):
    X, y, b = data
    _, _, _, gl, gs = gpu_loss_grads(X, y, b, L_, S_, tol=1e-13)

    def loss(l, s):
        with torch.no_grad():
            return pkg.MaternLoss.apply(torch.from_numpy(X).cuda(), cuda(y), cuda(b), cuda(l), cuda(s),
                                        tol=1e-13).item()

    h = 1e-4
    fd_l = (loss(L_ * (1 + h), S_) - loss(L_ * (1 - h), S_)) / (2 * h * L_)
    fd_s = (loss(L_, S_ * (1 + h)) - loss(L_, S_ * (1 - h))) / (2 * h * S_)
    assert abs(gl - fd_l) <= 1e-6 * abs(fd_l), (gl, fd_l)
    assert abs(gs - fd_s) <= 1e-6 * abs(fd_s), (gs, fd_s)


def test_adjoint_gradients_near_dense_autograd(data):
    """Against the exact (dense) kernel the difference is the H2 compression error of
    the 4x4x4-node interpolation, not an error of the adjoint."""
    X, y, b = data
    L, gy, gb, gl, gs = gpu_loss_grads(X, y, b, L_, S_)
    Xt = torch.tensor(X, dtype=torch.float64, device="cuda")
    lt, st = cuda(L_, True), cuda(S_, True)
    yt, bt = cuda(y, True), cuda(b, True)
    u = math.sqrt(3.0) * torch.cdist(Xt, Xt) / lt
    K = (1 + u) * torch.exp(-u) + st * torch.eye(N, dtype=torch.float64, device="cuda")
    Lt = 0.5 * yt @ torch.linalg.solve(K, yt) + torch.linalg.solve(K, bt).sum()
    Lt.backward()
    assert abs(L - Lt.item()) <= 1e-3 * abs(Lt.item())
    assert abs(gl - lt.grad.item()) <= 1e-2 * abs(lt.grad.item())
    assert abs(gs - st.grad.item()) <= 1e-2 * abs(st.grad.item())
    assert np.linalg.norm(gb - bt.grad.cpu().numpy()) <= 1e-2 * np.linalg.norm(gb)


def test_skeleton_gradients_match_dense_autograd_closely(data):
    """With bases skeletonized to 1e-9 the H2 loss is within the compression error of
    the exact one, so the adjoint gradients agree with dense float64 autograd to about
    1e-6 instead of the 1e-2 of the 4x4x4-node interpolation, and central differences of
    the rebuilt loss (step 1e-6, solves to 1e-13) match them to 1e-6."""
    X, y, b = data
    kw = dict(tol=1e-13, basis="skeleton", basis_tol=1e-10)
    Xd = torch.from_numpy(X).cuda()
    yt, bt, lt, st = cuda(y, True), cuda(b, True), cuda(L_, True), cuda(S_, True)
    L = pkg.MaternLoss.apply(Xd, yt, bt, lt, st, **kw)
    L.backward()
    Xt = torch.tensor(X, dtype=torch.float64, device="cuda")
    l2, s2, y2, b2 = cuda(L_, True), cuda(S_, True), cuda(y, True), cuda(b, True)
    u = math.sqrt(3.0) * torch.cdist(Xt, Xt) / l2
    K = (1 + u) * torch.exp(-u) + s2 * torch.eye(N, dtype=torch.float64, device="cuda")
    Lt = 0.5 * y2 @ torch.linalg.solve(K, y2) + torch.linalg.solve(K, b2).sum()
    Lt.backward()
    assert abs(L.item() - Lt.item()) <= 1e-7 * abs(Lt.item())
    assert abs(lt.grad.item() - l2.grad.item()) <= 1e-6 * abs(l2.grad.item())
    assert abs(st.grad.item() - s2.grad.item()) <= 1e-6 * abs(s2.grad.item())
    assert np.linalg.norm((bt.grad - b2.grad).cpu().numpy()) <= 1e-6 * np.linalg.norm(b2.grad.cpu().numpy())

    def loss(l, s):
        with torch.no_grad():
            return pkg.MaternLoss.apply(Xd, cuda(y), cuda(b), cuda(l), cuda(s), **kw).item()

    h = 1e-6
    fd_l = (loss(L_ * (1 + h), S_) - loss(L_ * (1 - h), S_)) / (2 * h * L_)
    fd_s = (loss(L_, S_ * (1 + h)) - loss(L_, S_ * (1 - h))) / (2 * h * S_)
    assert abs(lt.grad.item() - fd_l) <= 1e-6 * abs(fd_l), (lt.grad.item(), fd_l)
    assert abs(st.grad.item() - fd_s) <= 1e-6 * abs(fd_s), (st.grad.item(), fd_s)


def test_loss_call_rejects_a_foreign_derivative_matrix(data):
    X, y, b = data
    Xd = torch.from_numpy(X).cuda()
    K = pkg.H2Matrix(Xd, "matern32", length=L_, nugget=S_, leaf=64, q=4)
    G = pkg.H2Matrix(Xd, "gaussian", length=L_, nugget=S_, leaf=64, q=4)
    dG = G.sibling("dmatern32_dl", length=L_)
    o = pkg.H2Matrix._opts(tol=1e-10)
    loss, dl = pkg.ctypes.c_double(), pkg.ctypes.c_double()
    yy, bb = cuda(y), cuda(b)
    st = K._lib.h2mg_matern_loss_grad(K._h, dG._h, pkg._ptr(yy), pkg._ptr(bb), pkg.ctypes.byref(o),
                                      pkg.ctypes.byref(loss), None, None, pkg.ctypes.byref(dl), None, None,
                                      pkg._stream())
    assert st == 1          # dK is not K's sibling
    st = G._lib.h2mg_matern_loss_grad(G._h, None, pkg._ptr(yy), pkg._ptr(bb), pkg.ctypes.byref(o),
                                      pkg.ctypes.byref(loss), None, None, None, None, None, pkg._stream())
    assert st == 1          # not a Matern matrix
    dG.close()
    G.close()
    K.close()
