"""The many-right-hand-side product on the tensor cores (h2mg_apply_ex, TF32X3).

Every step of the level-1 product (U^T x and E^T x upward, the near and coupling blocks
read in both triangles, E y and U y downward) runs as 64 x 64 blocks times 64 x 128
panels through tcgen05 with split-TF32 operands. Checks, column by column:

* against the oracle's product on sampled columns, and against the float64 product on
  every column, with an error of the order of the FP32 copy's own (the split loses less
  than 2^-20 per product; tests/test_split_tf32.py);
* panels of 1, 16, 64, 128 and 130 columns (a ragged second pass), host and device
  buffers, zero columns, and a matrix without far field (the leaf step has no entries);
* the skeleton bases of the 2^20-point Gaussian's density;
* rejections: no FP32 copy, blocks other than 64.
"""
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


def colerr(y, ref):
    return np.linalg.norm(y - ref, axis=0) / np.linalg.norm(ref, axis=0)


@pytest.fixture(scope="module")
def cheb64():
    n = 20000
    X = W.uniform_points(n, 3, 11)
    A = pkg.H2Matrix(cuda(X), "gaussian", length=0.1, nugget=1e-3, leaf=64, q=4, eta=1.0, with_f32=True)
    h = H2Matrix(X, KernelSpec("gaussian", 0.1, 1e-3), 64, 4, 1.0)
    assert A.query("KD") == 64 and A.query("KC") == 64
    yield A, h, n
    A.close()


@pytest.mark.parametrize("nr", [1, 16, 64, 128, 130])
def test_panel_product_matches_float64_and_oracle(cheb64, nr):
    A, h, n = cheb64
    x = np.random.default_rng(nr).standard_normal((n, nr))
    xd = cuda(x)
    y64 = A.apply(xd).cpu().numpy().reshape(n, nr)
    ytc = A.apply(xd, precision="tf32x3").cpu().numpy().reshape(n, nr)
    yf = A.apply(xd, precision="mixed_f32").cpu().numpy().reshape(n, nr)
    etc, ef = colerr(ytc, y64), colerr(yf, y64)
    print(f"nr={nr}: tensor-core max rel err {etc.max():.2e}, FP32 CUDA-core {ef.max():.2e}")
    assert etc.max() < 1e-5, etc.max()
    assert etc.max() < 10 * ef.max() + 1e-7, (etc.max(), ef.max())
    for j in sorted({0, nr // 2, nr - 1}):
        yo = h.apply(x[:, j])
        assert np.linalg.norm(ytc[:, j] - yo) <= 1e-5 * np.linalg.norm(yo), j


def test_panel_host_buffers_zero_columns_and_ragged_pass(cheb64):
    A, h, n = cheb64
    x = np.random.default_rng(3).standard_normal((n, 130))
    x[:, 5] = 0.0
    x[:, 129] = 0.0
    y = A.apply(torch.from_numpy(x), precision="tf32x3").numpy()      # host in, host out
    yd = A.apply(cuda(x), precision="tf32x3").cpu().numpy()
    assert np.array_equal(y, yd)          # same launches, same order: identical bits
    assert not y[:, 5].any() and not y[:, 129].any()
    y64 = A.apply(cuda(x)).cpu().numpy()
    e = colerr(y[:, [0, 128]], y64[:, [0, 128]])
    assert e.max() < 1e-5, e


def test_panel_without_far_field():
    n = 3000
    X = W.uniform_points(n, 2, 4)
    A = pkg.H2Matrix(cuda(X), "exponential", length=0.2, nugget=1e-2, leaf=64, q=8, eta=0.0, with_f32=True)
    h = H2Matrix(X, KernelSpec("exponential", 0.2, 1e-2), 64, 8, 0.0)
    x = np.random.default_rng(9).standard_normal((n, 7))
    y = A.apply(cuda(x), precision="tf32x3").cpu().numpy()
    yo = np.stack([h.apply(x[:, j]) for j in range(7)], axis=1)
    assert colerr(y, yo).max() < 1e-5
    A.close()


def test_panel_skeleton_bases_at_the_bench_density():
    n = 16384
    X = W.uniform_points(n, 3, 2) * (n / 2.0 ** 20) ** (1 / 3)
    A = pkg.H2Matrix(cuda(X), "gaussian", length=0.05, nugget=1e-3, leaf=64, eta=1.0, basis="skeleton",
                     basis_tol=1e-9, with_f32=True)
    h = H2Matrix(X, KernelSpec("gaussian", 0.05, 1e-3), 64, 4, 1.0, basis="skeleton", tol=1e-9)
    x = np.random.default_rng(1).standard_normal((n, 128))
    xd = cuda(x)
    y64 = A.apply(xd).cpu().numpy()
    ytc = A.apply(xd, precision="tf32x3").cpu().numpy()
    yf = A.apply(xd, precision="mixed_f32").cpu().numpy()
    etc, ef = colerr(ytc, y64), colerr(yf, y64)
    print(f"skeleton, 128 columns: tensor-core max rel err {etc.max():.2e}, FP32 CUDA-core {ef.max():.2e}")
    assert etc.max() < 1e-5 and etc.max() < 10 * ef.max() + 1e-7, (etc.max(), ef.max())
    yo = h.apply(x[:, 77])
    assert np.linalg.norm(ytc[:, 77] - yo) <= 1e-5 * np.linalg.norm(yo)
    A.close()


def test_panel_rejections():
    X = W.uniform_points(4000, 3, 5)
    A = pkg.H2Matrix(cuda(X), "gaussian", length=0.1, nugget=1e-3, leaf=64, q=4)   # no FP32 copy
    with pytest.raises(pkg.H2MGError) as e:
        A.apply(cuda(np.ones(4000)), precision="tf32x3")
    assert e.value.name == "INVALID_ARG"
    A.close()
    B = pkg.H2Matrix(cuda(X), "gaussian", length=0.1, nugget=1e-3, leaf=64, q=3, with_f32=True)   # rank 27
    with pytest.raises(pkg.H2MGError) as e:
        B.apply(cuda(np.ones(4000)), precision="tf32x3")
    assert e.value.name == "UNSUPPORTED"
    # the other arithmetic of the same call still works
    y = B.apply(cuda(np.ones(4000)), precision="mixed_f32")
    assert torch.isfinite(y).all()
    B.close()
