"""h2mg_apply_noalloc: the H2 matrix-vector product for callers that cannot
allocate device memory (allocator callbacks, memory reserved in full by another
allocator).

Its output must match h2mg_apply's within the matvec tolerance used elsewhere
(1e-12 relative) on two calls in a row (the fixed scratch array keeps the first
call's contents), the second call must not change the device's free memory, and a
matrix whose product needs more than the fixed array is rejected with UNSUPPORTED.
This file is collected last so that a run stopping at the first failure has
already run every other test.
"""
import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2501_17656_gb300 as pkg  # noqa: E402

pkg.load_library(build_if_missing=True)


def test_noalloc_matches_apply_on_two_calls():
    p = W.workload(1)
    A = pkg.H2Matrix(torch.from_numpy(p["points"]).cuda(), "exponential", length=0.1, nugget=1e-2,
                     leaf=64, q=4, eta=1.0)
    g = torch.Generator(device="cuda").manual_seed(3)
    x1 = torch.randn(p["n"], dtype=torch.float64, device="cuda", generator=g)
    x2 = torch.randn(p["n"], dtype=torch.float64, device="cuda", generator=g)
    y1, y2 = torch.empty_like(x1), torch.empty_like(x2)
    ref1, ref2 = A.apply(x1), A.apply(x2)
    A.apply_noalloc(x1, y1)                 # first call: looks up the array's address
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    A.apply_noalloc(x2, y2)                 # second call reuses the same array
    torch.cuda.synchronize()
    free_after = torch.cuda.mem_get_info()[0]
    assert free_after == free_before
    for y, ref in ((y1, ref1), (y2, ref2)):
        err = float((y - ref).norm() / ref.norm())
        assert err < 1e-12, err
    # and the first result is still the product of x1 when recomputed after x2
    A.apply_noalloc(x1, y2)
    assert float((y2 - ref1).norm() / ref1.norm()) < 1e-12
    A.close()


def test_noalloc_rejects_host_vectors_and_oversized_problems():
    p = W.workload(1, n=2048)
    A = pkg.H2Matrix(torch.from_numpy(p["points"]).cuda(), "exponential", length=0.1, nugget=1e-2,
                     leaf=64, q=4, eta=1.0)
    xh = np.ones(2048)
    with pytest.raises(pkg.H2MGError) as e:
        A.apply_noalloc(xh, np.empty_like(xh))
    assert e.value.name == "INVALID_ARG"
    A.close()
    # 2-D, 3 x 3 nodes (KC = 16), leaf 32 at 2^19 points: 2^14 leaves and about 2^15
    # clusters, so three 4 MiB coefficient buffers and two 4 MiB point buffers,
    # about 20 MiB in all: above the fixed 16 MiB
    n = 1 << 19
    X = torch.from_numpy(W.uniform_points(n, 2, 2)).cuda()
    B = pkg.H2Matrix(X, "exponential", length=0.1, nugget=1e-2, leaf=32, q=3, eta=1.0)
    x = torch.ones(n, dtype=torch.float64, device="cuda")
    with pytest.raises(pkg.H2MGError) as e:
        B.apply_noalloc(x, torch.empty_like(x))
    assert e.value.name == "UNSUPPORTED"
    assert "bytes of scratch" in str(e.value)
    B.close()


def test_noalloc_rejects_wrong_lengths_before_the_library():
    """The library cannot see buffer sizes: a short x or y would be read or written
    past its end on the device, so the binding rejects them first."""
    p = W.workload(1, n=2048)
    A = pkg.H2Matrix(torch.from_numpy(p["points"]).cuda(), "exponential", length=0.1, nugget=1e-2,
                     leaf=64, q=4, eta=1.0)
    x = torch.ones(2048, dtype=torch.float64, device="cuda")
    for xx, yy in ((x[:2047], torch.empty_like(x)), (x, torch.empty(2047, dtype=torch.float64, device="cuda")),
                   (x, torch.empty((2048, 2), dtype=torch.float64, device="cuda"))):
        with pytest.raises(ValueError):
            A.apply_noalloc(xx, yy)
        with pytest.raises(ValueError):
            A.apply(xx, yy)
    y = torch.empty_like(x)
    A.apply_noalloc(x, y)           # a well-formed call still works afterwards
    ref = A.apply(x)
    assert float((y - ref).norm() / ref.norm()) < 1e-12
    A.close()
