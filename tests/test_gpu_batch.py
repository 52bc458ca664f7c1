"""Several right-hand sides through one product / one solve (columns grouped four at a
time in the library): every column must equal what the oracle gives for it alone.

* products: each column of A X against the oracle's A x_c at the matvec tolerance
  (1e-12 relative), for group sizes 1, 2, 3, 4 and 5 (a full group plus a ragged
  one), float64, double-float and the FP32 copy (float32 rounding bound), device and
  host buffers, column-major and row-major (n, nrhs) inputs;
* solves: every column converges to the float64 tolerance with a V-cycle count
  within 25% (at least +-2; two solves of the same system on either side differ by
  up to about that much, the V-cycle with CG smoothers being rounding-sensitive)
  of the oracle's single-column solve, and a zero column
  stops at cycle 0 with x = 0 while the rest of its group runs on.
"""
import ctypes

import numpy as np
import pytest

import workloads as W
from oracle import H2MG, H2Matrix, KernelSpec, SolveOpts, solve_fcg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2501_17656_gb300 as pkg  # noqa: E402

pkg.load_library(build_if_missing=True)


def colrel(G, R):
    return [float(np.linalg.norm(G[:, c] - R[:, c]) / np.linalg.norm(R[:, c])) for c in range(R.shape[1])]


@pytest.fixture(scope="module")
def w1():
    p = W.workload(1)
    A = pkg.H2Matrix(torch.from_numpy(p["points"]).cuda(), "exponential", length=0.1, nugget=1e-2, leaf=64, q=4,
                     with_f32=True)
    h = H2Matrix(p["points"], KernelSpec("exponential", 0.1, 1e-2), 64, 4, 1.0)
    yield p, A, h
    A.close()


@pytest.mark.parametrize("nrhs", [1, 2, 3, 4, 5])
def test_block_product_equals_columnwise_oracle(w1, nrhs):
    p, A, h = w1
    X = W.normal_rhs(p["n"], 7, nrhs) if nrhs > 1 else W.normal_rhs(p["n"], 7)[:, None]
    R = np.stack([h.apply(X[:, c]) for c in range(nrhs)], axis=1)
    Y = A.apply(torch.from_numpy(np.ascontiguousarray(X)).cuda()).cpu().numpy()
    assert max(colrel(Y, R)) < 1e-12
    # host buffers, column-major
    Yh = A.apply(np.asfortranarray(X))
    assert max(colrel(Yh, R)) < 1e-12


def test_block_product_double_float_and_fp32_copy():
    X0 = W.uniform_points(8192, 3, 2)
    h = H2Matrix(X0, KernelSpec("gaussian", 0.05, 1e-3), 64, 4, 1.0)
    V = W.normal_rhs(8192, 8, 5)
    R = np.stack([h.apply(V[:, c]) for c in range(5)], axis=1)
    A = pkg.H2Matrix(torch.from_numpy(X0).cuda(), "gaussian", length=0.05, nugget=1e-3, leaf=64, q=4,
                     storage="df64", with_f32=True)
    Y = A.apply(torch.from_numpy(np.ascontiguousarray(V)).cuda()).cpu().numpy()
    assert max(colrel(Y, R)) < 1e-12
    # the FP32 copy column by column (its four-column groups run inside the
    # mixed-precision solve below): float32 rounding of a float64 product
    Vt = torch.from_numpy(np.ascontiguousarray(V)).cuda()
    singles = np.stack([A.apply_level(1, Vt[:, c].contiguous(), precision="mixed_f32").cpu().numpy()
                        for c in range(5)], axis=1)
    assert max(colrel(singles, R)) < 1e-5
    A.close()


def test_batched_solve_each_column_converges_like_oracle(w1):
    """Flexible-CG outer loop (the V-cycle with CG smoothers is nonlinear, and the plain
    repeated V-cycle's non-monotone residual makes cycle counts rounding-sensitive)."""
    p, A, h = w1
    mg = H2MG(h)
    tol = 1e-8
    B = W.normal_rhs(p["n"], 11, 5)
    Xg, infos = A.solve(torch.from_numpy(np.ascontiguousarray(B)).cuda(), tol=tol, max_cycles=300, outer="fcg")
    assert len(infos) == 5 and all(i.converged for i in infos)
    Xg = Xg.cpu().numpy()
    for c in range(5):
        r = B[:, c] - h.apply(Xg[:, c])
        assert np.linalg.norm(r) / np.linalg.norm(B[:, c]) <= tol * 1.0001, c
        assert abs(infos[c].relres - np.linalg.norm(r) / np.linalg.norm(B[:, c])) <= 1e-3 * tol
        _, io = solve_fcg(mg, B[:, c], SolveOpts(tol=tol, max_cycles=300))
        assert io.converged
        assert abs(infos[c].cycles - io.cycles) <= max(2, 0.25 * io.cycles), (c, infos[c].cycles, io.cycles)


@pytest.mark.parametrize("outer", ["vcycle", "fcg"])
def test_batched_solve_zero_column_and_host_buffers(w1, outer):
    p, A, h = w1
    tol = 1e-9
    B = W.normal_rhs(p["n"], 12, 3)
    B[:, 1] = 0.0
    X = np.zeros((p["n"], 3), order="F")
    X, infos = A.solve(B, x=X, tol=tol, max_cycles=300, outer=outer)
    assert all(i.converged for i in infos)
    assert infos[1].cycles == 0 and infos[1].relres == 0.0
    assert np.all(X[:, 1] == 0.0)
    for c in (0, 2):
        r = B[:, c] - h.apply(X[:, c])
        assert np.linalg.norm(r) / np.linalg.norm(B[:, c]) <= tol * 1.0001


def test_batched_mixed_precision_solve_five_columns():
    X0 = W.uniform_points(8192, 3, 2)
    h = H2Matrix(X0, KernelSpec("gaussian", 0.05, 1e-3), 64, 4, 1.0)
    A = pkg.H2Matrix(torch.from_numpy(X0).cuda(), "gaussian", length=0.05, nugget=1e-3, leaf=64, q=4,
                     with_f32=True)
    B = W.normal_rhs(8192, 13, 5)
    Xg, infos = A.solve(torch.from_numpy(np.ascontiguousarray(B)).cuda(), tol=1e-10, max_cycles=100,
                        precision="mixed_f32", outer="fcg")
    assert all(i.converged for i in infos)
    Xg = Xg.cpu().numpy()
    for c in range(5):
        r = B[:, c] - h.apply(Xg[:, c])
        assert np.linalg.norm(r) / np.linalg.norm(B[:, c]) <= 1e-10 * 1.0001, c
    A.close()


def test_batched_calls_reject_bad_leading_dimension(w1):
    p, A, _ = w1
    lib = pkg.load_library()
    b = torch.zeros(2 * p["n"], dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    o = A._opts()
    info = pkg.SolveInfo()
    st = lib.h2mg_solve(A._h, b.data_ptr(), x.data_ptr(), 2, p["n"] - 1, ctypes.byref(o), ctypes.byref(info), 0)
    assert pkg.STATUS[st] == "INVALID_ARG"
    st = lib.h2mg_apply(A._h, b.data_ptr(), x.data_ptr(), 0, p["n"], 0)
    assert pkg.STATUS[st] == "INVALID_ARG"


@pytest.mark.parametrize("nrhs", [1, 3])
def test_graph_replayed_vcycle_matches_direct_launches(w1, nrhs):
    """The V-cycle captured as a CUDA graph and replayed: same convergence as direct
    launches and the launch counter advances by the graph's kernels; while profiling
    is on, the replayed graph carries event nodes and the profile sees every block
    product of the replays."""
    p, A, h = w1
    tol = 1e-9
    B = W.normal_rhs(p["n"], 14, nrhs) if nrhs > 1 else W.normal_rhs(p["n"], 14)
    Bt = torch.from_numpy(np.ascontiguousarray(B)).cuda()
    kw = dict(tol=tol, max_cycles=300, outer="fcg", precision="mixed_f32")
    Xd, idd = A.solve(Bt, **kw)
    l0 = pkg.H2Matrix.launch_count()
    Xg, ig = A.solve(Bt, use_graph=True, **kw)          # first: capture + replays
    l1 = pkg.H2Matrix.launch_count()
    A.profile(1)
    Xg2, ig2 = A.solve(Bt, use_graph=True, **kw)        # profiled graph (event nodes)
    l2 = pkg.H2Matrix.launch_count()
    nk, kms, kby = A.profile(0)
    idd, ig, ig2 = ([i] if nrhs == 1 else i for i in (idd, ig, ig2))
    Bm = B.reshape(p["n"], nrhs)
    for X, infos in ((Xd, idd), (Xg, ig), (Xg2, ig2)):
        Xn = X.cpu().numpy().reshape(p["n"], nrhs)
        for c in range(nrhs):
            assert infos[c].converged
            r = Bm[:, c] - h.apply(Xn[:, c])
            assert np.linalg.norm(r) / np.linalg.norm(Bm[:, c]) <= tol * 1.0001
    # mixed precision: the oracle's own count for these columns spans 95..109 cycles
    # under 1e-15 relative perturbations of b, so the band is 25%
    for c in range(nrhs):
        assert abs(ig[c].cycles - idd[c].cycles) <= max(2, 0.25 * idd[c].cycles)
    assert l1 - l0 > 0 and l2 - l1 > 0
    # every V-cycle runs at least one block product per level and smoother step; the
    # profiled replays see the same products per outer iteration as direct launches
    assert nk >= max(i.cycles for i in ig2) and kms > 0 and kby > 0
    A.profile(1)
    _, idd2 = A.solve(Bt, use_graph=False, **kw)
    nd, _, _ = A.profile(0)
    idd2 = [idd2] if nrhs == 1 else idd2
    cyc_g, cyc_d = max(i.cycles for i in ig2), max(i.cycles for i in idd2)
    assert abs(nk / max(cyc_g, 1) - nd / max(cyc_d, 1)) <= 0.05 * nd / max(cyc_d, 1)


@pytest.fixture(scope="module")
def uneven():
    """Independent problems of uneven size and kind: three perturbed spheres with the
    single-layer kernel (sizes from the surface workload's list) and the 4096-point
    exponential point cloud."""
    from oracle import surface_diag
    ms = sorted(set(W.surface_problem_sizes()))[:3]
    probs = []
    for j, m in enumerate(ms):
        c, a, _ = W.perturbed_icosphere(m, j)
        A = pkg.H2Matrix(torch.from_numpy(c).cuda(), "laplace_sl", weights=torch.from_numpy(a).cuda(), leaf=64, q=4,
                         with_f32=True)
        h = H2Matrix(c, KernelSpec("laplace_sl", 1.0, 0.0, 2, a, surface_diag(a)), 64, 4, 1.0)
        probs.append((A, h, W.normal_rhs(c.shape[0], 3 + j)))
    p = W.workload(1)
    A = pkg.H2Matrix(torch.from_numpy(p["points"]).cuda(), "exponential", length=0.1, nugget=1e-2, leaf=64, q=4,
                     with_f32=True)
    h = H2Matrix(p["points"], KernelSpec("exponential", 0.1, 1e-2), 64, 4, 1.0)
    probs.append((A, h, p["b"]))
    yield probs
    for A, _, _ in probs:
        A.close()


@pytest.mark.parametrize("use_graph", [False, True])
def test_independent_problems_solved_together_like_oracle(uneven, use_graph):
    tol = 1e-9
    mats = [A for A, _, _ in uneven]
    bs = [torch.from_numpy(b).cuda() for _, _, b in uneven]
    xs, infos = pkg.solve_batched(mats, bs, tol=tol, max_cycles=300, outer="fcg", use_graph=use_graph)
    assert len(infos) == len(uneven)
    for (A, h, b), x, info in zip(uneven, xs, infos):
        assert info.converged
        r = b - h.apply(x.cpu().numpy())
        assert np.linalg.norm(r) / np.linalg.norm(b) <= tol * 1.0001
        _, io = solve_fcg(H2MG(h), b, SolveOpts(tol=tol, max_cycles=300))
        assert abs(info.cycles - io.cycles) <= max(2, 0.25 * io.cycles), (info.cycles, io.cycles)
        # the same problem alone on the GPU
        _, i1 = A.solve(torch.from_numpy(b).cuda(), tol=tol, max_cycles=300, outer="fcg")
        assert abs(info.cycles - i1.cycles) <= max(2, 0.25 * i1.cycles)


def test_independent_problems_mixed_precision_host_buffers(uneven):
    mats = [A for A, _, _ in uneven]
    bs = [b.copy() for _, _, b in uneven]
    xs, infos = pkg.solve_batched(mats, bs, tol=1e-10, max_cycles=300, outer="fcg", precision="mixed_f32",
                                  use_graph=True)
    for (A, h, b), x, info in zip(uneven, xs, infos):
        assert isinstance(x, np.ndarray) and info.converged
        assert np.linalg.norm(b - h.apply(x)) / np.linalg.norm(b) <= 1e-10 * 1.0001


def test_independent_problems_reject_duplicates_and_report_per_problem(uneven):
    A0 = uneven[0][0]
    b0 = torch.from_numpy(uneven[0][2]).cuda()
    with pytest.raises(pkg.H2MGError) as e:
        pkg.solve_batched([A0, A0], [b0, b0.clone()])
    assert e.value.name == "INVALID_ARG"
    # a problem that cannot converge in one cycle is reported per problem
    mats = [A for A, _, _ in uneven]
    bs = [torch.from_numpy(b).cuda() for _, _, b in uneven]
    xs, infos = pkg.solve_batched(mats, bs, tol=1e-17, max_cycles=1, raise_on_fail=False, outer="fcg")
    assert all(i.cycles == 1 and not i.converged for i in infos)
