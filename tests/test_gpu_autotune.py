"""The block-product autotuner: it reports a timing per operator and column group,
never picks a slower split than the fixed rule, and leaves every product and a
V-cycle equal to the oracle's (a launch shape changes only the order of the atomic
sums)."""
import numpy as np
import pytest

import workloads as W
from oracle import H2MG, H2Matrix, KernelSpec

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2501_17656_gb300 as pkg  # noqa: E402

pkg.load_library(build_if_missing=True)


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def test_autotune_reports_and_keeps_products_exact():
    X = W.uniform_points(16384, 3, 2)
    # a nugget well above the 3x3x3-node interpolation error keeps every level positive definite
    A = pkg.H2Matrix(torch.from_numpy(X).cuda(), "gaussian", length=0.2, nugget=1e-1, leaf=64, q=3, eta=1.0,
                     with_f32=True)
    h = H2Matrix(X, KernelSpec("gaussian", 0.2, 1e-1), 64, 3, 1.0)
    rep = A.autotune()
    # every operator (close part, then the coupling operator of each level), two
    # primary-format column groups and three FP32 ones
    assert len(rep) == 5 * (A.levels + 1)
    ops = {r[0] for r in rep}
    assert 0 in ops and 1 in ops
    for op, nr, fixed, tuned in rep:
        assert nr in (1, 2, 4) and fixed > 0 and tuned > 0
        assert tuned <= fixed * 1.0001
    x = np.random.default_rng(1).standard_normal(16384)
    assert rel(A.apply(torch.from_numpy(x).cuda()).cpu().numpy(), h.apply(x)) < 1e-12
    mg = H2MG(h)
    KC = A.query("KC")
    for i in range(2, mg.l + 1):
        v = np.random.default_rng(i).standard_normal(mg.size(i))
        off = h.coef_offsets(mg.m(i))
        vp = np.zeros((1 << mg.m(i)) * KC)
        for j in range(1 << mg.m(i)):
            vp[j * KC: j * KC + off[j + 1] - off[j]] = v[off[j]:off[j + 1]]
        y = A.apply_level(i, torch.from_numpy(vp).cuda()).cpu().numpy()
        yu = np.concatenate([y[j * KC: j * KC + off[j + 1] - off[j]] for j in range(1 << mg.m(i))])
        assert rel(yu, mg.apply(i, v)) < 1e-12
        y32 = A.apply_level(i, torch.from_numpy(vp).cuda(), "mixed_f32").cpu().numpy()
        yu32 = np.concatenate([y32[j * KC: j * KC + off[j + 1] - off[j]] for j in range(1 << mg.m(i))])
        assert rel(yu32, mg.apply(i, v)) < 1e-5
    # a V-cycle with short smoothers through the tuned launches equals the oracle's
    from oracle import SolveOpts
    from oracle.mg import vcycle
    if mg.chol is not None:
        bv = np.random.default_rng(9).standard_normal(16384)
        xg = A.vcycle(torch.zeros(16384, dtype=torch.float64, device="cuda"), torch.from_numpy(bv).cuda(),
                      n_f=1, n_c=2).cpu().numpy()
        xo = vcycle(mg, np.zeros(16384), bv, SolveOpts(n_f=1, n_c=2))
        assert rel(xg, xo) < 1e-9
    A.close()
