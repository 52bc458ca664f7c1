"""CPU oracle for the H2-MG solver: a plain, slow, float64 NumPy/SciPy restatement
of the paper (Sections 3.1-3.4).

This package is TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / reference leg of ``bench.py`` may import it. It shares
no code with the CUDA library under ``paper_2501_17656_gb300/`` and never imports
it. Its inputs come from ``workloads`` only.
"""
from .kernels import dense_kernel_matrix, kmat, surface_diag  # noqa: F401
from .h2 import ClusterTree, H2Matrix, KernelSpec, block_partition  # noqa: F401
from .mg import H2MG, SolveInfo, SolveOpts, cg, cycle, solve, solve_cg, solve_fcg, solve_mixed, vcycle  # noqa: F401
