"""GB300 H2-MG: Python binding of the C library ``libh2mg.so`` (include/h2mg.h).

This module only marshals arguments: every step of the build, the matrix-vector
product and the H2-MG solve runs in the library's CUDA kernels. It fails loudly if
the library is missing; there is no CPU fallback.

Vectors may be torch tensors (CUDA or CPU), or NumPy arrays; the library reads
device pointers in place and stages host pointers itself. Work goes to the current
torch CUDA stream when torch has CUDA, else to the default stream.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

__all__ = ["H2Matrix", "KERNELS", "SolveInfo", "H2MGError", "load_library", "library_path", "dot",
           "MaternLoss"]

_HERE = os.path.dirname(os.path.abspath(__file__))
library_path = os.path.join(_HERE, "libh2mg.so")

KERNELS = {"gaussian": 0, "exponential": 1, "matern32": 2, "laplace_sl": 3, "poly": 4,
           "dmatern32_dl": 5}
STORAGE = {"f64": 0, "df64": 1}
PRECISION = {"f64": 0, "mixed_f32": 1, "f64_dd": 2, "tf32x3": 3}
OUTER = {"vcycle": 0, "fcg": 1, "cg": 2}
CYCLE = {"V": 0, "W": 1, "F": 2}
STATUS = {0: "OK", 1: "INVALID_ARG", 2: "OOM", 3: "CUDA", 4: "NOT_SPD", 5: "NOT_CONVERGED",
          6: "NAN", 7: "TIMEOUT", 8: "UNSUPPORTED"}

Q = dict(N=0, DIM=1, L=2, TSTAR=3, LEVELS=4, KD=5, KC=6, RANK=7, NEAR_PAIRS=8, FAR_PAIRS=9,
         LEVEL_SIZE=10, BYTES_PRIMARY=11, BYTES_F32=12, APPLY_BYTES=13, DEVICE_BYTES=14,
         PRODUCT_BYTES_F32=15, PANEL_ENTRIES=16)
X = dict(PERM=0, LEAF_OFFSETS=1, NEAR=2, FAR=3, RANKS=4, BOXES=5, SKELETON=6)
BASIS = {"chebyshev": 0, "skeleton": 1}

EXPORTED = ["h2mg_build", "h2mg_apply", "h2mg_solve", "h2mg_destroy", "h2mg_error_string",
            "h2mg_last_error", "h2mg_query", "h2mg_export", "h2mg_apply_level",
            "h2mg_coarse_solve", "h2mg_smooth", "h2mg_vcycle", "h2mg_launch_count", "h2mg_profile",
            "h2mg_transfer", "h2mg_apply_noalloc", "h2mg_build_sibling", "h2mg_dot", "h2mg_solve_batched",
            "h2mg_autotune", "h2mg_matern_loss_grad", "h2mg_apply_ex"]


class H2MGError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status
        self.name = STATUS.get(status, str(status))


class _Kernel(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("length", ctypes.c_double), ("nugget", ctypes.c_double),
                ("degree", ctypes.c_int), ("weights", ctypes.c_void_p), ("diag", ctypes.c_void_p)]


class _BuildOpts(ctypes.Structure):
    _fields_ = [("leaf_size", ctypes.c_int), ("cheb_q", ctypes.c_int), ("eta", ctypes.c_double),
                ("storage", ctypes.c_int), ("with_f32", ctypes.c_int), ("coarse_level", ctypes.c_int),
                ("basis", ctypes.c_int), ("basis_tol", ctypes.c_double), ("rank_max", ctypes.c_int)]


class _SolveOpts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_cycles", ctypes.c_int), ("n_f", ctypes.c_int),
                ("n_c", ctypes.c_int), ("precision", ctypes.c_int),
                ("explicit_restrict_residual", ctypes.c_int), ("outer", ctypes.c_int),
                ("use_graph", ctypes.c_int), ("skip_square_levels", ctypes.c_int), ("cycle", ctypes.c_int),
                ("residual_dd", ctypes.c_int)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("cycles", ctypes.c_int), ("converged", ctypes.c_int), ("relres", ctypes.c_double),
                ("relres_hist", ctypes.c_double * 256), ("ms_solve", ctypes.c_double)]

    def history(self):
        return [self.relres_hist[i] for i in range(min(self.cycles + 1, 256))]


_lib = None


def load_library(build_if_missing: bool = False):
    """Load libh2mg.so (optionally building it first). Raises if it cannot be loaded."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(library_path):
        if not build_if_missing:
            raise RuntimeError(f"{library_path} is missing: build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        from . import _build
        _build.build()
    lib = ctypes.CDLL(library_path)
    vp, i64, ci, cd = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
    lib.h2mg_build.argtypes = [vp, i64, ci, ctypes.POINTER(_Kernel), ctypes.POINTER(_BuildOpts), vp,
                               ctypes.POINTER(vp)]
    lib.h2mg_apply.argtypes = [vp, vp, vp, ci, i64, vp]
    lib.h2mg_apply_ex.argtypes = [vp, ci, vp, vp, ci, i64, vp]
    lib.h2mg_solve.argtypes = [vp, vp, vp, ci, i64, ctypes.POINTER(_SolveOpts), ctypes.POINTER(SolveInfo), vp]
    lib.h2mg_destroy.argtypes = [vp]
    lib.h2mg_error_string.argtypes = [ci]
    lib.h2mg_error_string.restype = ctypes.c_char_p
    lib.h2mg_last_error.argtypes = []
    lib.h2mg_last_error.restype = ctypes.c_char_p
    lib.h2mg_query.argtypes = [vp, ci, ci, ctypes.POINTER(i64)]
    lib.h2mg_export.argtypes = [vp, ci, ci, vp, i64, ctypes.POINTER(i64)]
    lib.h2mg_apply_level.argtypes = [vp, ci, ci, vp, vp, vp]
    lib.h2mg_coarse_solve.argtypes = [vp, vp, vp, vp]
    lib.h2mg_smooth.argtypes = [vp, ci, ci, vp, vp, ci, vp, vp, vp]
    lib.h2mg_vcycle.argtypes = [vp, vp, vp, vp, ctypes.POINTER(_SolveOpts), vp]
    lib.h2mg_launch_count.argtypes = []
    lib.h2mg_transfer.argtypes = [vp, ci, ci, vp, vp, vp]
    lib.h2mg_apply_noalloc.argtypes = [vp, vp, vp, vp]
    lib.h2mg_build_sibling.argtypes = [vp, ctypes.POINTER(_Kernel), vp, ctypes.POINTER(vp)]
    lib.h2mg_dot.argtypes = [vp, vp, i64, ctypes.POINTER(cd), vp]
    lib.h2mg_solve_batched.argtypes = [ci, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp),
                                       ctypes.POINTER(_SolveOpts), ctypes.POINTER(SolveInfo), vp]
    lib.h2mg_profile.argtypes = [vp, ci, ctypes.POINTER(i64), ctypes.POINTER(cd), ctypes.POINTER(cd)]
    lib.h2mg_autotune.argtypes = [vp, vp, ctypes.POINTER(cd), ci, ctypes.POINTER(ci)]
    pd = ctypes.POINTER(cd)
    lib.h2mg_matern_loss_grad.argtypes = [vp, vp, vp, vp, ctypes.POINTER(_SolveOpts), pd, vp, vp, pd, pd,
                                          ctypes.POINTER(SolveInfo), vp]
    for name in EXPORTED:
        if name not in ("h2mg_error_string", "h2mg_last_error", "h2mg_launch_count"):
            getattr(lib, name).restype = ci
    lib.h2mg_launch_count.restype = i64
    _lib = lib
    return lib


def _check(status: int):
    if status != 0:
        msg = _lib.h2mg_last_error().decode() or _lib.h2mg_error_string(status).decode()
        raise H2MGError(status, msg)


def _current_device():
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_device()
    except ImportError:
        pass
    return None


def _stream():
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except ImportError:
        pass
    return 0


def _ptr(a):
    """Data pointer of a torch tensor or NumPy array (float64, contiguous)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not (a.flags.c_contiguous or a.flags.f_contiguous):
            raise TypeError("arrays must be contiguous float64")
        return a.ctypes.data
    import torch
    if isinstance(a, torch.Tensor):
        if a.dtype != torch.float64 or not a.is_contiguous():
            raise TypeError("tensors must be contiguous float64")
        return a.data_ptr()
    raise TypeError(f"unsupported buffer type {type(a)}")


def _expect(a, n, what, cols=False, dev=None):
    """Rejects a vector (or, with ``cols``, an (n, nrhs) block) whose first dimension is
    not ``n``, or a CUDA tensor on another device than the current one: the library
    cannot see buffer sizes, so a short buffer would be read or written past its end."""
    if a is None:
        return
    shape = tuple(a.shape)
    if len(shape) == 0 or shape[0] != n or (len(shape) > (2 if cols else 1)):
        raise ValueError(f"{what} must have shape ({n},){' or (' + str(n) + ', nrhs)' if cols else ''}, "
                         f"got {shape}")
    if not isinstance(a, np.ndarray):
        import torch
        if isinstance(a, torch.Tensor) and a.is_cuda:
            cur = torch.cuda.current_device()
            if a.device.index != cur or (dev is not None and dev != cur):
                raise ValueError(f"{what} is on {a.device} and the matrix on cuda:{dev}, "
                                 f"but cuda:{cur} is current")


def _like(x, n):
    """A new float64 buffer on the same device/kind as x."""
    if isinstance(x, np.ndarray):
        return np.zeros(n, dtype=np.float64)
    import torch
    return torch.zeros(n, dtype=torch.float64, device=x.device)


def _colmajor(a):
    """(buffer, nrhs): a 1-D vector, or a 2-D (n, nrhs) array / tensor as a
    column-major buffer (the library's layout: column c at offset c * n). The buffer is
    ``a``'s own memory when ``a`` is already column-major, else a packed copy."""
    if len(a.shape) == 1:
        return a, 1
    if isinstance(a, np.ndarray):
        return np.asfortranarray(a), int(a.shape[1])
    t = a.t()
    return (t if t.is_contiguous() else t.contiguous()), int(a.shape[1])


def _new_cols(like, n, nrhs):
    """A zeroed column-major (n, nrhs) buffer beside ``like`` (1-D when nrhs is None)."""
    if nrhs is None:
        return _like(like, n)
    if isinstance(like, np.ndarray):
        return np.zeros((n, nrhs), dtype=np.float64, order="F")
    import torch
    return torch.zeros((nrhs, n), dtype=torch.float64, device=like.device).t()


def _copy_back(dst, buf):
    """Write a packed column-major result into ``dst`` when ``buf`` is not its memory."""
    if len(dst.shape) == 1:
        return
    if isinstance(dst, np.ndarray):
        if buf is not dst:
            dst[...] = buf
    elif buf.data_ptr() != dst.data_ptr():
        dst.copy_(buf.t())


def dot(x, y) -> float:
    """x^T y (float64) reduced by the library on the GPU."""
    out = ctypes.c_double()
    n = int(x.shape[0])
    _expect(x, n, "x")
    _expect(y, n, "y")
    _check(load_library().h2mg_dot(_ptr(x), _ptr(y), n, ctypes.byref(out), _stream()))
    return float(out.value)


class H2Matrix:
    """An H2 matrix built on the GPU from points and a kernel (Sec. 3.1 of the paper),
    with its H2-MG multigrid hierarchy (Sec. 3.3)."""

    def __init__(self, points, kernel: str = "gaussian", length: float = 1.0, nugget: float = 0.0,
                 degree: int = 2, weights=None, diag=None, leaf: int = 64, q: int = 4,
                 eta: float = 1.0, storage: str = "f64", with_f32: bool = False,
                 coarse_level: int = -1, basis: str = "chebyshev", basis_tol: float = 1e-9,
                 rank_max: int = 64):
        lib = load_library()
        self._lib = lib
        pts = points
        if isinstance(pts, np.ndarray):
            pts = np.ascontiguousarray(pts, dtype=np.float64)
        n, dim = int(pts.shape[0]), int(pts.shape[1]) if len(pts.shape) > 1 else 1
        self._keep = [pts, weights, diag]
        k = _Kernel(KERNELS[kernel], float(length), float(nugget), int(degree), _ptr(weights), _ptr(diag))
        o = _BuildOpts(int(leaf), int(q), float(eta), STORAGE[storage], int(bool(with_f32)), int(coarse_level),
                       BASIS[basis], float(basis_tol), int(rank_max))
        h = ctypes.c_void_p()
        _check(lib.h2mg_build(_ptr(pts), n, dim, ctypes.byref(k), ctypes.byref(o), _stream(), ctypes.byref(h)))
        self._h = h
        self.n, self.dim = n, dim
        self.device = _current_device()
        self._keep = None

    # ----------------------------------------------------------------- siblings
    def sibling(self, kernel: str, length: float = 1.0, nugget: float = 0.0, degree: int = 2) -> "H2Matrix":
        """The H2 matrix of another kernel on this matrix's tree and partition (products
        only), with its nodes and bases when they are Chebyshev, with skeletons of its own
        kernel when they are skeletons; e.g. ``sibling("dmatern32_dl", length)`` = dA/dlength."""
        k = _Kernel(KERNELS[kernel], float(length), float(nugget), int(degree), None, None)
        h = ctypes.c_void_p()
        _check(self._lib.h2mg_build_sibling(self._h, ctypes.byref(k), _stream(), ctypes.byref(h)))
        out = H2Matrix.__new__(H2Matrix)
        out._lib, out._h, out.n, out.dim, out._keep = self._lib, h, self.n, self.dim, None
        out.device = self.device
        out._base = self          # the sibling uses this matrix's device structures
        return out

    # ----------------------------------------------------------------- lifetime
    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.h2mg_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ----------------------------------------------------------------- queries
    def query(self, what: str, arg: int = 0) -> int:
        v = ctypes.c_int64()
        _check(self._lib.h2mg_query(self._h, Q[what], int(arg), ctypes.byref(v)))
        return int(v.value)

    def export(self, what: str, arg: int = 0) -> np.ndarray:
        nb = ctypes.c_int64()
        _check(self._lib.h2mg_export(self._h, X[what], int(arg), None, 0, ctypes.byref(nb)))
        dtype = np.float64 if what == "BOXES" else np.int32
        buf = np.zeros(max(int(nb.value) // np.dtype(dtype).itemsize, 1), dtype=dtype)
        _check(self._lib.h2mg_export(self._h, X[what], int(arg), buf.ctypes.data, buf.nbytes, ctypes.byref(nb)))
        return buf[: int(nb.value) // np.dtype(dtype).itemsize]

    def profile(self, enable: int):
        """Start (1) / stop (0) timing of the block-product launches; returns
        (launches, ms, bytes) recorded so far."""
        n, ms, by = ctypes.c_int64(), ctypes.c_double(), ctypes.c_double()
        _check(self._lib.h2mg_profile(self._h, int(enable), ctypes.byref(n), ctypes.byref(ms), ctypes.byref(by)))
        return int(n.value), float(ms.value), float(by.value)

    def autotune(self):
        """Tune the block product's CTAs per block row on trial launches (h2mg_autotune).
        Returns a list of (operator, columns, fixed-rule ms, tuned ms)."""
        cap = 256
        buf = (ctypes.c_double * (4 * cap))()
        cnt = ctypes.c_int()
        _check(self._lib.h2mg_autotune(self._h, _stream(), buf, cap, ctypes.byref(cnt)))
        return [(int(buf[4 * k]), int(buf[4 * k + 1]), buf[4 * k + 2], buf[4 * k + 3])
                for k in range(min(cnt.value, cap))]

    @staticmethod
    def launch_count() -> int:
        return int(load_library().h2mg_launch_count())

    @property
    def levels(self) -> int:
        return self.query("LEVELS")

    def level_size(self, i: int) -> int:
        return self.query("LEVEL_SIZE", i)

    # ----------------------------------------------------------------- products
    def apply(self, x, y=None, precision: str | None = None):
        """y = A x for a vector or an (n, nrhs) block of columns. Default: the primary
        storage, the columns through the products in groups of four. ``precision``
        "f64", "mixed_f32" (the FP32 copy on the CUDA cores) or "tf32x3" (the FP32 copy
        on the tensor cores, 128 columns per block read; see h2mg_apply_ex)."""
        _expect(x, self.n, "x", cols=True, dev=self.device)
        xb, nrhs = _colmajor(x)
        out = y if y is not None else _new_cols(x, self.n, None if len(x.shape) == 1 else nrhs)
        _expect(out, self.n, "y", cols=True, dev=self.device)
        if tuple(out.shape) != tuple(x.shape):
            raise ValueError(f"y must have the shape of x {tuple(x.shape)}, got {tuple(out.shape)}")
        yb, _ = _colmajor(out)
        if precision is None:
            _check(self._lib.h2mg_apply(self._h, _ptr(xb), _ptr(yb), nrhs, self.n, _stream()))
        else:
            _check(self._lib.h2mg_apply_ex(self._h, PRECISION[precision], _ptr(xb), _ptr(yb), nrhs, self.n,
                                           _stream()))
        _copy_back(out, yb)
        return out

    def apply_noalloc(self, x, y):
        """y = A x without any device allocation (device tensors only; scratch in a
        fixed array shared by all calls -- see h2mg_apply_noalloc)."""
        _expect(x, self.n, "x", dev=self.device)
        _expect(y, self.n, "y", dev=self.device)
        _check(self._lib.h2mg_apply_noalloc(self._h, _ptr(x), _ptr(y), _stream()))
        return y

    def apply_level(self, i: int, x, precision: str = "f64", y=None):
        n = self.level_size(i)
        _expect(x, n, "x", dev=self.device)
        if y is None:
            y = _like(x, n)
        _expect(y, n, "y", dev=self.device)
        _check(self._lib.h2mg_apply_level(self._h, int(i), PRECISION[precision], _ptr(x), _ptr(y), _stream()))
        return y

    def restrict(self, i: int, v):
        """U_i^T v (level i -> i+1)."""
        _expect(v, self.level_size(i), "v", dev=self.device)
        out = _like(v, self.level_size(i + 1))
        _check(self._lib.h2mg_transfer(self._h, int(i), 0, _ptr(v), _ptr(out), _stream()))
        return out

    def prolong(self, i: int, e):
        """U_i e (level i+1 -> i)."""
        _expect(e, self.level_size(i + 1), "e", dev=self.device)
        out = _like(e, self.level_size(i))
        _check(self._lib.h2mg_transfer(self._h, int(i), 1, _ptr(e), _ptr(out), _stream()))
        return out

    def coarse_solve(self, r, e=None):
        nl = self.level_size(self.levels)
        _expect(r, nl, "r", dev=self.device)
        if e is None:
            e = _like(r, nl)
        _expect(e, nl, "e", dev=self.device)
        _check(self._lib.h2mg_coarse_solve(self._h, _ptr(r), _ptr(e), _stream()))
        return e

    def smooth(self, i: int, f, x0=None, n: int = 1, precision: str = "f64"):
        _expect(f, self.level_size(i), "f", dev=self.device)
        _expect(x0, self.level_size(i), "x0", dev=self.device)
        x = _like(f, self.level_size(i))
        r = _like(f, self.level_size(i))
        _check(self._lib.h2mg_smooth(self._h, int(i), PRECISION[precision], _ptr(f), _ptr(x0), int(n),
                                     _ptr(x), _ptr(r), _stream()))
        return x, r

    @staticmethod
    def _opts(tol=1e-10, max_cycles=100, n_f=1, n_c=40, precision="f64", explicit_restrict_residual=False,
              outer="vcycle", use_graph=False, skip_square_levels=False, cycle="V", residual_dd=False):
        return _SolveOpts(float(tol), int(max_cycles), int(n_f), int(n_c), PRECISION[precision],
                          int(bool(explicit_restrict_residual)), OUTER[outer], int(bool(use_graph)),
                          int(bool(skip_square_levels)), CYCLE[cycle],
                          2 if residual_dd == "auto" else int(bool(residual_dd)))

    def vcycle(self, x0, r1, **kw):
        _expect(x0, self.n, "x0", dev=self.device)
        _expect(r1, self.n, "r1", dev=self.device)
        x = _like(x0, self.n)
        o = self._opts(**kw)
        _check(self._lib.h2mg_vcycle(self._h, _ptr(x0), _ptr(r1), _ptr(x), ctypes.byref(o), _stream()))
        return x

    def solve(self, b, x=None, raise_on_fail: bool = True, **kw):
        """Solve A x = b by H2-MG (Algorithm 1 repeated) for a vector or an (n, nrhs)
        block of columns, solved together in groups of four. Returns (x, info): one
        SolveInfo for a vector, a list with one per column for a block."""
        _expect(b, self.n, "b", cols=True, dev=self.device)
        bb, nrhs = _colmajor(b)
        if x is None:
            x = _new_cols(b, self.n, None if len(b.shape) == 1 else nrhs)
        _expect(x, self.n, "x", cols=True, dev=self.device)
        if tuple(x.shape) != tuple(b.shape):
            raise ValueError(f"x must have the shape of b {tuple(b.shape)}, got {tuple(x.shape)}")
        xb, _ = _colmajor(x)
        o = self._opts(**kw)
        infos = (SolveInfo * nrhs)()
        st = self._lib.h2mg_solve(self._h, _ptr(bb), _ptr(xb), nrhs, self.n, ctypes.byref(o), infos, _stream())
        _copy_back(x, xb)
        if st != 0 and (raise_on_fail or st not in (5,)):
            _check(st)
        return x, (infos[0] if len(b.shape) == 1 else list(infos))


# --------------------------------------------------------------------------- adjoint
class MaternLoss:
    """L(y, b, length, nugget) = 1/2 y^T K^{-1} y + 1^T K^{-1} b for the Matern-3/2 kernel
    matrix K = (1 + sqrt3 r/l) exp(-sqrt3 r/l) + s I in H2 form, as a torch.autograd
    function. The loss and its adjoint gradients (dL/dy = K^{-1} y, dL/db = K^{-1} 1,
    dL/dl and dL/ds through the derivative sibling dK/dl and dK/ds = I) come from one
    library call (h2mg_matern_loss_grad): this class only marshals arguments and scales
    the stored gradients by the incoming one. The forward pass builds K (and dK/dl when
    a gradient is wanted) and keeps only the gradient vectors and scalars."""

    @staticmethod
    def apply(points, y, b, length, nugget, leaf=64, q=4, eta=1.0, tol=1e-12, max_cycles=200,
              outer="fcg", n_f=1, n_c=40, precision="f64", use_graph=False, basis="chebyshev",
              basis_tol=1e-9, cycle="V", residual_dd=False):
        """``precision="mixed_f32"`` runs the V-cycles on an FP32 copy inside the float64
        outer loop (the solutions still meet ``tol`` in float64); ``basis="skeleton"``
        builds K (and so dK/dl, on the same skeletons) to the tolerance ``basis_tol``."""
        import torch

        class _Fn(torch.autograd.Function):
            @staticmethod
            def forward(ctx, y_, b_, l_, s_):
                K = H2Matrix(points, "matern32", length=float(l_), nugget=float(s_), leaf=leaf, q=q, eta=eta,
                             with_f32=(precision == "mixed_f32"), basis=basis, basis_tol=basis_tol)
                want = any(ctx.needs_input_grad)
                dK = K.sibling("dmatern32_dl", length=float(l_)) if want else None
                o = H2Matrix._opts(tol=tol, max_cycles=max_cycles, outer=outer, n_f=n_f, n_c=n_c,
                                   precision=precision, use_graph=use_graph, cycle=cycle, residual_dd=residual_dd)
                yd, bd = y_.detach().contiguous(), b_.detach().contiguous()
                _expect(yd, K.n, "y", dev=K.device)
                _expect(bd, K.n, "b", dev=K.device)
                loss, dl, ds = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
                gy = torch.empty_like(yd) if want else None
                gb = torch.empty_like(yd) if want else None
                infos = (SolveInfo * 3)()
                st = K._lib.h2mg_matern_loss_grad(K._h, dK._h if dK is not None else None, _ptr(yd), _ptr(bd),
                                                  ctypes.byref(o), ctypes.byref(loss), _ptr(gy), _ptr(gb),
                                                  ctypes.byref(dl) if want else None,
                                                  ctypes.byref(ds) if want else None, infos, _stream())
                if dK is not None:
                    dK.close()
                K.close()
                _check(st)
                ctx.save_for_backward(*(v for v in (gy, gb) if v is not None))
                ctx.scalars = (dl.value, ds.value) if want else None
                return torch.tensor(loss.value, dtype=torch.float64, device=y_.device)

            @staticmethod
            def backward(ctx, g):
                gy, gb = ctx.saved_tensors
                gv = float(g)
                dl, ds = ctx.scalars
                dev = gy.device
                return (gv * gy, gv * gb, torch.tensor(gv * dl, dtype=torch.float64, device=dev),
                        torch.tensor(gv * ds, dtype=torch.float64, device=dev))

        return _Fn.apply(y, b, length, nugget)


def solve_batched(mats, bs, xs=None, raise_on_fail: bool = True, **kw):
    """Solve independent problems mats[p] x_p = bs[p] together (h2mg_solve_batched):
    the V-cycles of all problems run from one graph launch per outer iteration when
    ``use_graph=True``. Returns (xs, [SolveInfo per problem])."""
    P = len(mats)
    if len(bs) != P or (xs is not None and len(xs) != P):
        raise ValueError("need one right-hand side (and one x) per matrix")
    for m, b in zip(mats, bs):
        _expect(b, m.n, "b", dev=m.device)
    if xs is None:
        xs = [_like(b, int(b.shape[0])) for b in bs]
    for m, x in zip(mats, xs):
        _expect(x, m.n, "x", dev=m.device)
    arr = ctypes.c_void_p * P
    hs = arr(*[m._h.value for m in mats])
    bp = arr(*[_ptr(b) for b in bs])
    xp = arr(*[_ptr(x) for x in xs])
    o = H2Matrix._opts(**kw)
    infos = (SolveInfo * P)()
    lib = load_library()
    st = lib.h2mg_solve_batched(P, hs, bp, xp, ctypes.byref(o), infos, _stream())
    if st != 0 and (raise_on_fail or st not in (5,)):
        _check(st)
    return xs, list(infos)
