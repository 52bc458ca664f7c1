"""H2-MG of the oracle: Galerkin coarse operators, CG smoother, Algorithm 1 (one
V-cycle), repeated V-cycles, and the mixed-precision refinement loop.

Test infrastructure: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` leg of ``bench.py`` may import this package.

Section 3.3 of the paper. With orthonormal bases the restricted operator is
A_2 = U_1^T D V_1^T + D_2 + U_2 (... (D_l + U_l S_l V_l) ...) V_2 (eq. a2_str), an
H2 matrix of the same structure whose close part is the reduced U_1^T D U_1. The
oracle groups the near part level by level (a reading of eq. a2_str; identical
sums): for every inadmissible pair (c, c') of tree level m(i),

    P_i(c, c') = sum over child pairs (a, a') of
                 E'_a^T [P_{i-1}(a, a') if (a, a') is inadmissible, else S(a, a')] E'_a'

with P_1 = D and, at i = 2, P_2(c, c') = U_c^T D(c, c') U_c'. Then
A_i = P_i + (the coupling chain of levels t*..m(i), with the identity basis at
level m(i)). The coarsest level is l = L - t* + 1 (tree level t*+1), where A_l is
assembled densely (its coupling chain has a single transfer) and solved by
Cholesky (dir_sol, Section 3.3).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla

from .h2 import BlockOp, H2Matrix


@dataclass
class SolveOpts:
    tol: float = 1e-8
    max_cycles: int = 100
    n_f: int = 1                      # fine-level CG iterations (Remark rem:fine_coarse)
    n_c: int = 40                     # coarse-level CG iterations
    explicit_restrict_residual: bool = False
    coarse_level: int = -1            # -1: natural l = L - t* + 1
    skip_square_levels: bool = False  # no smoothing where U_{i-1} is square (A_i similar to A_{i-1})
    cycle: str = "V"                  # multigrid cycle of the outer loops: "V", "W" or "F"


@dataclass
class SolveInfo:
    cycles: int = 0
    relres: float = float("nan")
    converged: bool = False
    history: list = field(default_factory=list)


class H2MG:
    """Multigrid hierarchy A_1..A_l on an oracle H2 matrix."""

    def __init__(self, h: H2Matrix, coarse_level: int = -1):
        self.h = h
        T = h.tree
        self.L = T.L
        self.l_natural = 1 if h.tstar is None else T.L - h.tstar + 1
        self.l = self.l_natural if coarse_level is None or coarse_level < 0 else int(coarse_level)
        if not (1 <= self.l <= self.l_natural):
            raise ValueError(f"coarse_level must be in [1, {self.l_natural}]")
        self._build_near()
        self._dense_coarse()

    # level -> tree level of its coefficient space
    def m(self, i: int) -> int:
        return self.L - i + 2

    def size(self, i: int) -> int:
        if i == 1:
            return self.h.tree.n
        return int(self.h.coef_offsets(self.m(i))[-1])

    # -- coarse near fields P_i ----------------------------------------------------
    def _pair_index(self, ell):
        return {(int(t), int(s)): k for k, (t, s) in enumerate(self.h.inadm[ell])}

    def _far_index(self, ell):
        return {(int(t), int(s)): k for k, (t, s) in enumerate(self.h.far[ell])}

    def _build_near(self):
        h = self.h
        self.P = {}
        if self.l < 2:
            return
        Lt = self.L
        # i = 2: U_c^T D(c, c') U_c'
        self.P[2] = [h.U[int(t)].T @ B @ h.U[int(s)] for (t, s), B in zip(h.near, h.D)]
        for i in range(3, self.l + 1):
            mc, mf = self.m(i), self.m(i - 1)
            fine_in = self._pair_index(mf)
            fine_far = self._far_index(mf)
            Pf = self.P[i - 1]
            Sf = h.S.get(mf, [])
            blocks = []
            for (c, cp) in h.inadm[mc]:
                acc = None
                for a in (2 * c, 2 * c + 1):
                    for ap in (2 * cp, 2 * cp + 1):
                        key = (int(a), int(ap))
                        if key in fine_in:
                            M = Pf[fine_in[key]]
                        else:
                            M = Sf[fine_far[key]]
                        term = h.Et[(mf, int(a))].T @ M @ h.Et[(mf, int(ap))]
                        acc = term if acc is None else acc + term
                blocks.append(acc)
            self.P[i] = blocks
        del Lt

    # -- operators A_i ----------------------------------------------------------------
    def near_op(self, i: int):
        """P_i as a block operator on the level-m(i) coefficients."""
        if not hasattr(self, "_near_ops"):
            self._near_ops = {}
        if i not in self._near_ops:
            off = self.h.coef_offsets(self.m(i))
            self._near_ops[i] = BlockOp(off, off, self.h.inadm[self.m(i)], self.P[i])
        return self._near_ops[i]

    def apply(self, i: int, x: np.ndarray) -> np.ndarray:
        """A_i x (i = 1: user point order; i >= 2: level-m(i) coefficient order)."""
        h = self.h
        if i == 1:
            return h.apply(x)
        m = self.m(i)
        y = self.near_op(i).matvec(x)
        xh = {m: x}
        h._up(xh, h.tstar, m)
        yh = {}
        h._couple(xh, yh, h.tstar, m)
        h._down(yh, h.tstar, m)
        return y + yh[m]

    def restrict(self, i: int, v: np.ndarray) -> np.ndarray:
        """U_i^T v: from level i to level i+1 (r_{i+1} = U_i^T (...), Alg. 1)."""
        h = self.h
        if i == 1:
            return h.leaf_restrict(v[h.tree.perm])
        xh = {self.m(i): v}
        h._up(xh, self.m(i) - 1, self.m(i))
        return xh[self.m(i) - 1]

    def prolong(self, i: int, e: np.ndarray) -> np.ndarray:
        """V_i^T e = U_i e: from level i+1 to level i (Alg. 1, prolongation)."""
        h = self.h
        if i == 1:
            out = np.empty((h.tree.n,) + e.shape[1:], dtype=e.dtype)
            out[h.tree.perm] = h.leaf_prolong(e)
            return out
        return h.down_op(self.m(i)).matvec(e)

    def _dense_coarse(self):
        """A_l as a dense matrix (A_l applied to the identity) and its Cholesky factor."""
        n = self.size(self.l)
        # A_l applied to the identity, 256 columns at a time (bounded gather sizes)
        self.Al = np.concatenate([self.apply(self.l, np.eye(n)[:, c:c + 256]) for c in range(0, n, 256)],
                                 axis=1) if n > 0 else np.zeros((0, 0))
        self.Al = 0.5 * (self.Al + self.Al.T)     # symmetric by construction; remove round-off
        try:
            self.chol = sla.cho_factor(self.Al, lower=True)
        except np.linalg.LinAlgError:
            self.chol = None

    def dir_sol(self, r: np.ndarray) -> np.ndarray:
        """e_l = dir_sol(A_l, r_l) by the Cholesky factor (in float64)."""
        if self.chol is None:
            raise np.linalg.LinAlgError("coarse operator is not positive definite")
        return sla.cho_solve(self.chol, r.astype(np.float64))


# ---------------------------------------------------------------------------------
# CG smoother (Hestenes-Stiefel) and one V-cycle (Algorithm 1)
# ---------------------------------------------------------------------------------

def cg(apply, f: np.ndarray, x0: np.ndarray | None, n: int):
    """``n`` iterations of textbook CG on A x = f from x0 (Iter(A, f, x0), Section 3.3).

    Returns (x, r) with r the recurrence residual. Stops early when p^T A p <= 0
    (breakdown; also covers a zero residual) or when r^T r <= (1e-30 |f|)^2.
    """
    if x0 is None:
        x = np.zeros_like(f)
        r = f.copy()
    else:
        x = x0.copy()
        r = f - apply(x)
    p = r.copy()
    rho = float(r @ r)
    stop = (1e-30 * float(np.sqrt(f @ f))) ** 2
    for _ in range(n):
        q = apply(p)
        pq = float(p @ q)
        if not pq > 0.0:
            break
        alpha = rho / pq
        x = x + alpha * p
        r = r - alpha * q
        rho_new = float(r @ r)
        if rho_new <= stop:
            break
        p = r + (rho_new / rho) * p
        rho = rho_new
    return x, r


def vcycle(mg: H2MG, x0: np.ndarray, r1: np.ndarray, opts: SolveOpts, ops=None) -> np.ndarray:
    """One V-cycle of Algorithm 1 given x0 and r_1 = b - A_1 x0; returns x*.

    ``ops`` optionally supplies another copy of the operators (the rounded copy of
    the mixed-precision loop); the coarse solve stays in float64.
    """
    ops = mg if ops is None else ops
    l = mg.l
    if l == 1:
        return x0 + mg.dir_sol(r1).astype(r1.dtype)
    def iters(i):
        # a level whose restriction U_{i-1} is square (N_i = N_{i-1}; the columns are
        # orthonormal) is an orthogonal similarity of the finer one, not a coarser space
        if i == 1:
            return opts.n_f
        if opts.skip_square_levels and mg.size(i) == mg.size(i - 1):
            return 0
        return opts.n_c

    r = {1: r1}
    et = {}
    for i in range(1, l):
        n_i = iters(i)
        A = (lambda v, i=i: ops.apply(i, v))
        et[i], rho = cg(A, r[i], None, n_i)
        res = r[i] - A(et[i]) if opts.explicit_restrict_residual else rho
        r[i + 1] = ops.restrict(i, res)
    e = mg.dir_sol(r[l]).astype(r1.dtype)
    for i in range(l - 1, 0, -1):
        n_i = iters(i)
        A = (lambda v, i=i: ops.apply(i, v))
        et[i] = et[i] + ops.prolong(i, e)
        e, _ = cg(A, r[i], et[i], n_i)
    return x0 + e


def _iters(mg: H2MG, opts: SolveOpts, i: int) -> int:
    if i == 1:
        return opts.n_f
    if opts.skip_square_levels and mg.size(i) == mg.size(i - 1):
        return 0
    return opts.n_c


def cycle(mg: H2MG, x0: np.ndarray, r1: np.ndarray, opts: SolveOpts, kind: str = "V", ops=None) -> np.ndarray:
    """One multigrid cycle of type ``kind`` given x0 and r_1 = b - A_1 x0; returns x*.

    The recursive form of the textbook cycles, with the smoother, transfers and coarse
    solve of Algorithm 1: on level i < l the correction of A_i e = f starts from a
    guess g (zero on the first visit), is pre-smoothed, e~ = Iter(A_i, f, g); the
    residual f - A_i e~ is restricted, r_{i+1} = U_i^T (f - A_i e~); the coarse
    correction is gamma visits of level i + 1 on A_{i+1} e = r_{i+1} (each from the
    previous visit's result); then e~ += V_i^T e_{i+1} and e = Iter(A_i, f, e~). Level
    l solves directly, e_l = dir_sol(A_l, r_l). A V-cycle visits the coarser level once
    (this is Algorithm 1), a W-cycle twice, and an F-cycle runs an F-cycle and then a
    V-cycle there (Sec. 3.3 names W- and F-cycles as further options)."""
    ops = mg if ops is None else ops
    l = mg.l
    dt = r1.dtype

    def visit(i, f, g, k):
        if i == l:
            return mg.dir_sol(f).astype(dt)
        n_i = _iters(mg, opts, i)
        A = (lambda v, i=i: ops.apply(i, v))
        et, rho = cg(A, f, g, n_i)
        res = f - A(et) if opts.explicit_restrict_residual else rho
        rc = ops.restrict(i, res)
        kids = {"V": ("V",), "W": ("W", "W"), "F": ("F", "V")}[k]
        e = None
        for kk in kids:
            e = visit(i + 1, rc, e, kk)
        et = et + ops.prolong(i, e)
        e, _ = cg(A, f, et, n_i)
        return e

    return x0 + visit(1, r1, None, kind)


def anorm_error(mg: H2MG, x: np.ndarray, x_true: np.ndarray, nb: float) -> float:
    """The paper's stopping quantity (e^T A e)^{1/2} / |b|_2 with e = x - x_true
    (Sec. 4.1, for right-hand sides b = A x_true)."""
    e = x - x_true
    return float(np.sqrt(max(float(e @ mg.apply(1, e)), 0.0))) / nb


def solve(mg: H2MG, b: np.ndarray, opts: SolveOpts, x0: np.ndarray | None = None,
          x_true: np.ndarray | None = None):
    """Repeated cycles until |b - A x| / |b| <= tol (x* feeds the next cycle):
    Algorithm 1's V-cycle, or the W- or F-cycle of ``opts.cycle``. With ``x_true``
    the test is the paper's A-norm error (e^T A e)^{1/2} / |b| < tol instead."""
    x = np.zeros_like(b) if x0 is None else x0.astype(np.float64).copy()
    nb = float(np.linalg.norm(b))
    info = SolveInfo()
    for cyc in range(opts.max_cycles + 1):
        r = b - mg.apply(1, x)
        rel = float(np.linalg.norm(r)) / nb if nb > 0 else 0.0
        if x_true is not None:
            rel = anorm_error(mg, x, x_true, nb)
        info.history.append(rel)
        info.cycles, info.relres = cyc, rel
        if rel <= opts.tol:
            info.converged = True
            break
        if cyc == opts.max_cycles:
            break
        x = vcycle(mg, x, r, opts) if opts.cycle == "V" else cycle(mg, x, r, opts, opts.cycle)
    return x, info


def solve_cg(mg: H2MG, b: np.ndarray, opts: SolveOpts, x_true: np.ndarray | None = None):
    """Unpreconditioned CG on A x = b from x0 = 0, the paper's comparison solver
    (Sec. 4: CG iterations against V-cycles), textbook recurrences: q = A p,
    alpha = rho / p^T q, x += alpha p, r -= alpha q, rho' = r^T r, p = r + (rho'/rho) p.
    Stops when the recurrence residual |r| / |b| <= tol (with ``x_true``: the A-norm
    error, as in ``solve``); ``cycles`` counts CG iterations (one product each) and
    ``relres`` is recomputed explicitly at the end."""
    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rho = float(r @ r)
    nb = float(np.linalg.norm(b))
    info = SolveInfo()
    for it in range(opts.max_cycles + 1):
        rel = float(np.sqrt(rho)) / nb if nb > 0 else 0.0
        if x_true is not None:
            rel = anorm_error(mg, x, x_true, nb)
        info.history.append(rel)
        info.cycles = it
        if rel <= opts.tol:
            info.converged = True
            break
        if it == opts.max_cycles:
            break
        q = mg.apply(1, p)
        pq = float(p @ q)
        if not pq > 0.0:
            break
        alpha = rho / pq
        x = x + alpha * p
        r = r - alpha * q
        rho_new = float(r @ r)
        p = r + (rho_new / rho) * p
        rho = rho_new
    info.relres = float(np.linalg.norm(b - mg.apply(1, x))) / nb if nb > 0 else 0.0
    return x, info


def solve_fcg(mg: H2MG, b: np.ndarray, opts: SolveOpts, low=None, precond=None):
    """Flexible CG preconditioned by one V-cycle (multigrid used to precondition
    another iteration, Section 3.2). The V-cycle with CG smoothers is a nonlinear
    map, so each new direction is made A-orthogonal to the previous one (flexible
    CG with one stored direction). The residual is recomputed explicitly in float64
    each iteration; ``low`` runs the V-cycle on rounded operators as in
    ``solve_mixed``; ``opts.cycle`` selects a W- or F-cycle instead. ``precond``
    (a map r -> z) replaces the cycle altogether. ``cycles`` counts cycles."""
    ops = None if low is None else LowPrecisionOps(mg, low)
    x = np.zeros_like(b)
    nb = float(np.linalg.norm(b))
    info = SolveInfo()
    p_prev = q_prev = None
    for cyc in range(opts.max_cycles + 1):
        r = b - mg.apply(1, x)
        rel = float(np.linalg.norm(r)) / nb if nb > 0 else 0.0
        info.history.append(rel)
        info.cycles, info.relres = cyc, rel
        if rel <= opts.tol:
            info.converged = True
            break
        if cyc == opts.max_cycles:
            break
        if precond is not None:
            z = precond(r)
        elif ops is None:
            z = vcycle(mg, np.zeros_like(r), r, opts) if opts.cycle == "V" else \
                cycle(mg, np.zeros_like(r), r, opts, opts.cycle)
        else:
            rl = r.astype(low)
            z = (vcycle(mg, np.zeros_like(rl), rl, opts, ops=ops) if opts.cycle == "V" else
                 cycle(mg, np.zeros_like(rl), rl, opts, opts.cycle, ops=ops)).astype(np.float64)
        if p_prev is None:
            p = z
        else:
            beta = -float(z @ q_prev) / float(p_prev @ q_prev)
            p = z + beta * p_prev
        q = mg.apply(1, p)
        alpha = float(p @ r) / float(p @ q)
        x = x + alpha * p
        p_prev, q_prev = p, q
    return x, info


def solve_mixed(mg: H2MG, b: np.ndarray, opts: SolveOpts, low=np.float32):
    """Iterative refinement: float64 residual and update around a V-cycle whose
    operators and vectors are rounded to ``low`` (the coarse solve stays float64)."""
    lowmg = LowPrecisionOps(mg, low)
    x = np.zeros_like(b)
    nb = float(np.linalg.norm(b))
    info = SolveInfo()
    for cyc in range(opts.max_cycles + 1):
        r = b - mg.apply(1, x)
        rel = float(np.linalg.norm(r)) / nb if nb > 0 else 0.0
        info.history.append(rel)
        info.cycles, info.relres = cyc, rel
        if rel <= opts.tol:
            info.converged = True
            break
        if cyc == opts.max_cycles:
            break
        rl = r.astype(low)
        e = vcycle(mg, np.zeros_like(rl), rl, opts, ops=lowmg) if opts.cycle == "V" else \
            cycle(mg, np.zeros_like(rl), rl, opts, opts.cycle, ops=lowmg)
        x = x + e.astype(np.float64)
    return x, info


class LowPrecisionOps:
    """The level operators, restriction and prolongation with every stored block
    rounded to ``dtype`` (products then run in that precision)."""

    def __init__(self, mg: H2MG, dtype):
        self.mg = mg
        self.h = mg.h.astype(dtype)
        self.P = {i: [b.astype(dtype) for b in lst] for i, lst in mg.P.items()}
        self.l = mg.l
        sub = H2MG.__new__(H2MG)
        sub.h, sub.P, sub.L, sub.l = self.h, self.P, mg.L, mg.l
        self._sub = sub

    def m(self, i):
        return self.mg.m(i)

    def apply(self, i, x):
        return self._sub.apply(i, x)

    def restrict(self, i, v):
        return self._sub.restrict(i, v)

    def prolong(self, i, e):
        return self._sub.prolong(i, e)
