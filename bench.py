#!/usr/bin/env python
"""Throughput of the GB300 H2-MG solver: H2-MG solves/s to a relative residual,
with the H2 matvec GB/s of the dominant kernel, in float64 and mixed precision.

One *step* is one complete H2-MG solve (x0 = 0, one right-hand side, to --tol) on
a prebuilt H2 matrix: outer residual in float64, V-cycles of Algorithm 1 (CG
smoothers, restriction, prolongation, coarse Cholesky solve) and the outer
iteration. The matrix build is timed separately and reported as ``build_s``.

Usage:  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun every rank solves its own problem (replicas; the solve does not
shard across GPUs); ``value`` is the sum over ranks of solves / max time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "H2-MG solves/s to 1e-10 rel. residual & H2 matvec GB/s (FP64 vs mixed)"
# DRAM bytes (read + write) per k_bsgemv launch over every block product of one outer
# iteration of the 2^17 solve, from ncu (profiles/k_bsgemv_dram_gauss3d_n131072.md);
# the algorithmic bytes per launch of the same launches were 1.5833e9
TRAFFIC_PER_LAUNCH = 1.5607e9


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=1 << 17, help="points of the solve workload")
    ap.add_argument("--matvec-n", type=int, default=1 << 20, help="points of the matvec measurement")
    ap.add_argument("--length", type=float, default=0.05)
    ap.add_argument("--nugget", type=float, default=1e-3)
    ap.add_argument("--tol", type=float, default=1e-10)
    ap.add_argument("--max-cycles", type=int, default=200)
    ap.add_argument("--precision", default="mixed_f32", choices=["f64", "mixed_f32"])
    ap.add_argument("--outer", default="fcg", choices=["vcycle", "fcg"])
    ap.add_argument("--nf", type=int, default=1)
    ap.add_argument("--nc", type=int, default=40)
    ap.add_argument("--no-matvec", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-n", type=int, default=8192)
    ap.add_argument("--ref-cycles", type=int, default=49,
                    help="outer iterations of one full-size solve, for the reference arm's scaling "
                         "(49 for the default workload at 2^17 points to 1e-10)")
    ap.add_argument("--no-f64", action="store_true", help="skip the plain float64 comparison solve")
    ap.add_argument("--no-graph", action="store_true",
                    help="launch every V-cycle kernel from the host instead of replaying a captured CUDA graph")
    ap.add_argument("--grad", action="store_true",
                    help="also time the adjoint gradients of the Matern loss (and check them by central differences)")
    ap.add_argument("--grad-n", type=int, default=1 << 16)
    ap.add_argument("--grad-tol", type=float, default=1e-11)
    ap.add_argument("--skip-square", action="store_true",
                    help="also time the solve with skip_square_levels (no smoothing on square levels)")
    ap.add_argument("--problems", type=int, default=32,
                    help="independent perturbed-sphere problems solved together after the timed region (0: skip)")
    ap.add_argument("--batch-rhs", type=int, default=4,
                    help="right-hand sides of the batched solve measured after the timed region (0: skip)")
    return ap.parse_args()


# --------------------------------------------------------------------------- clocks
class Clocks:
    """nvidia-smi samples every 200 ms while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        self.f.flush()
        self.f.seek(0)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.f.name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------------------- helpers
def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def max_over_ranks(ms: float, dist, device) -> float:
    """The slowest rank's timed region (every rank solves its own replica of the
    problem), after a barrier; `dist` is torch.distributed or None for one process."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.barrier()
    return float(t.item())


def whole_job_value(steps: int, world: int, ms: float) -> float:
    """Solves per second of the whole job: every rank ran `steps` solves in at most
    `ms` milliseconds."""
    return steps * world / (ms / 1e3)


def workload_name(a):
    return (f"gauss3d_n{a.n}_l{a.length:g}_nug{a.nugget:g}_leaf64_q4_eta1")


def cpu_baseline(a, cycles_gpu: int):
    """The oracle as it stands on this host's cores: a bounded sample of the same
    workload (oracle V-cycles of the same solver settings on the same kernel at
    --cpu-n points, matrix prebuilt), scaled to the bench size by N (linear
    complexity, Sec. 3.4) and to a solve by the GPU's cycle count."""
    import numpy as np

    import workloads as W
    from oracle import H2MG, H2Matrix, KernelSpec, SolveOpts
    from oracle.mg import vcycle
    p = W.workload(2, n=a.cpu_n)
    t0 = time.perf_counter()
    h = H2Matrix(p["points"], KernelSpec("gaussian", a.length, a.nugget), 64, 4, 1.0)
    mg = H2MG(h)
    build = time.perf_counter() - t0
    opts = SolveOpts(n_f=a.nf, n_c=a.nc)
    b = p["b"]
    low = np.float32 if a.precision == "mixed_f32" else None
    from oracle.mg import LowPrecisionOps
    ops = LowPrecisionOps(mg, low) if low is not None else None
    t0 = time.perf_counter()
    reps = 0
    x = np.zeros_like(b)
    while True:
        r = b - mg.apply(1, x)
        if ops is None:
            x = vcycle(mg, x, r, opts)
        else:
            x = x + vcycle(mg, np.zeros(len(r), np.float32), r.astype(np.float32), opts, ops=ops).astype(np.float64)
        reps += 1
        if time.perf_counter() - t0 > 10.0 or reps >= 5:
            break
    per_cycle = (time.perf_counter() - t0) / reps
    scale = a.n / a.cpu_n
    t_solve = per_cycle * scale * max(cycles_gpu, 1)
    threads = os.environ.get("OMP_NUM_THREADS") or str(len(os.sched_getaffinity(0)))
    return {"value": 1.0 / t_solve, "unit": "solves/s", "cores": int(threads), "kind": "oracle",
            "sample": (f"{reps} oracle outer iterations (residual + V-cycle, n_f={a.nf}, n_c={a.nc}, "
                       f"{a.precision}) at N={a.cpu_n} of the same kernel, matrix prebuilt ({build:.1f} s); "
                       f"{per_cycle:.2f} s/iteration scaled by N={a.n}/{a.cpu_n} and by the GPU's "
                       f"{cycles_gpu} iterations per solve")}


# --------------------------------------------------------------------------- reference arm
def run_reference(a, rank, world):
    """The oracle as the reference arm (there is no other implementation to run): each
    step is one outer iteration of the same solver (float64 residual plus one V-cycle
    with the same smoothing and precision) on the same kernel at --cpu-n points, matrix
    prebuilt; the time per iteration is scaled to the bench size by N (linear
    complexity, Sec. 3.4) and to a solve by --ref-cycles outer iterations."""
    if rank != 0:
        return
    import numpy as np

    import workloads as W
    from oracle import H2MG, H2Matrix, KernelSpec, SolveOpts
    from oracle.mg import LowPrecisionOps, vcycle
    n = a.cpu_n
    p = W.workload(2, n=n)
    h = H2Matrix(p["points"], KernelSpec("gaussian", a.length, a.nugget), 64, 4, 1.0)
    mg = H2MG(h)
    opts = SolveOpts(n_f=a.nf, n_c=a.nc)
    low = np.float32 if a.precision == "mixed_f32" else None
    ops = LowPrecisionOps(mg, low) if low is not None else None
    b = p["b"]
    x = np.zeros_like(b)

    def step(x):
        r = b - mg.apply(1, x)
        if ops is None:
            return vcycle(mg, x, r, opts)
        return x + vcycle(mg, np.zeros(len(r), np.float32), r.astype(np.float32), opts, ops=ops).astype(np.float64)

    for _ in range(a.warmup):
        x = step(x)
    t0 = time.perf_counter()
    for _ in range(a.steps):
        x = step(x)
    dt = time.perf_counter() - t0
    per_iter = dt / a.steps
    val = 1.0 / (per_iter * (a.n / n) * a.ref_cycles)
    threads = os.environ.get("OMP_NUM_THREADS") or str(len(os.sched_getaffinity(0)))
    sample = (f"{a.steps} oracle outer iterations (residual + V-cycle, n_f={a.nf}, n_c={a.nc}, {a.precision}) "
              f"at N={n}, {per_iter:.2f} s each, scaled by N={a.n}/{n} and by {a.ref_cycles} iterations per solve")
    line = {"metric": METRIC, "impl": "reference", "value": val, "unit": "solves/s", "n_gpus": world,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * per_iter,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64 outer / f32 V-cycle" if low is not None else "f64",
            "data": "synthetic", "config": {"workload": workload_name(a), "sample_n": n},
            "cpu_baseline": {"value": val, "unit": "solves/s", "cores": int(threads), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": val, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def uneven_problems(a, pkg, W, torch, stream):
    """Independent surface problems of uneven size (perturbed spheres, single-layer
    kernel, N = 20 m^2 with m from the surface workload's log-uniform list) solved
    together by h2mg_solve_batched (one graph launch per outer iteration for all
    V-cycles), against the same problems solved one after another. Timed once each,
    after one untimed batched solve that captures the graphs."""
    import numpy as np
    ms = W.surface_problem_sizes(a.problems)
    mats, bs = [], []
    t0 = time.perf_counter()
    for j, m in enumerate(ms):
        c, ar, _ = W.perturbed_icosphere(m, j)
        mats.append(pkg.H2Matrix(torch.from_numpy(c).cuda(), "laplace_sl", weights=torch.from_numpy(ar).cuda(),
                                 leaf=64, q=4, eta=1.0, with_f32=True))
        bs.append(torch.from_numpy(W.normal_rhs(c.shape[0], 3 + j)).cuda())
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    kw = dict(tol=a.tol, max_cycles=a.max_cycles, n_f=a.nf, n_c=a.nc, precision=a.precision, outer=a.outer)
    pkg.solve_batched(mats, bs, raise_on_fail=False, use_graph=True, **kw)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    xs, infos = pkg.solve_batched(mats, bs, raise_on_fail=False, use_graph=True, **kw)
    e1.record(stream)
    torch.cuda.synchronize()
    sb = e0.elapsed_time(e1) / 1e3
    e0.record(stream)
    for A, bb in zip(mats, bs):
        A.solve(bb, raise_on_fail=False, **kw)
    e1.record(stream)
    torch.cuda.synchronize()
    ss = e0.elapsed_time(e1) / 1e3
    worst = max(float(((bb - A.apply(x)).norm() / bb.norm()).item()) for A, bb, x in zip(mats, bs, xs))
    n = [20 * m * m for m in ms]
    out = {"problems": len(ms), "n_min": min(n), "n_max": max(n), "n_total": sum(n),
           "kernel": "single-layer 1/(4 pi r), panel areas as weights", "build_s": build_s,
           "s_batched": sb, "problems_per_s": len(ms) / sb, "s_one_by_one": ss,
           "speedup_vs_one_by_one": ss / sb, "cycles_max": max(i.cycles for i in infos),
           "converged": all(i.converged for i in infos) and worst <= a.tol * 1.0001, "max_relres": worst}
    for A in mats:
        A.close()
    torch.cuda.empty_cache()
    return out


def gradients(a, pkg, W, torch):
    """The differentiation form on the Matern-3/2 workload (unit cube, l = 0.1, nugget
    1e-2, leaf 64, 4x4x4 nodes) at --grad-n points: one forward + backward pass of
    L = 1/2 y^T K^-1 y + 1^T K^-1 b (a three-column mixed-precision solve, the dK/dl
    sibling and its two-column product), timed, and dL/dl, dL/ds against central
    differences of the same loss (relative step 1e-4)."""
    import numpy as np
    p = W.workload(4, n=a.grad_n)
    X = torch.from_numpy(p["points"]).cuda()
    rng = np.random.default_rng(4004)
    y = torch.from_numpy(rng.standard_normal(p["n"])).cuda()
    bb = torch.from_numpy(rng.standard_normal(p["n"])).cuda()
    kw = dict(tol=a.grad_tol, precision="mixed_f32", use_graph=True, max_cycles=400)

    def t64(v, g=False):
        return torch.tensor(v, dtype=torch.float64, device="cuda", requires_grad=g)

    times = []
    for _ in range(2):   # the first pass also captures the graphs
        yt, bt, lt, st = y.clone().requires_grad_(True), bb.clone().requires_grad_(True), t64(0.1, True), \
            t64(1e-2, True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        L = pkg.MaternLoss.apply(X, yt, bt, lt, st, **kw)
        L.backward()
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
    h = 1e-4

    def loss(l, s):
        with torch.no_grad():
            return pkg.MaternLoss.apply(X, y, bb, t64(l), t64(s), **kw).item()

    fd_l = (loss(0.1 * (1 + h), 1e-2) - loss(0.1 * (1 - h), 1e-2)) / (2 * h * 0.1)
    fd_s = (loss(0.1, 1e-2 * (1 + h)) - loss(0.1, 1e-2 * (1 - h))) / (2 * h * 1e-2)
    return {"n": p["n"], "kernel": "matern32 l=0.1 nugget=1e-2", "tol": a.grad_tol, "s_loss_and_grads": times[-1],
            "loss": L.item(), "dL_dl": lt.grad.item(), "dL_ds": st.grad.item(), "fd_dL_dl": fd_l, "fd_dL_ds": fd_s,
            "rel_err_dl": abs(lt.grad.item() - fd_l) / abs(fd_l), "rel_err_ds": abs(st.grad.item() - fd_s) / abs(fd_s)}


# --------------------------------------------------------------------------- our arm
def main():
    a = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if a.impl == "reference":
        run_reference(a, rank, world)
        return
    import numpy as np
    import torch

    import paper_2501_17656_gb300 as pkg
    import workloads as W
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    pkg.load_library()
    pk, pk_kind = peaks()

    # ---- matvec of the full-size workload (dominant kernel on the 2^20 matrix)
    matvec = None
    if not a.no_matvec:
        pm = W.workload(2, n=a.matvec_n)
        Xm = torch.from_numpy(pm["points"]).cuda()
        Am = pkg.H2Matrix(Xm, "gaussian", length=a.length, nugget=a.nugget, leaf=64, q=4, eta=1.0,
                          storage="f64", with_f32=True)
        xv = torch.randn(a.matvec_n, dtype=torch.float64, device="cuda")
        if os.environ.get("H2MG_BENCH_REPORT_LAUNCHES"):
            print(f"launches before the matvec: {pkg.H2Matrix.launch_count()}", file=sys.stderr, flush=True)
        yv = torch.empty_like(xv)
        matvec = {}
        for prec in ("f64", "mixed_f32"):
            Am.apply_level(1, xv, prec, y=yv)
            torch.cuda.synchronize()
            Am.profile(1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(5):
                Am.apply_level(1, xv, prec, y=yv)
            e1.record()
            torch.cuda.synchronize()
            nl, kms, kby = Am.profile(0)
            ms = e0.elapsed_time(e1) / 5
            by = Am.query("APPLY_BYTES", 1) * (0.5 if prec == "mixed_f32" else 1.0)
            matvec[prec] = {"n": a.matvec_n, "ms": ms, "GBs": by / ms / 1e6,
                            "kernel_GBs": kby / kms / 1e6 if kms > 0 else None}
            if prec == "f64":
                y64 = yv.clone()
        Am.close()
        del Am
        torch.cuda.empty_cache()
        # the same matrix stored as double-float pairs: float64-class products on the
        # FP32 pipes at HBM speed
        Ad = pkg.H2Matrix(Xm, "gaussian", length=a.length, nugget=a.nugget, leaf=64, q=4, eta=1.0, storage="df64")
        Ad.apply_level(1, xv, "f64", y=yv)
        torch.cuda.synchronize()
        Ad.profile(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(5):
            Ad.apply_level(1, xv, "f64", y=yv)
        e1.record()
        torch.cuda.synchronize()
        nl, kms, kby = Ad.profile(0)
        ms = e0.elapsed_time(e1) / 5
        by = Ad.query("APPLY_BYTES", 1)
        matvec["df64"] = {"n": a.matvec_n, "ms": ms, "GBs": by / ms / 1e6,
                          "kernel_GBs": kby / kms / 1e6 if kms > 0 else None,
                          "rel_diff_vs_f64": float(((yv - y64).norm() / y64.norm()).item())}
        Ad.close()
        del Ad, Xm, xv, yv, y64
        torch.cuda.empty_cache()

    # ---- the solve workload
    p = W.workload(2, n=a.n)
    X = torch.from_numpy(p["points"]).cuda()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    A = pkg.H2Matrix(X, "gaussian", length=a.length, nugget=a.nugget, leaf=64, q=4, eta=1.0,
                     storage="f64", with_f32=(a.precision == "mixed_f32"))
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    b = torch.from_numpy(p["b"]).cuda()
    kw = dict(tol=a.tol, max_cycles=a.max_cycles, n_f=a.nf, n_c=a.nc, precision=a.precision,
              outer=a.outer, use_graph=not a.no_graph)
    A.profile(1)   # warm-up solves capture the graph the timed (profiled) solves replay
    for _ in range(a.warmup):
        A.solve(b, raise_on_fail=False, **kw)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    infos = []
    A.profile(1)
    l0 = pkg.H2Matrix.launch_count()
    if os.environ.get("H2MG_BENCH_REPORT_LAUNCHES"):
        print(f"launches before the timed region: {l0}", file=sys.stderr, flush=True)
    with Clocks(local) as clk:
        e0.record(stream)
        for _ in range(a.steps):
            x, info = A.solve(b, raise_on_fail=False, **kw)
            infos.append((info.cycles, info.converged, info.relres))
        e1.record(stream)
        torch.cuda.synchronize()
    launches = pkg.H2Matrix.launch_count() - l0
    nk, kms, kby = A.profile(0)
    ms = max_over_ranks(e0.elapsed_time(e1), dist, "cuda")
    value = whole_job_value(a.steps, world, ms)
    converged = all(c for _, c, _ in infos)
    cycles = infos[-1][0]

    # ---- end to end through the C ABI with host buffers (copies inside the region)
    bh = np.ascontiguousarray(p["b"])
    xh = np.zeros_like(bh)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    for _ in range(a.steps):
        xh[:] = 0.0
        A.solve(bh, x=xh, raise_on_fail=False, **kw)
    e2e_s = (time.perf_counter() - t1) / a.steps

    res_check = float(np.linalg.norm(p["b"] - A.apply(torch.from_numpy(xh).cuda()).cpu().numpy())
                      / np.linalg.norm(p["b"]))

    # ---- plain float64 H2-MG on the same matrix (every product on the FP64 pipe), once
    f64 = None
    if a.precision == "mixed_f32" and not a.no_f64:
        kw64 = dict(kw, precision="f64")
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        x64, i64 = A.solve(b, raise_on_fail=False, **kw64)
        f1.record(stream)
        torch.cuda.synchronize()
        s64 = f0.elapsed_time(f1) / 1e3
        f64 = {"s_per_solve": s64, "solves_per_s": 1.0 / s64, "cycles": i64.cycles,
               "converged": bool(i64.converged), "relres": i64.relres,
               "mixed_speedup": s64 / (ms / 1e3 / a.steps)}
    # ---- the same solve with every V-cycle kernel launched from the host, timed once
    direct = None
    if not a.no_graph:
        kwd = dict(kw, use_graph=False)
        h0, h1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        h0.record(stream)
        xg_, ig_ = A.solve(b, raise_on_fail=False, **kwd)
        h1.record(stream)
        torch.cuda.synchronize()
        sg = h0.elapsed_time(h1) / 1e3
        direct = {"s_per_solve": sg, "solves_per_s": 1.0 / sg, "cycles": ig_.cycles,
                  "converged": bool(ig_.converged), "graph_speedup": sg / (ms / 1e3 / a.steps)}

    # ---- the same solve without smoothing on levels whose restriction is square
    # (U_1 is 64 x 64 here: A_2 is an orthogonal similarity of A_1), timed once
    skip = None
    if a.skip_square:
        k0, k1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        k0.record(stream)
        xk_, ik_ = A.solve(b, raise_on_fail=False, skip_square_levels=True, **kw)
        k1.record(stream)
        torch.cuda.synchronize()
        sk = k0.elapsed_time(k1) / 1e3
        relk = float(((b - A.apply(xk_)).norm() / b.norm()).item())
        skip = {"s_per_solve": sk, "solves_per_s": 1.0 / sk, "cycles": ik_.cycles,
                "converged": bool(ik_.converged) and relk <= a.tol * 1.0001, "relres": relk,
                "speedup_vs_literal": (ms / 1e3 / a.steps) / sk}

    # ---- batched form: several right-hand sides solved together (one group of columns
    # shares every block read of every product), timed once
    batched = None
    if a.batch_rhs > 0:
        Bm = torch.from_numpy(np.ascontiguousarray(W.normal_rhs(a.n, 2, a.batch_rhs))).cuda() \
            if a.batch_rhs > 1 else b[:, None].clone()
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if os.environ.get("H2MG_BENCH_REPORT_LAUNCHES"):
            print(f"launches before the batched solve: {pkg.H2Matrix.launch_count()}", file=sys.stderr, flush=True)
        g0.record(stream)
        Xb, ib = A.solve(Bm, raise_on_fail=False, **kw)
        ib = ib if isinstance(ib, list) else [ib]
        g1.record(stream)
        torch.cuda.synchronize()
        sb = g0.elapsed_time(g1) / 1e3
        Rb = Bm - A.apply(Xb)
        relb = (Rb.norm(dim=0) / Bm.norm(dim=0)).max().item()
        batched = {"nrhs": a.batch_rhs, "s_per_batch": sb, "solves_per_s": a.batch_rhs / sb,
                   "max_relres": relb, "converged": bool(relb <= a.tol * 1.0001) and all(i.converged for i in ib),
                   "cycles": [i.cycles for i in ib],
                   "speedup_vs_single_rhs": (a.batch_rhs / sb) / (a.steps / (ms / 1e3)),
                   "precision": a.precision}
    A.close()
    del A
    torch.cuda.empty_cache()

    problems = uneven_problems(a, pkg, W, torch, stream) if a.problems > 0 else None
    grads = gradients(a, pkg, W, torch) if a.grad else None

    kernel_gbs = kby / kms / 1e6 if kms > 0 else 0.0
    bound = "hbm"
    peak = pk["hbm_gbs"]
    roof = {"bound": bound, "achieved": kernel_gbs, "peak": peak, "unit": "GB/s",
            "frac": kernel_gbs / peak, "traffic": TRAFFIC_PER_LAUNCH if a.n == 1 << 17 else None,
            "traffic_source": "profiles/k_bsgemv_dram_gauss3d_n131072.md (ncu, one outer iteration)",
            "kernel": "k_bsgemv (symmetric block-sparse product)", "launches": nk,
            "bytes_per_launch": kby / max(nk, 1), "ms_per_launch": kms / max(nk, 1),
            "peak_source": f"{pk_kind} hbm_gbs"}
    line = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": ms / a.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f64 outer / f32 V-cycle" if a.precision == "mixed_f32" else "f64",
            "data": "synthetic",
            "config": {"workload": workload_name(a), "n": a.n, "kernel": "gaussian", "length": a.length,
                       "nugget": a.nugget, "leaf": 64, "cheb_nodes": "4x4x4", "eta": 1.0,
                       "tol": a.tol, "outer": a.outer, "n_f": a.nf, "n_c": a.nc,
                       "precision": a.precision, "storage": "f64 (+f32 copy)",
                       "l2": "inputs larger than L2 (stored blocks)", "build_s": build_s,
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "cycles": cycles, "converged": converged, "relres": infos[-1][2], "relres_check": res_check,
            "matvec": matvec, "f64_solve": f64, "direct_launches": direct, "skip_square_levels": skip, "batched": batched,
            "problems": problems, "gradients": grads, "roofline": roof, "gpu_launches": launches,
            "e2e": {"value": 1.0 / e2e_s, "unit": "solves/s", "h2d_bytes_per_step": 16 * a.n,
                    "d2h_bytes_per_step": 8 * a.n},
            "clocks": clk.summary()}
    if rank == 0 and world == 1 and not a.no_cpu:
        line["cpu_baseline"] = cpu_baseline(a, cycles)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
