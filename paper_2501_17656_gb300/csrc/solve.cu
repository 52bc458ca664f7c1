// solve.cu -- the smoother Iter(A_i, f, x0) (textbook CG), restriction U_i^T and
// prolongation V_i^T = U_i, one V-cycle of Algorithm 1 and the outer iteration
// (Sec. 3.3). All multigrid vectors are float64 on the device; the scalars of CG
// live in device memory so that a V-cycle never waits for the host.
#include <algorithm>
#include <chrono>
#include <cmath>

#include "internal.h"

namespace h2mg {

// ----------------------------------------------------------------------------- reductions
constexpr int NPART = 256;
struct CGState {
  double rho[2];   // r^T r, double-buffered by iteration parity
  double thresh;
  int stopped;
};

__device__ double block_reduce_sum(double v) {
  __shared__ double sh[32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += sh[i];
  __syncthreads();
  return s;   // valid in thread 0
}

__global__ void k_dot_part(const double* __restrict__ a, const double* __restrict__ b, int64_t n,
                           double* __restrict__ part) {
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    s = fma(a[i], b[i], s);
  s = block_reduce_sum(s);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__device__ double sum_parts(const double* part, int np) {
  double s = 0.0;
  for (int i = 0; i < np; ++i) s += part[i];
  return s;
}

static int part_grid(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>(NPART, (n + 1023) / 1024)); }

// init: rho = r.r, thresh = (1e-30 |f|)^2
__global__ void k_cg_init(const double* __restrict__ prr, int nrr, const double* __restrict__ pff, int nff,
                          CGState* st) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double rr = sum_parts(prr, nrr), ff = sum_parts(pff, nff);
    double t = 1e-30 * sqrt(ff);
    st->rho[0] = rr;
    st->thresh = t * t;
    st->stopped = 0;
  }
}

// Sum of np (<= 256) partials, by every CTA (blockDim 256).
__device__ double cta_sum_parts(const double* __restrict__ part, int np) {
  __shared__ double sh[8];
  double v = threadIdx.x < np ? part[threadIdx.x] : 0.0;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  for (int i = 0; i < 8; ++i) s += sh[i];
  __syncthreads();
  return s;
}

// alpha = rho / p^T q (stop before the update if p^T q <= 0); x += alpha p;
// r -= alpha q; partials of r^T r. Every CTA takes the same decision.
__global__ void __launch_bounds__(256) k_cg_update(double* __restrict__ x, double* __restrict__ r,
                                                   const double* __restrict__ p, const double* __restrict__ q,
                                                   int64_t n, CGState* st, const double* __restrict__ ppq, int np,
                                                   int par, double* __restrict__ part) {
  const double pq = cta_sum_parts(ppq, np);
  bool go = !st->stopped;
  if (go && !(pq > 0.0)) {
    go = false;
    if (blockIdx.x == 0 && threadIdx.x == 0) st->stopped = 1;
  }
  const double al = go ? st->rho[par] / pq : 0.0;
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double ri = r[i];
    if (go) {
      x[i] = fma(al, p[i], x[i]);
      ri = fma(-al, q[i], ri);
      r[i] = ri;
    }
    s = fma(ri, ri, s);
  }
  s = block_reduce_sum(s);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// rho' = r^T r; stop (after the update) if rho' <= thresh; else p = r + (rho'/rho) p.
__global__ void __launch_bounds__(256) k_cg_p(double* __restrict__ p, const double* __restrict__ r, int64_t n,
                                              CGState* st, const double* __restrict__ prr, int np, int par) {
  const double rn = cta_sum_parts(prr, np);
  if (st->stopped) return;
  if (rn <= st->thresh) {
    if (blockIdx.x == 0 && threadIdx.x == 0) st->stopped = 1;
    return;
  }
  const double be = rn / st->rho[par];
  if (blockIdx.x == 0 && threadIdx.x == 0) st->rho[par ^ 1] = rn;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = fma(be, p[i], r[i]);
}

// y = a*x + b*y  (elementwise)
__global__ void k_axpby(double a, const double* __restrict__ x, double b, double* __restrict__ y, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = a * x[i] + b * y[i];
}
// z = x - y
__global__ void k_sub(const double* __restrict__ x, const double* __restrict__ y, double* __restrict__ z, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    z[i] = x[i] - y[i];
}
// z = x + y
__global__ void k_add(const double* __restrict__ x, const double* __restrict__ y, double* __restrict__ z, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    z[i] = x[i] + y[i];
}

static int vec_grid(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>(2048, (n + 255) / 256)); }

// ----------------------------------------------------------------------------- transfers
// r2[j*KC + b] = sum_i U_j[i, b] v[perm[leafoff[j] + i]]
__global__ void k_restrict_leaf(const double* __restrict__ UT, int KD, int KC, const double* __restrict__ v,
                                const int* __restrict__ leafoff, const int* __restrict__ perm,
                                double* __restrict__ out) {
  __shared__ double xs[64];
  int j = blockIdx.x;
  int p0 = leafoff[j], nj = leafoff[j + 1] - p0;
  for (int i = threadIdx.x; i < KD; i += blockDim.x) xs[i] = i < nj ? v[perm[p0 + i]] : 0.0;
  __syncthreads();
  const double* Uj = UT + (int64_t)j * KD * KC;
  for (int b = threadIdx.x; b < KC; b += blockDim.x) {
    double acc = 0.0;
    for (int i = 0; i < KD; ++i) acc += Uj[b + i * KC] * xs[i];
    out[(int64_t)j * KC + b] = acc;
  }
}
// v[perm[...]] += sum_b U_j[i, b] e[j*KC + b]
__global__ void k_prolong_leaf(const double* __restrict__ U, int KD, int KC, const double* __restrict__ e,
                               const int* __restrict__ leafoff, const int* __restrict__ perm,
                               double* __restrict__ v) {
  __shared__ double es[64];
  int j = blockIdx.x;
  for (int b = threadIdx.x; b < KC; b += blockDim.x) es[b] = e[(int64_t)j * KC + b];
  __syncthreads();
  int p0 = leafoff[j], nj = leafoff[j + 1] - p0;
  const double* Uj = U + (int64_t)j * KD * KC;
  for (int i = threadIdx.x; i < nj; i += blockDim.x) {
    double acc = 0.0;
    for (int b = 0; b < KC; ++b) acc += Uj[i + b * KD] * es[b];
    v[perm[p0 + i]] += acc;
  }
}
// out[p*KC + b] = sum_{c in children(p)} sum_a E'_c[a, b] v[c*KC + a]
__global__ void k_restrict(const double* __restrict__ ET, int KC, const double* __restrict__ v,
                           double* __restrict__ out) {
  __shared__ double xs[128];
  int p = blockIdx.x;
  for (int i = threadIdx.x; i < 2 * KC; i += blockDim.x) xs[i] = v[(int64_t)2 * p * KC + i];
  __syncthreads();
  for (int b = threadIdx.x; b < KC; b += blockDim.x) {
    double acc = 0.0;
    for (int c = 0; c < 2; ++c) {
      const double* E = ET + (int64_t)(2 * p + c) * KC * KC;
      for (int a = 0; a < KC; ++a) acc += E[b + a * KC] * xs[c * KC + a];
    }
    out[(int64_t)p * KC + b] = acc;
  }
}
// v[c*KC + a] += sum_b E'_c[a, b] e[parent*KC + b]
__global__ void k_prolong(const double* __restrict__ E, int KC, const double* __restrict__ e,
                          double* __restrict__ v) {
  __shared__ double es[64];
  int c = blockIdx.x;
  for (int b = threadIdx.x; b < KC; b += blockDim.x) es[b] = e[(int64_t)(c >> 1) * KC + b];
  __syncthreads();
  const double* Ec = E + (int64_t)c * KC * KC;
  for (int a = threadIdx.x; a < KC; a += blockDim.x) {
    double acc = 0.0;
    for (int b = 0; b < KC; ++b) acc += Ec[a + b * KC] * es[b];
    v[(int64_t)c * KC + a] += acc;
  }
}

// ----------------------------------------------------------------------------- host
int64_t level_size(const Matrix& M, int i) {
  if (i == 1) return M.n;
  return (int64_t)(1 << (M.L - i + 2)) * M.KC;
}

struct Work {
  double *r[40], *et[40];
  double *cr, *cp, *cq, *t1, *t2;
  double *pa, *pb;
  CGState* st;
};

static Work work(Matrix& M) {
  Work W{};
  if (!M.wvec.p) {
    size_t tot = 0;
    for (int i = 1; i <= M.lev; ++i) tot += 2 * (size_t)level_size(M, i);
    size_t nmax = 0;
    for (int i = 1; i <= M.lev; ++i) nmax = std::max(nmax, (size_t)level_size(M, i));
    tot += 5 * nmax;
    M.wvec.bytes = sizeof(double) * tot;
    M.wvec.p = M.alloc(M.wvec.bytes);
    M.wred.bytes = sizeof(double) * 2 * NPART + sizeof(CGState) + 64;
    M.wred.p = M.alloc(M.wred.bytes);
  }
  double* p = (double*)M.wvec.p;
  size_t nmax = 0;
  for (int i = 1; i <= M.lev; ++i) {
    W.r[i] = p;
    p += level_size(M, i);
    W.et[i] = p;
    p += level_size(M, i);
    nmax = std::max(nmax, (size_t)level_size(M, i));
  }
  W.cr = p; p += nmax;
  W.cp = p; p += nmax;
  W.cq = p; p += nmax;
  W.t1 = p; p += nmax;
  W.t2 = p; p += nmax;
  W.pa = (double*)M.wred.p;
  W.pb = W.pa + NPART;
  W.st = (CGState*)(W.pb + NPART);
  return W;
}

static void dot_part(const double* a, const double* b, int64_t n, double* part, cudaStream_t s) {
  { k_dot_part<<<part_grid(n), 256, 0, s>>>(a, b, n, part); ::h2mg::count_launch(); }
  H2_LAUNCH_CHECK();
}

// n CG iterations on A_i x = f from x0 (nullptr: zero). x receives the iterate; r (if
// not null) the recurrence residual. Follows Hestenes-Stiefel with the breakdown
// guard p^T A p <= 0 and the stop r^T r <= (1e-30 |f|)^2.
void smooth(Matrix& M, int i, bool f32, const double* f, const double* x0, int n, double* x,
            double* r, cudaStream_t s) {
  Work W = work(M);
  int64_t N = level_size(M, i);
  double* rr = r ? r : W.cr;
  int g = vec_grid(N);
  if (x0 == nullptr) {
    H2_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * N, s));
    H2_CUDA(cudaMemcpyAsync(rr, f, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
  } else {
    if (x != x0) H2_CUDA(cudaMemcpyAsync(x, x0, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
    apply_level(M, i, f32, x, W.cq, s);
    { k_sub<<<g, 256, 0, s>>>(f, W.cq, rr, N); ::h2mg::count_launch(); }
    H2_LAUNCH_CHECK();
  }
  H2_CUDA(cudaMemcpyAsync(W.cp, rr, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
  dot_part(rr, rr, N, W.pa, s);
  dot_part(f, f, N, W.pb, s);
  { k_cg_init<<<1, 32, 0, s>>>(W.pa, part_grid(N), W.pb, part_grid(N), W.st); ::h2mg::count_launch(); }
  H2_LAUNCH_CHECK();
  for (int it = 0; it < n; ++it) {
    const int par = it & 1;
    apply_level(M, i, f32, W.cp, W.cq, s);
    dot_part(W.cp, W.cq, N, W.pa, s);
    { k_cg_update<<<part_grid(N), 256, 0, s>>>(x, rr, W.cp, W.cq, N, W.st, W.pa, part_grid(N), par, W.pb); ::h2mg::count_launch(); }
    H2_LAUNCH_CHECK();
    { k_cg_p<<<g, 256, 0, s>>>(W.cp, rr, N, W.st, W.pb, part_grid(N), par); ::h2mg::count_launch(); }
    H2_LAUNCH_CHECK();
  }
}

void restrict_level(Matrix& M, int i, const double* v, double* out, cudaStream_t s) {
  const int KC = M.KC, KD = M.KD, L = M.L;
  if (i == 1) {
    { k_restrict_leaf<<<1 << L, std::max(KC, 32), 0, s>>>(M.d_UT, KD, KC, v, M.d_leafoff, M.d_perm, out); ::h2mg::count_launch(); }
  } else {
    int m = L - i + 2;
    { k_restrict<<<1 << (m - 1), std::max(KC, 32), 0, s>>>(M.d_ET + (size_t)M.slot0(m) * KC * KC, KC, v, out); ::h2mg::count_launch(); }
  }
  H2_LAUNCH_CHECK();
}

void prolong_add(Matrix& M, int i, const double* e, double* out, cudaStream_t s) {
  const int KC = M.KC, KD = M.KD, L = M.L;
  if (i == 1) {
    { k_prolong_leaf<<<1 << L, std::max(KD, 32), 0, s>>>(M.d_U, KD, KC, e, M.d_leafoff, M.d_perm, out); ::h2mg::count_launch(); }
  } else {
    int m = L - i + 2;
    { k_prolong<<<1 << m, std::max(KC, 32), 0, s>>>(M.d_E + (size_t)M.slot0(m) * KC * KC, KC, e, out); ::h2mg::count_launch(); }
  }
  H2_LAUNCH_CHECK();
}

// One V-cycle of Algorithm 1: x_out = x0 + e_1 given r1 = b - A x0.
void vcycle(Matrix& M, const h2mg_solve_opts& o, const double* x0, const double* r1, double* xout,
            cudaStream_t s) {
  Work W = work(M);
  const bool f32 = o.precision == H2MG_PREC_MIXED_F32;
  const int l = M.lev;
  int64_t n1 = M.n;
  if (l == 1) {
    coarse_solve(M, r1, W.et[1], s);
  } else {
    const double* ri = r1;
    for (int i = 1; i < l; ++i) {
      int ni = (i == 1) ? o.n_f : o.n_c;
      int64_t N = level_size(M, i);
      smooth(M, i, f32, ri, nullptr, ni, W.et[i], W.cr, s);        // e~_i = Iter(A_i, r_i, 0)
      const double* res = W.cr;                                      // r_i - A_i e~_i (recurrence)
      if (o.explicit_restrict_residual) {
        apply_level(M, i, f32, W.et[i], W.cq, s);
        { k_sub<<<vec_grid(N), 256, 0, s>>>(ri, W.cq, W.cr, N); ::h2mg::count_launch(); }
        H2_LAUNCH_CHECK();
      }
      restrict_level(M, i, res, W.r[i + 1], s);                      // r_{i+1} = U_i^T (...)
      if (i > 1) {
        // keep r_i: the up-sweep smooths against it again
      }
      ri = W.r[i + 1];
      if (i == 1) {
        // r_1 is the caller's buffer; nothing to copy
      }
    }
    coarse_solve(M, W.r[l], W.et[l], s);                             // e_l = dir_sol(A_l, r_l)
    for (int i = l - 1; i >= 1; --i) {
      int ni = (i == 1) ? o.n_f : o.n_c;
      prolong_add(M, i, W.et[i + 1], W.et[i], s);                    // e~_i += V_i^T e_{i+1}
      const double* fi = (i == 1) ? r1 : W.r[i];
      smooth(M, i, f32, fi, W.et[i], ni, W.et[i], nullptr, s);       // e_i = Iter(A_i, r_i, e~_i)
    }
  }
  { k_add<<<vec_grid(n1), 256, 0, s>>>(x0, W.et[1], xout, n1); ::h2mg::count_launch(); }         // x* = x0 + e_1
  H2_LAUNCH_CHECK();
}

static double norm2(Matrix& M, const double* v, int64_t n, cudaStream_t s) {
  Work W = work(M);
  dot_part(v, v, n, W.pa, s);
  std::vector<double> h(part_grid(n));
  H2_CUDA(cudaMemcpyAsync(h.data(), W.pa, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, s));
  H2_CUDA(cudaStreamSynchronize(s));
  double t = 0.0;
  for (double x : h) t += x;
  return std::sqrt(t);
}

// x^T y on the device (two-pass deterministic sum), read back to the host.
double device_dot(const double* a, const double* b, int64_t n, cudaStream_t s) {
  if (n == 0) return 0.0;
  double* part = nullptr;
  H2_CUDA(cudaMalloc(&part, sizeof(double) * NPART));
  double t = 0.0;
  try {
    dot_part(a, b, n, part, s);
    std::vector<double> h(part_grid(n));
    H2_CUDA(cudaMemcpyAsync(h.data(), part, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, s));
    H2_CUDA(cudaStreamSynchronize(s));
    for (double v : h) t += v;
  } catch (...) {
    cudaFree(part);
    throw;
  }
  cudaFree(part);
  return t;
}

static double dot_host(Matrix& M, const double* a, const double* b, int64_t n, cudaStream_t s) {
  Work W = work(M);
  dot_part(a, b, n, W.pa, s);
  std::vector<double> h(part_grid(n));
  H2_CUDA(cudaMemcpyAsync(h.data(), W.pa, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, s));
  H2_CUDA(cudaStreamSynchronize(s));
  double t = 0.0;
  for (double v : h) t += v;
  return t;
}

// Outer iteration: repeated V-cycles x <- x + V(b - A x) (Sec. 3.3), or flexible CG
// preconditioned by one V-cycle (the new direction is made A-orthogonal to the
// previous one because the V-cycle with CG smoothers is a nonlinear map). The
// residual b - A x is recomputed in float64 before every cycle.
h2mg_status solve(Matrix& M, const double* b, double* x, const h2mg_solve_opts& o, h2mg_solve_info* info,
                  cudaStream_t s) {
  Work W = work(M);
  const int64_t n = M.n;
  auto t0 = std::chrono::steady_clock::now();
  double nb = norm2(M, b, n, s);
  H2_REQUIRE(std::isfinite(nb), H2MG_ERR_NAN, "right-hand side is not finite");
  h2mg_solve_info loc{};
  h2mg_status st = H2MG_ERR_NOT_CONVERGED;
  double* r = W.t1;
  const bool fcg = o.outer == H2MG_OUTER_FCG;
  double* z = nullptr;
  double *p = nullptr, *q = nullptr, *pp = nullptr, *qp = nullptr;
  if (fcg) {
    if (!M.wfcg.p) {
      M.wfcg.bytes = sizeof(double) * 5 * (size_t)n;
      M.wfcg.p = M.alloc(M.wfcg.bytes);
    }
    z = (double*)M.wfcg.p;
    p = z + n;
    q = p + n;
    pp = q + n;
    qp = pp + n;
  }
  int g = vec_grid(n);
  for (int cyc = 0; cyc <= o.max_cycles; ++cyc) {
    apply_level(M, 1, false, x, W.t2, s);
    { k_sub<<<g, 256, 0, s>>>(b, W.t2, r, n); ::h2mg::count_launch(); }
    H2_LAUNCH_CHECK();
    double rel = nb > 0 ? norm2(M, r, n, s) / nb : 0.0;
    if (cyc < 256) loc.relres_hist[cyc] = rel;
    loc.cycles = cyc;
    loc.relres = rel;
    if (!std::isfinite(rel)) {
      st = H2MG_ERR_NAN;
      break;
    }
    if (rel <= o.tol) {
      st = H2MG_OK;
      loc.converged = 1;
      break;
    }
    if (cyc == o.max_cycles) break;
    if (!fcg) {
      vcycle(M, o, x, r, x, s);
      continue;
    }
    H2_CUDA(cudaMemsetAsync(z, 0, sizeof(double) * n, s));
    vcycle(M, o, z, r, z, s);                                   // z = V(r) from zero
    if (cyc == 0) {
      H2_CUDA(cudaMemcpyAsync(p, z, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    } else {
      double beta = -dot_host(M, z, qp, n, s) / dot_host(M, pp, qp, n, s);
      H2_CUDA(cudaMemcpyAsync(p, z, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
      { k_axpby<<<g, 256, 0, s>>>(beta, pp, 1.0, p, n); ::h2mg::count_launch(); }           // p = z + beta p_prev
      H2_LAUNCH_CHECK();
    }
    apply_level(M, 1, false, p, q, s);
    double alpha = dot_host(M, p, r, n, s) / dot_host(M, p, q, n, s);
    { k_axpby<<<g, 256, 0, s>>>(alpha, p, 1.0, x, n); ::h2mg::count_launch(); }             // x += alpha p
    H2_LAUNCH_CHECK();
    std::swap(p, pp);
    std::swap(q, qp);
  }
  H2_CUDA(cudaStreamSynchronize(s));
  loc.ms_solve = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (info) *info = loc;
  return st;
}

}  // namespace h2mg
