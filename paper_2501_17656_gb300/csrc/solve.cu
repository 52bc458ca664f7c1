// solve.cu -- the smoother Iter(A_i, f, x0) (textbook CG), restriction U_i^T and
// prolongation V_i^T = U_i, one V-cycle of Algorithm 1 and the outer iteration
// (Sec. 3.3). All multigrid vectors are float64 on the device, column-major with
// leading dimension N_i; up to NRMAX right-hand sides go through every step together
// (one product launch per step reads each stored block once for all of them), each
// with its own CG scalars kept in device memory, so a V-cycle never waits for the host.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <mutex>

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

// part[col * NPART + block] = partial of a_col^T b_col (column = blockIdx.y)
__global__ void k_dot_part(const double* __restrict__ a, const double* __restrict__ b, int64_t n, int64_t ld,
                           double* __restrict__ part) {
  const double* ac = a + blockIdx.y * ld;
  const double* bc = b + blockIdx.y * ld;
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    s = fma(ac[i], bc[i], s);
  s = block_reduce_sum(s);
  if (threadIdx.x == 0) part[blockIdx.y * NPART + blockIdx.x] = s;
}

__device__ double sum_parts(const double* part, int np) {
  double s = 0.0;
  for (int i = 0; i < np; ++i) s += part[i];
  return s;
}

static int part_grid(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>(NPART, (n + 1023) / 1024)); }

// per column (thread c): rho = r.r, thresh = (1e-30 |f|)^2
__global__ void k_cg_init(const double* __restrict__ prr, const double* __restrict__ pff, int np, int nr,
                          CGState* st) {
  const int c = threadIdx.x;
  if (c >= nr) return;
  double rr = sum_parts(prr + c * NPART, np), ff = sum_parts(pff + c * NPART, np);
  double t = 1e-30 * sqrt(ff);
  st[c].rho[0] = rr;
  st[c].thresh = t * t;
  st[c].stopped = 0;
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
// r -= alpha q; partials of r^T r. Every CTA of a column (blockIdx.y) takes the same
// decision from the same partials.
__global__ void __launch_bounds__(256) k_cg_update(double* __restrict__ x, double* __restrict__ r,
                                                   const double* __restrict__ p, const double* __restrict__ q,
                                                   int64_t n, int64_t ld, CGState* st,
                                                   const double* __restrict__ ppq, int np, int par,
                                                   double* __restrict__ part) {
  const int c = blockIdx.y;
  x += c * ld;
  r += c * ld;
  p += c * ld;
  q += c * ld;
  const double pq = cta_sum_parts(ppq + c * NPART, np);
  bool go = !st[c].stopped;
  if (go && !(pq > 0.0)) {
    go = false;
    if (blockIdx.x == 0 && threadIdx.x == 0) st[c].stopped = 1;
  }
  const double al = go ? st[c].rho[par] / pq : 0.0;
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
  if (threadIdx.x == 0) part[c * NPART + blockIdx.x] = s;
}

// rho' = r^T r; stop (after the update) if rho' <= thresh; else p = r + (rho'/rho) p.
__global__ void __launch_bounds__(256) k_cg_p(double* __restrict__ p, const double* __restrict__ r, int64_t n,
                                              int64_t ld, CGState* st, const double* __restrict__ prr, int np,
                                              int par) {
  const int c = blockIdx.y;
  p += c * ld;
  r += c * ld;
  const double rn = cta_sum_parts(prr + c * NPART, np);
  if (st[c].stopped) return;
  if (rn <= st[c].thresh) {
    if (blockIdx.x == 0 && threadIdx.x == 0) st[c].stopped = 1;
    return;
  }
  const double be = rn / st[c].rho[par];
  if (blockIdx.x == 0 && threadIdx.x == 0) st[c].rho[par ^ 1] = rn;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = fma(be, p[i], r[i]);
}

// y_c += a[c] x_c for every column c = blockIdx.y (a in device memory)
__global__ void k_axpy_cols(const double* __restrict__ a, const double* __restrict__ x, double* __restrict__ y,
                            int64_t n, int64_t ld) {
  const int c = blockIdx.y;
  const double al = a[c];
  x += c * ld;
  y += c * ld;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = fma(al, x[i], y[i]);
}
// y_c = x_c + b[c] y_c for every column c = blockIdx.y (b in device memory)
__global__ void k_xpby_cols(const double* __restrict__ b, const double* __restrict__ x, double* __restrict__ y,
                            int64_t n, int64_t ld) {
  const int c = blockIdx.y;
  const double be = b[c];
  x += c * ld;
  y += c * ld;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = fma(be, y[i], x[i]);
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
// Column blockIdx.y of each: input leading dimension ldv / lde, output ldo / ldv.
// out[j*KC + b] = sum_i U_j[i, b] v[perm[leafoff[j] + i]]
__global__ void k_restrict_leaf(const double* __restrict__ UT, int KD, int KC, const double* __restrict__ v,
                                int64_t ldv, const int* __restrict__ leafoff, const int* __restrict__ perm,
                                double* __restrict__ out, int64_t ldo) {
  __shared__ double xs[64];
  v += blockIdx.y * ldv;
  out += blockIdx.y * ldo;
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
                               int64_t lde, const int* __restrict__ leafoff, const int* __restrict__ perm,
                               double* __restrict__ v, int64_t ldv) {
  __shared__ double es[64];
  e += blockIdx.y * lde;
  v += blockIdx.y * ldv;
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
__global__ void k_restrict(const double* __restrict__ ET, int KC, const double* __restrict__ v, int64_t ldv,
                           double* __restrict__ out, int64_t ldo) {
  __shared__ double xs[128];
  v += blockIdx.y * ldv;
  out += blockIdx.y * ldo;
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
__global__ void k_prolong(const double* __restrict__ E, int KC, const double* __restrict__ e, int64_t lde,
                          double* __restrict__ v, int64_t ldv) {
  __shared__ double es[64];
  e += blockIdx.y * lde;
  v += blockIdx.y * ldv;
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
  double *pa, *pb, *scal;
  CGState* st;
};

// Multigrid workspaces for NRMAX columns, allocated on first use.
static Work work(Matrix& M) {
  Work W{};
  size_t tot = 0, nmax = 0;
  for (int i = 1; i <= M.lev; ++i) {
    tot += 2 * (size_t)level_size(M, i);
    nmax = std::max(nmax, (size_t)level_size(M, i));
  }
  tot += 5 * nmax;
  if (!M.wvec.p) {
    M.wvec.bytes = sizeof(double) * tot * NRMAX;
    M.wvec.p = M.alloc(M.wvec.bytes);
    M.wred.bytes = sizeof(double) * (2 * NPART + 8) * NRMAX + sizeof(CGState) * NRMAX + 64;
    M.wred.p = M.alloc(M.wred.bytes);
    M.wfcg.bytes = sizeof(double) * 4 * (size_t)M.n * NRMAX;   // flexible-CG directions
    M.wfcg.p = M.alloc(M.wfcg.bytes);
  }
  double* p = (double*)M.wvec.p;
  for (int i = 1; i <= M.lev; ++i) {
    W.r[i] = p;
    p += level_size(M, i) * NRMAX;
    W.et[i] = p;
    p += level_size(M, i) * NRMAX;
  }
  W.cr = p; p += nmax * NRMAX;
  W.cp = p; p += nmax * NRMAX;
  W.cq = p; p += nmax * NRMAX;
  W.t1 = p; p += nmax * NRMAX;
  W.t2 = p; p += nmax * NRMAX;
  W.pa = (double*)M.wred.p;
  W.pb = W.pa + NPART * NRMAX;
  W.scal = W.pb + NPART * NRMAX;
  W.st = (CGState*)(W.scal + 8 * NRMAX);
  return W;
}

// Allocated with the matrix, so that solves on any stream find them ready.
void alloc_solve_workspace(Matrix& M) { work(M); }

static void dot_part(const double* a, const double* b, int64_t n, int64_t ld, int nr, double* part,
                     cudaStream_t s) {
  { k_dot_part<<<dim3(part_grid(n), nr), 256, 0, s>>>(a, b, n, ld, part); ::h2mg::count_launch(); }
  H2_LAUNCH_CHECK();
}

// n CG iterations on A_i X = F from X0 (nullptr: zero) for nr columns of length N_i.
// X receives the iterates; R (if not null) the recurrence residuals. Hestenes-Stiefel
// with, per column, the breakdown guard p^T A p <= 0 and the stop r^T r <= (1e-30 |f|)^2.
void smooth_multi(Matrix& M, int i, bool f32, const double* f, const double* x0, int n, double* x, double* r,
                  int nr, cudaStream_t s) {
  H2_REQUIRE(nr >= 1 && nr <= NRMAX, H2MG_ERR_INVALID_ARG, "too many columns for one smoother call");
  Work W = work(M);
  const int64_t N = level_size(M, i), tot = N * nr;
  double* rr = r ? r : W.cr;
  const int g = vec_grid(N), np = part_grid(N);
  if (n == 0 && x0 != nullptr && r == nullptr) {   // no iteration, residual not wanted
    if (x != x0) H2_CUDA(cudaMemcpyAsync(x, x0, sizeof(double) * tot, cudaMemcpyDeviceToDevice, s));
    return;
  }
  if (x0 == nullptr) {
    H2_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * tot, s));
    H2_CUDA(cudaMemcpyAsync(rr, f, sizeof(double) * tot, cudaMemcpyDeviceToDevice, s));
    if (n == 0) return;
  } else {
    if (x != x0) H2_CUDA(cudaMemcpyAsync(x, x0, sizeof(double) * tot, cudaMemcpyDeviceToDevice, s));
    apply_level_multi(M, i, f32, x, N, W.cq, N, nr, s);
    { k_sub<<<vec_grid(tot), 256, 0, s>>>(f, W.cq, rr, tot); ::h2mg::count_launch(); }
    H2_LAUNCH_CHECK();
  }
  H2_CUDA(cudaMemcpyAsync(W.cp, rr, sizeof(double) * tot, cudaMemcpyDeviceToDevice, s));
  dot_part(rr, rr, N, N, nr, W.pa, s);
  dot_part(f, f, N, N, nr, W.pb, s);
  { k_cg_init<<<1, 32, 0, s>>>(W.pa, W.pb, np, nr, W.st); ::h2mg::count_launch(); }
  H2_LAUNCH_CHECK();
  for (int it = 0; it < n; ++it) {
    const int par = it & 1;
    apply_level_multi(M, i, f32, W.cp, N, W.cq, N, nr, s);
    dot_part(W.cp, W.cq, N, N, nr, W.pa, s);
    { k_cg_update<<<dim3(np, nr), 256, 0, s>>>(x, rr, W.cp, W.cq, N, N, W.st, W.pa, np, par, W.pb); ::h2mg::count_launch(); }
    H2_LAUNCH_CHECK();
    { k_cg_p<<<dim3(g, nr), 256, 0, s>>>(W.cp, rr, N, N, W.st, W.pb, np, par); ::h2mg::count_launch(); }
    H2_LAUNCH_CHECK();
  }
}

void smooth(Matrix& M, int i, bool f32, const double* f, const double* x0, int n, double* x, double* r,
            cudaStream_t s) {
  smooth_multi(M, i, f32, f, x0, n, x, r, 1, s);
}

static void restrict_multi(Matrix& M, int i, const double* v, double* out, int nr, cudaStream_t s) {
  const int KC = M.KC, KD = M.KD, L = M.L;
  const int64_t nf = level_size(M, i), nc = level_size(M, i + 1);
  if (i == 1) {
    { k_restrict_leaf<<<dim3(1 << L, nr), std::max(KC, 32), 0, s>>>(M.d_UT, KD, KC, v, nf, M.d_leafoff, M.d_perm,
                                                                    out, nc); ::h2mg::count_launch(); }
  } else {
    int m = L - i + 2;
    { k_restrict<<<dim3(1 << (m - 1), nr), std::max(KC, 32), 0, s>>>(M.d_ET + (size_t)M.slot0(m) * KC * KC, KC, v,
                                                                     nf, out, nc); ::h2mg::count_launch(); }
  }
  H2_LAUNCH_CHECK();
}

static void prolong_add_multi(Matrix& M, int i, const double* e, double* out, int nr, cudaStream_t s) {
  const int KC = M.KC, KD = M.KD, L = M.L;
  const int64_t nf = level_size(M, i), nc = level_size(M, i + 1);
  if (i == 1) {
    { k_prolong_leaf<<<dim3(1 << L, nr), std::max(KD, 32), 0, s>>>(M.d_U, KD, KC, e, nc, M.d_leafoff, M.d_perm,
                                                                   out, nf); ::h2mg::count_launch(); }
  } else {
    int m = L - i + 2;
    { k_prolong<<<dim3(1 << m, nr), std::max(KC, 32), 0, s>>>(M.d_E + (size_t)M.slot0(m) * KC * KC, KC, e, nc,
                                                              out, nf); ::h2mg::count_launch(); }
  }
  H2_LAUNCH_CHECK();
}

void restrict_level(Matrix& M, int i, const double* v, double* out, cudaStream_t s) {
  restrict_multi(M, i, v, out, 1, s);
}
void prolong_add(Matrix& M, int i, const double* e, double* out, cudaStream_t s) {
  prolong_add_multi(M, i, e, out, 1, s);
}

// True if the restriction U_{i-1} into level i >= 2 is square: every cluster of tree
// level m(i) has as many basis columns as rows (points for leaves, the children's
// ranks above), so A_i = U_{i-1}^T A_{i-1} U_{i-1} is an orthogonal similarity.
static bool square_level(const Matrix& M, int i) {
  if (i < 2 || M.tstar < 0) return false;
  const int m = M.L - i + 2;
  if (m < M.tstar || m > M.L) return false;
  for (int c = 0; c < (1 << m); ++c) {
    const int rank = M.h_rank[M.slot0(m) + c];
    int rows;
    if (m == M.L) {
      rows = M.offsets[M.L][c + 1] - M.offsets[M.L][c];
    } else {
      if (m + 1 > M.L) return false;
      rows = M.h_rank[M.slot0(m + 1) + 2 * c] + M.h_rank[M.slot0(m + 1) + 2 * c + 1];
    }
    if (rank != rows) return false;
  }
  return true;
}

// One visit of level i in a multigrid cycle of type `kind` on A_i e = f (nr columns,
// leading dimension N_i), into W.et[i]; the first visit starts from zero, later ones
// from W.et[i] as the previous visit left it. Level l solves directly. Otherwise:
// pre-smoothing e~ = Iter(A_i, f, start); r_{i+1} = U_i^T (f - A_i e~) (CG's recurrence
// residual, or an explicit product); the coarser level is visited once (V: this is
// Algorithm 1), twice (W), or F-then-V (F), each visit from the previous one's
// result; e~ += V_i^T e_{i+1}; post-smoothing e = Iter(A_i, f, e~).
static void cycle_visit(Matrix& M, const h2mg_solve_opts& o, int i, const double* f, bool from_zero, int kind,
                        int nr, cudaStream_t s) {
  Work W = work(M);
  const bool f32 = o.precision == H2MG_PREC_MIXED_F32;
  const int l = M.lev;
  if (i == l) {
    coarse_solve_multi(M, f, W.et[l], nr, s);                        // e_l = dir_sol(A_l, r_l)
    return;
  }
  const int ni = (i == 1) ? o.n_f : ((o.skip_square_levels && square_level(M, i)) ? 0 : o.n_c);
  const int64_t N = level_size(M, i);
  smooth_multi(M, i, f32, f, from_zero ? nullptr : W.et[i], ni, W.et[i], W.cr, nr, s);   // e~_i = Iter(A_i, r_i, .)
  if (o.explicit_restrict_residual) {                                // r_i - A_i e~_i, explicitly
    apply_level_multi(M, i, f32, W.et[i], N, W.cq, N, nr, s);
    { k_sub<<<vec_grid(N * nr), 256, 0, s>>>(f, W.cq, W.cr, N * nr); ::h2mg::count_launch(); }
    H2_LAUNCH_CHECK();
  }
  restrict_multi(M, i, W.cr, W.r[i + 1], nr, s);                     // r_{i+1} = U_i^T (r_i - A_i e~_i)
  const int kids[3][2] = {{H2MG_CYCLE_V, -1}, {H2MG_CYCLE_W, H2MG_CYCLE_W}, {H2MG_CYCLE_F, H2MG_CYCLE_V}};
  for (int k = 0; k < 2 && kids[kind][k] >= 0; ++k) cycle_visit(M, o, i + 1, W.r[i + 1], k == 0, kids[kind][k], nr, s);
  prolong_add_multi(M, i, W.et[i + 1], W.et[i], nr, s);              // e~_i += V_i^T e_{i+1}
  smooth_multi(M, i, f32, f, W.et[i], ni, W.et[i], nullptr, nr, s);  // e_i = Iter(A_i, r_i, e~_i)
}

// e_1 of one multigrid cycle (o.cycle; the V-cycle is Algorithm 1) for nr columns of
// r_1 (n x nr, leading dimension n), into the level-1 error buffer W.et[1]. No host
// synchronisation and no allocation: the sequence can be captured into a CUDA graph.
static void vcycle_core(Matrix& M, const h2mg_solve_opts& o, const double* r1, int nr, cudaStream_t s) {
  H2_REQUIRE(nr >= 1 && nr <= NRMAX, H2MG_ERR_INVALID_ARG, "too many columns for one V-cycle");
  H2_REQUIRE(o.cycle >= H2MG_CYCLE_V && o.cycle <= H2MG_CYCLE_F, H2MG_ERR_INVALID_ARG, "unknown cycle type");
  cycle_visit(M, o, 1, r1, true, o.cycle, nr, s);
}

// One V-cycle for nr columns: x_out = x0 + e_1 given r1 = b - A x0 (x0, r1 and x_out
// are n x nr with leading dimension n; x_out may be x0).
void vcycle_multi(Matrix& M, const h2mg_solve_opts& o, const double* x0, const double* r1, double* xout, int nr,
                  cudaStream_t s) {
  Work W = work(M);
  vcycle_core(M, o, r1, nr, s);
  const int64_t n1 = M.n;
  { k_add<<<vec_grid(n1 * nr), 256, 0, s>>>(x0, W.et[1], xout, n1 * nr); ::h2mg::count_launch(); }   // x* = x0 + e_1
  H2_LAUNCH_CHECK();
}

void vcycle(Matrix& M, const h2mg_solve_opts& o, const double* x0, const double* r1, double* xout, cudaStream_t s) {
  vcycle_multi(M, o, x0, r1, xout, 1, s);
}

// ----------------------------------------------------------------------------- graphs
// A V-cycle (vcycle_core on the solve's residual buffer) captured once per solve
// setting and column count; replayed with one launch per outer iteration, or used as
// one branch of a graph over several independent problems.
struct GraphEntry {
  int nr, n_f, n_c, f32, err, skip, prof, cyc;
  cudaGraph_t graph = nullptr;        // the captured sequence
  cudaGraphExec_t exec = nullptr;     // instantiated on first replay
  int64_t launches = 0;               // kernels per replay
  std::vector<cudaEvent_t> ev;        // profiled graphs: (start, stop) around each block product
  std::vector<double> bytes;          // and its algorithmic bytes
};
struct GraphSet {
  std::vector<GraphEntry> g;
  int pending = -1;                   // profiled entry replayed since the last collection
};

void destroy_graphs(Matrix& M) {
  if (M.graphs) {
    for (auto& e : M.graphs->g) {
      if (e.exec) best_effort(cudaGraphExecDestroy(e.exec), "cudaGraphExecDestroy");
      if (e.graph) best_effort(cudaGraphDestroy(e.graph), "cudaGraphDestroy");
      for (auto v : e.ev) best_effort(cudaEventDestroy(v), "cudaEventDestroy (graph)");
    }
    delete M.graphs;
    M.graphs = nullptr;
  }
  if (M.cap_stream) {
    best_effort(cudaStreamDestroy(M.cap_stream), "cudaStreamDestroy (capture)");
    M.cap_stream = nullptr;
  }
}

// Block products of one cycle, from above (event pairs of a profiled graph): level i
// is visited once per V-cycle, 2^(i-1) times per W-cycle and i times per F-cycle.
static size_t products_bound(const Matrix& M, const h2mg_solve_opts& o, int nr) {
  size_t applies = 0;
  for (int i = 1; i < M.lev; ++i) {
    const size_t visits = o.cycle == H2MG_CYCLE_W ? ((size_t)1 << std::min(i - 1, 40))
                          : o.cycle == H2MG_CYCLE_F ? (size_t)i : 1;
    applies += visits * (2 * (size_t)((i == 1) ? o.n_f : o.n_c) + 3);
  }
  return applies * 2 * (size_t)nr;   // at most two products per column group, nr groups
}

// The captured V-cycle for these settings (with event nodes around every block
// product when `prof`), captured on first use. Returns its index.
static int vcycle_graph(Matrix& M, const h2mg_solve_opts& o, int nr, int prof) {
  if (!M.graphs) M.graphs = new GraphSet();
  const int f32 = o.precision == H2MG_PREC_MIXED_F32;
  for (size_t k = 0; k < M.graphs->g.size(); ++k) {
    const GraphEntry& e = M.graphs->g[k];
    if (e.nr == nr && e.n_f == o.n_f && e.n_c == o.n_c && e.f32 == f32 && e.err == o.explicit_restrict_residual &&
        e.skip == o.skip_square_levels && e.prof == prof && e.cyc == o.cycle)
      return (int)k;
  }
  if (!M.cap_stream) H2_CUDA(cudaStreamCreateWithFlags(&M.cap_stream, cudaStreamNonBlocking));
  Work W = work(M);
  GraphEntry e{nr, o.n_f, o.n_c, f32, o.explicit_restrict_residual, o.skip_square_levels, prof, o.cycle};
  auto drop_events = [&](size_t from) {
    for (size_t k = from; k < e.ev.size(); ++k) best_effort(cudaEventDestroy(e.ev[k]), "cudaEventDestroy (graph)");
    e.ev.resize(std::min(from, e.ev.size()));
  };
  Profile& P = M.prof;
  if (prof) {
    // created before the capture: only their records are captured
    const size_t pairs = products_bound(M, o, nr);
    e.ev.reserve(2 * pairs);
    for (size_t k = 0; k < 2 * pairs; ++k) {
      cudaEvent_t v;
      const cudaError_t err = cudaEventCreate(&v);
      if (err != cudaSuccess) {
        drop_events(0);
        H2_CUDA(err);
      }
      e.ev.push_back(v);
    }
  }
  const int64_t l0 = h2mg_launch_count();
  H2_CUDA(cudaStreamBeginCapture(M.cap_stream, cudaStreamCaptureModeThreadLocal));
  if (prof) {
    P.cap_ev = &e.ev;
    P.cap_bytes = &e.bytes;
    P.cap_next = 0;
  }
  try {
    vcycle_core(M, o, W.t1, nr, M.cap_stream);
  } catch (...) {
    P.cap_ev = nullptr;
    P.cap_bytes = nullptr;
    cudaGraph_t g = nullptr;
    best_effort(cudaStreamEndCapture(M.cap_stream, &g), "cudaStreamEndCapture (after an error)");
    if (g) best_effort(cudaGraphDestroy(g), "cudaGraphDestroy (after an error)");
    drop_events(0);
    add_launches(l0 - h2mg_launch_count());
    throw;
  }
  const size_t used = 2 * P.cap_next;
  P.cap_ev = nullptr;
  P.cap_bytes = nullptr;
  e.launches = h2mg_launch_count() - l0;
  add_launches(-e.launches);   // captured, not run
  const cudaError_t err = cudaStreamEndCapture(M.cap_stream, &e.graph);
  if (err != cudaSuccess) {
    drop_events(0);
    H2_CUDA(err);
  }
  drop_events(used);
  M.graphs->g.push_back(std::move(e));
  return (int)M.graphs->g.size() - 1;
}

// Adds the block-product times of the last profiled replay (finished by now: called
// after a stream synchronisation) to the profile.
static void graph_collect(Matrix& M) {
  if (!M.graphs || M.graphs->pending < 0) return;
  const GraphEntry& e = M.graphs->g[M.graphs->pending];
  M.graphs->pending = -1;
  for (size_t k = 0; k + 1 < e.ev.size(); k += 2) {
    float f = 0.f;
    H2_CUDA(cudaEventElapsedTime(&f, e.ev[k], e.ev[k + 1]));
    M.prof.g_ms += f;
    M.prof.g_bytes += e.bytes[k / 2];
    M.prof.g_launches++;
  }
}

// e_1 of one V-cycle from the solve's residual buffer W.t1 into W.et[1]: replayed
// from a captured graph when the options ask for it (while h2mg_profile is on, the
// graph carries event nodes around its block products), else launched directly.
static void vcycle_solve_step(Matrix& M, const h2mg_solve_opts& o, int nr, cudaStream_t s) {
  Work W = work(M);
  if (!o.use_graph) {
    vcycle_core(M, o, W.t1, nr, s);
    return;
  }
  graph_collect(M);
  const int k = vcycle_graph(M, o, nr, M.prof.on ? (M.prof.f32_only ? 2 : 1) : 0);
  GraphEntry& e = M.graphs->g[k];
  if (!e.exec) H2_CUDA(cudaGraphInstantiate(&e.exec, e.graph, 0));
  H2_CUDA(cudaGraphLaunch(e.exec, s));
  add_launches(e.launches);
  if (e.prof) M.graphs->pending = k;
}

// out[c] = sum of the np partials of column c (blockIdx.x), in a fixed order.
__global__ void __launch_bounds__(256) k_sum_parts(const double* __restrict__ part, int np,
                                                   double* __restrict__ out) {
  const double t = cta_sum_parts(part + blockIdx.x * NPART, np);
  if (threadIdx.x == 0) out[blockIdx.x] = t;
}

// Partials and result of h2mg_dot, per device: allocated on the first call on that
// device and kept until the process exits (each call synchronises before returning,
// so calls from one thread never overlap; a mutex serialises threads).
static std::mutex g_dot_mu;
static double* g_dot_ws[128] = {nullptr};

// x^T y on the device (partials, then their fixed-order sum), read back to the host.
double device_dot(const double* a, const double* b, int64_t n, cudaStream_t s) {
  if (n == 0) return 0.0;
  int dev = 0;
  H2_CUDA(cudaGetDevice(&dev));
  H2_REQUIRE(dev >= 0 && dev < 128, H2MG_ERR_UNSUPPORTED, "device ordinal out of range");
  std::lock_guard<std::mutex> lk(g_dot_mu);
  if (!g_dot_ws[dev]) H2_CUDA(cudaMalloc(&g_dot_ws[dev], sizeof(double) * (NPART + 32)));
  double* part = g_dot_ws[dev];
  dot_part(a, b, n, n, 1, part, s);
  { k_sum_parts<<<1, 256, 0, s>>>(part, part_grid(n), part + NPART); ::h2mg::count_launch(); }
  H2_LAUNCH_CHECK();
  double t = 0.0;
  H2_CUDA(cudaMemcpyAsync(&t, part + NPART, sizeof(double), cudaMemcpyDeviceToHost, s));
  H2_CUDA(cudaStreamSynchronize(s));
  return t;
}

// out[c] = a_c^T b_c for nr columns of length n (leading dimension n): partials and
// their sums on the device, the nr results read back.
static void dots_host(Matrix& M, const double* a, const double* b, int64_t n, int nr, double* out, cudaStream_t s) {
  Work W = work(M);
  dot_part(a, b, n, n, nr, W.pa, s);
  { k_sum_parts<<<nr, 256, 0, s>>>(W.pa, part_grid(n), W.scal + 4 * NRMAX); ::h2mg::count_launch(); }
  H2_LAUNCH_CHECK();
  H2_CUDA(cudaMemcpyAsync(out, W.scal + 4 * NRMAX, sizeof(double) * nr, cudaMemcpyDeviceToHost, s));
  H2_CUDA(cudaStreamSynchronize(s));
}

// The same, for callers outside this file.
void dots(Matrix& M, const double* a, const double* b, int64_t n, int nr, double* out, cudaStream_t s) {
  dots_host(M, a, b, n, nr, out, s);
}

// y_c += alpha[c] x_c with the coefficients from the host.
static void axpy_cols(Matrix& M, const double* alpha, const double* x, double* y, int64_t n, int nr,
                      cudaStream_t s) {
  Work W = work(M);
  H2_CUDA(cudaMemcpyAsync(W.scal, alpha, sizeof(double) * nr, cudaMemcpyHostToDevice, s));
  { k_axpy_cols<<<dim3(vec_grid(n), nr), 256, 0, s>>>(W.scal, x, y, n, n); ::h2mg::count_launch(); }
  H2_LAUNCH_CHECK();
}

// The float64 outer residual r = b - A x for nr columns: the float64 product, or, with
// o.residual_dd, the product with double-double sums (one launch sequence per column).
// dd[c] (optional) selects the double-double product per column: with residual_dd = 1
// every column, with 2 (automatic) the columns the caller marks; nullptr = none.
static void outer_residual(Matrix& M, const h2mg_solve_opts& o, const double* b, const double* x, double* r,
                           double* tmp, int64_t n, int nr, cudaStream_t s, const bool* dd = nullptr) {
  bool any = false, all = true;
  for (int c = 0; c < nr; ++c) {
    const bool u = M.fmt == FMT_F64 && (o.residual_dd == 1 || (o.residual_dd == 2 && dd && dd[c]));
    any = any || u;
    all = all && u;
  }
  if (!all) apply_level_multi(M, 1, false, x, n, tmp, n, nr, s);
  if (any)
    for (int c = 0; c < nr; ++c)
      if (M.fmt == FMT_F64 && (o.residual_dd == 1 || (o.residual_dd == 2 && dd && dd[c])))
        apply_level1_dd(M, x + c * n, tmp + c * n, s);
  { k_sub<<<vec_grid(n * nr), 256, 0, s>>>(b, tmp, r, n * nr); ::h2mg::count_launch(); }
  H2_LAUNCH_CHECK();
}

// y_c = x_c + beta[c] y_c with the coefficients from the host.
static void xpby_cols(Matrix& M, const double* beta, const double* x, double* y, int64_t n, int nr, cudaStream_t s) {
  Work W = work(M);
  H2_CUDA(cudaMemcpyAsync(W.scal + NRMAX, beta, sizeof(double) * nr, cudaMemcpyHostToDevice, s));
  { k_xpby_cols<<<dim3(vec_grid(n), nr), 256, 0, s>>>(W.scal + NRMAX, x, y, n, n); ::h2mg::count_launch(); }
  H2_LAUNCH_CHECK();
}

// Unpreconditioned CG on A x = b for nr columns, the comparison solver of the paper's
// experiments (Sec. 4): q = A p, alpha = rho / p^T q, x += alpha p, r -= alpha q,
// rho' = r^T r, p = r + (rho'/rho) p, from x's initial guess (r = b - A x). A column
// stops when its recurrence residual |r| / |b| <= tol (or at a breakdown p^T A p <= 0);
// info.cycles counts CG iterations (one product of the primary copy each) and
// info.relres is the explicitly recomputed float64 residual.
static h2mg_status solve_cg_multi(Matrix& M, const double* b, double* x, int nr, const h2mg_solve_opts& o,
                                  h2mg_solve_info* info, cudaStream_t s) {
  Work W = work(M);
  const int64_t n = M.n;
  auto t0 = std::chrono::steady_clock::now();
  double nb[NRMAX], rho[NRMAX], rn[NRMAX], pq[NRMAX], al[NRMAX], be[NRMAX];
  bool done[NRMAX], conv[NRMAX];
  double* r = W.t1;
  double* p = (double*)M.wfcg.p;
  double* q = p + n * NRMAX;
  dots_host(M, b, b, n, nr, nb, s);
  for (int c = 0; c < nr; ++c) {
    H2_REQUIRE(std::isfinite(nb[c]), H2MG_ERR_NAN, "right-hand side is not finite");
    nb[c] = std::sqrt(nb[c]);
    done[c] = conv[c] = false;
    info[c] = h2mg_solve_info{};
  }
  apply_level_multi(M, 1, false, x, n, W.t2, n, nr, s);
  { k_sub<<<vec_grid(n * nr), 256, 0, s>>>(b, W.t2, r, n * nr); ::h2mg::count_launch(); }
  H2_LAUNCH_CHECK();
  H2_CUDA(cudaMemcpyAsync(p, r, sizeof(double) * n * nr, cudaMemcpyDeviceToDevice, s));
  dots_host(M, r, r, n, nr, rho, s);
  bool nan = false;
  for (int it = 0; it <= o.max_cycles; ++it) {
    bool all = true;
    for (int c = 0; c < nr; ++c) {
      if (done[c]) continue;
      const double rel = nb[c] > 0 ? std::sqrt(rho[c]) / nb[c] : 0.0;
      if (it < 256) info[c].relres_hist[it] = rel;
      info[c].cycles = it;
      if (!std::isfinite(rel)) {
        nan = true;
        done[c] = true;
      } else if (rel <= o.tol) {
        conv[c] = true;
        done[c] = true;
      }
      all = all && done[c];
    }
    if (all || nan || it == o.max_cycles) break;
    apply_level_multi(M, 1, false, p, n, q, n, nr, s);
    dots_host(M, p, q, n, nr, pq, s);
    for (int c = 0; c < nr; ++c) {
      if (!done[c] && !(pq[c] > 0.0)) done[c] = true;   // breakdown: stop this column
      al[c] = done[c] ? 0.0 : rho[c] / pq[c];
    }
    axpy_cols(M, al, p, x, n, nr, s);                         // x += alpha p
    for (int c = 0; c < nr; ++c) al[c] = -al[c];
    axpy_cols(M, al, q, r, n, nr, s);                         // r -= alpha q
    dots_host(M, r, r, n, nr, rn, s);
    for (int c = 0; c < nr; ++c) {
      be[c] = done[c] ? 0.0 : rn[c] / rho[c];
      if (!done[c]) rho[c] = rn[c];
    }
    xpby_cols(M, be, r, p, n, nr, s);                         // p = r + beta p
  }
  // the explicit float64 residual of the result
  outer_residual(M, o, b, x, r, W.t2, n, nr, s);
  double rr[NRMAX];
  dots_host(M, r, r, n, nr, rr, s);
  const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  h2mg_status st = H2MG_OK;
  for (int c = 0; c < nr; ++c) {
    info[c].relres = nb[c] > 0 ? std::sqrt(rr[c]) / nb[c] : 0.0;
    info[c].converged = conv[c] ? 1 : 0;
    info[c].ms_solve = ms;
    if (!conv[c]) st = H2MG_ERR_NOT_CONVERGED;
    if (!std::isfinite(info[c].relres)) nan = true;
  }
  if (nan) st = H2MG_ERR_NAN;
  return st;
}

// Outer iteration for nr columns (b, x: n x nr, leading dimension n): repeated
// V-cycles x <- x + V(b - A x) (Sec. 3.3), or flexible CG preconditioned by one
// V-cycle (each new direction is made A-orthogonal to the previous one because the
// V-cycle with CG smoothers is a nonlinear map). The float64 residual b - A x is
// recomputed before every cycle; a column that has met the tolerance keeps its x
// from then on. info[c] receives column c's statistics.
h2mg_status solve_multi(Matrix& M, const double* b, double* x, int nr, const h2mg_solve_opts& o,
                        h2mg_solve_info* info, cudaStream_t s) {
  H2_REQUIRE(nr >= 1 && nr <= NRMAX, H2MG_ERR_INVALID_ARG, "too many columns for one solve");
  if (o.outer == H2MG_OUTER_CG) return solve_cg_multi(M, b, x, nr, o, info, s);
  Work W = work(M);
  const int64_t n = M.n;
  auto t0 = std::chrono::steady_clock::now();
  double nb[NRMAX], rel[NRMAX], alpha[NRMAX], beta[NRMAX], d1[NRMAX], d2[NRMAX];
  bool done[NRMAX];
  dots_host(M, b, b, n, nr, nb, s);
  for (int c = 0; c < nr; ++c) {
    H2_REQUIRE(std::isfinite(nb[c]), H2MG_ERR_NAN, "right-hand side is not finite");
    nb[c] = std::sqrt(nb[c]);
    done[c] = false;
    info[c] = h2mg_solve_info{};
  }
  double* r = W.t1;
  const bool fcg = o.outer == H2MG_OUTER_FCG;
  double *z = nullptr, *p = nullptr, *q = nullptr, *pp = nullptr, *qp = nullptr;
  if (fcg) {
    p = (double*)M.wfcg.p;
    q = p + n * NRMAX;
    pp = q + n * NRMAX;
    qp = pp + n * NRMAX;
  }
  bool nan = false;
  bool near[NRMAX];   // automatic extended residual: switched on for this column
  double best[NRMAX];
  int since[NRMAX];
  for (int c = 0; c < nr; ++c) {
    near[c] = false;
    best[c] = INFINITY;
    since[c] = 0;
  }
  for (int cyc = 0; cyc <= o.max_cycles; ++cyc) {
    outer_residual(M, o, b, x, r, W.t2, n, nr, s, near);
    dots_host(M, r, r, n, nr, rel, s);
    if (o.residual_dd == 2) {
      // A column switches to the extended product once its float64 residual is within
      // 100 tol. A column whose float64 residual has made no new minimum for 5 cycles
      // is probed: its residual is recomputed with the extended product, and if that
      // is below 0.8 of the float64 one, the float64 residual is dominated by the
      // rounding of its sum (the floor, which can lie near or above tol) and the
      // column switches; otherwise the stagnation is the iteration's own and float64
      // stays. Either way this cycle uses the recomputed residual.
      bool redo = false, probe[NRMAX];
      for (int c = 0; c < nr; ++c) {
        probe[c] = false;
        const double rr = nb[c] > 0 ? std::sqrt(rel[c]) / nb[c] : 0.0;
        if (near[c] || done[c] || !std::isfinite(rr)) continue;
        if (rr < best[c]) {
          best[c] = rr;
          since[c] = 0;
        } else {
          ++since[c];
        }
        if (rr <= 100.0 * o.tol)
          near[c] = redo = true;
        else if (since[c] >= 5)
          probe[c] = redo = true;
      }
      if (redo) {
        bool ext[NRMAX];
        for (int c = 0; c < nr; ++c) ext[c] = near[c] || probe[c];
        double reld[NRMAX];
        outer_residual(M, o, b, x, r, W.t2, n, nr, s, ext);
        dots_host(M, r, r, n, nr, reld, s);
        for (int c = 0; c < nr; ++c) {
          if (probe[c]) {
            if (std::sqrt(reld[c]) < 0.8 * std::sqrt(rel[c])) near[c] = true;
            since[c] = 0;
          }
          rel[c] = reld[c];
        }
      }
    }
    graph_collect(M);
    bool all = true;
    for (int c = 0; c < nr; ++c) {
      if (done[c]) continue;
      rel[c] = nb[c] > 0 ? std::sqrt(rel[c]) / nb[c] : 0.0;
      if (cyc < 256) info[c].relres_hist[cyc] = rel[c];
      info[c].cycles = cyc;
      info[c].relres = rel[c];
      if (!std::isfinite(rel[c])) {
        nan = true;
        done[c] = true;
      } else if (rel[c] <= o.tol) {
        info[c].converged = 1;
        done[c] = true;
      }
      all = all && done[c];
    }
    if (all || nan || cyc == o.max_cycles) break;
    vcycle_solve_step(M, o, nr, s);                         // W.et[1] = V(r) from zero
    if (!fcg) {
      // x* = x0 + e_1 (Algorithm 1) for the columns still running
      for (int c = 0; c < nr; ++c) alpha[c] = done[c] ? 0.0 : 1.0;
      axpy_cols(M, alpha, W.et[1], x, n, nr, s);
      continue;
    }
    z = W.et[1];
    H2_CUDA(cudaMemcpyAsync(p, z, sizeof(double) * n * nr, cudaMemcpyDeviceToDevice, s));
    if (cyc > 0) {
      dots_host(M, z, qp, n, nr, d1, s);
      dots_host(M, pp, qp, n, nr, d2, s);
      for (int c = 0; c < nr; ++c) beta[c] = d2[c] != 0.0 ? -d1[c] / d2[c] : 0.0;
      axpy_cols(M, beta, pp, p, n, nr, s);                   // p = z + beta p_prev
    }
    apply_level_multi(M, 1, false, p, n, q, n, nr, s);
    dots_host(M, p, r, n, nr, d1, s);
    dots_host(M, p, q, n, nr, d2, s);
    for (int c = 0; c < nr; ++c) alpha[c] = (!done[c] && d2[c] > 0.0) ? d1[c] / d2[c] : 0.0;
    axpy_cols(M, alpha, p, x, n, nr, s);                     // x += alpha p
    std::swap(p, pp);
    std::swap(q, qp);
  }
  H2_CUDA(cudaStreamSynchronize(s));
  graph_collect(M);
  const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  h2mg_status st = H2MG_OK;
  for (int c = 0; c < nr; ++c) {
    info[c].ms_solve = ms;
    if (!info[c].converged) st = H2MG_ERR_NOT_CONVERGED;
  }
  if (nan) st = H2MG_ERR_NAN;
  return st;
}

// ----------------------------------------------------------------------------- many problems
// Pinned host copies of dot-product partials of several problems, read with one
// synchronisation.
struct HostParts {
  double* h = nullptr;
  explicit HostParts(size_t n) { H2_CUDA(cudaMallocHost(&h, sizeof(double) * n)); }
  ~HostParts() {
    if (h) best_effort(cudaFreeHost(h), "cudaFreeHost");
  }
};

// out[p] = a_p^T b_p for every problem p with want[p], one synchronisation in all.
static void dots_many(const std::vector<Matrix*>& Ms, const std::vector<const double*>& a,
                      const std::vector<const double*>& b, const std::vector<char>& want, HostParts& hp,
                      double* out, cudaStream_t s) {
  const size_t P = Ms.size();
  for (size_t p = 0; p < P; ++p) {
    if (!want[p]) continue;
    Work W = work(*Ms[p]);
    dot_part(a[p], b[p], Ms[p]->n, Ms[p]->n, 1, W.pa, s);
    { k_sum_parts<<<1, 256, 0, s>>>(W.pa, part_grid(Ms[p]->n), W.scal + 4 * NRMAX); ::h2mg::count_launch(); }
    H2_LAUNCH_CHECK();
    H2_CUDA(cudaMemcpyAsync(hp.h + p, W.scal + 4 * NRMAX, sizeof(double), cudaMemcpyDeviceToHost, s));
  }
  H2_CUDA(cudaStreamSynchronize(s));
  for (size_t p = 0; p < P; ++p)
    if (want[p]) out[p] = hp.h[p];
}

// One graph whose branches are the captured V-cycles of the problems in `sel`:
// independent branches, so the kernels of different problems run concurrently.
struct BatchGraph {
  cudaGraphExec_t exec = nullptr;
  int64_t launches = 0;
  std::vector<char> sel;
  ~BatchGraph() {
    if (exec) best_effort(cudaGraphExecDestroy(exec), "cudaGraphExecDestroy (batch)");
  }
  void build(const std::vector<Matrix*>& Ms, const h2mg_solve_opts& o, const std::vector<char>& active) {
    if (exec) {
      best_effort(cudaGraphExecDestroy(exec), "cudaGraphExecDestroy (batch)");
      exec = nullptr;
    }
    cudaGraph_t G = nullptr;
    H2_CUDA(cudaGraphCreate(&G, 0));
    launches = 0;
    try {
      for (size_t p = 0; p < Ms.size(); ++p) {
        if (!active[p]) continue;
        const int k = vcycle_graph(*Ms[p], o, 1, 0);
        const GraphEntry& e = Ms[p]->graphs->g[k];
        cudaGraphNode_t node;
        H2_CUDA(cudaGraphAddChildGraphNode(&node, G, nullptr, 0, e.graph));
        launches += e.launches;
      }
      H2_CUDA(cudaGraphInstantiate(&exec, G, 0));
    } catch (...) {
      best_effort(cudaGraphDestroy(G), "cudaGraphDestroy (batch)");
      throw;
    }
    best_effort(cudaGraphDestroy(G), "cudaGraphDestroy (batch)");
    sel = active;
  }
};

// Independent problems A_p x_p = b_p (one column each) solved together by the outer
// iteration of solve_multi: every outer iteration computes all residuals (one
// synchronisation for all norms), runs the V-cycles of all unconverged problems
// (with use_graph: one launch of a graph with one branch per problem, rebuilt when
// half of its problems have converged; a converged problem's branch then runs on its
// last residual and is ignored), and the outer updates (one synchronisation per group
// of dot products).
h2mg_status solve_batched(const std::vector<Matrix*>& Ms, const double* const* b, double* const* x,
                          const h2mg_solve_opts& o, h2mg_solve_info* info, cudaStream_t s) {
  const size_t P = Ms.size();
  auto t0 = std::chrono::steady_clock::now();
  HostParts hp(P * NPART);
  std::vector<char> all(P, 1), done(P, 0), act(P, 1);
  std::vector<double> nb(P), rel(P), d1(P), d2(P);
  std::vector<const double*> va(P), vb(P);
  std::vector<double *> r(P), pv(P), q(P), pp(P), qp(P), t2(P);
  for (size_t p = 0; p < P; ++p) {
    Work W = work(*Ms[p]);
    r[p] = W.t1;
    t2[p] = W.t2;
    const int64_t n = Ms[p]->n;
    pv[p] = (double*)Ms[p]->wfcg.p;
    q[p] = pv[p] + n * NRMAX;
    pp[p] = q[p] + n * NRMAX;
    qp[p] = pp[p] + n * NRMAX;
    va[p] = b[p];
    vb[p] = b[p];
    info[p] = h2mg_solve_info{};
  }
  dots_many(Ms, va, vb, all, hp, nb.data(), s);
  for (size_t p = 0; p < P; ++p) {
    H2_REQUIRE(std::isfinite(nb[p]), H2MG_ERR_NAN, "right-hand side is not finite");
    nb[p] = std::sqrt(nb[p]);
  }
  const bool fcg = o.outer == H2MG_OUTER_FCG;
  BatchGraph bg;
  bool nan = false;
  for (int cyc = 0; cyc <= o.max_cycles; ++cyc) {
    for (size_t p = 0; p < P; ++p) {
      act[p] = !done[p];
      if (!act[p]) continue;
      const int64_t n = Ms[p]->n;
      outer_residual(*Ms[p], o, b[p], x[p], r[p], t2[p], n, 1, s);
      va[p] = r[p];
      vb[p] = r[p];
    }
    dots_many(Ms, va, vb, act, hp, rel.data(), s);
    size_t left = 0;
    for (size_t p = 0; p < P; ++p) {
      if (!act[p]) continue;
      const double rr = nb[p] > 0 ? std::sqrt(rel[p]) / nb[p] : 0.0;
      if (cyc < 256) info[p].relres_hist[cyc] = rr;
      info[p].cycles = cyc;
      info[p].relres = rr;
      if (!std::isfinite(rr)) {
        nan = true;
        done[p] = 1;
      } else if (rr <= o.tol) {
        info[p].converged = 1;
        done[p] = 1;
      }
      left += !done[p];
    }
    if (left == 0 || nan || cyc == o.max_cycles) break;
    for (size_t p = 0; p < P; ++p) act[p] = !done[p];
    // V-cycles of every unconverged problem: W.et[1] = V(r)
    if (o.use_graph && !Ms[0]->prof.on) {
      size_t built = 0;
      for (char c : bg.sel) built += c;
      if (!bg.exec || left * 2 <= built) bg.build(Ms, o, act);
      H2_CUDA(cudaGraphLaunch(bg.exec, s));
      add_launches(bg.launches);
    } else {
      for (size_t p = 0; p < P; ++p)
        if (act[p]) vcycle_core(*Ms[p], o, r[p], 1, s);
    }
    std::vector<double> alpha(P, 0.0);
    if (!fcg) {
      for (size_t p = 0; p < P; ++p)
        if (act[p]) {
          const double one = 1.0;
          axpy_cols(*Ms[p], &one, work(*Ms[p]).et[1], x[p], Ms[p]->n, 1, s);   // x* = x0 + e_1
        }
      continue;
    }
    for (size_t p = 0; p < P; ++p)
      if (act[p])
        H2_CUDA(cudaMemcpyAsync(pv[p], work(*Ms[p]).et[1], sizeof(double) * Ms[p]->n, cudaMemcpyDeviceToDevice, s));
    if (cyc > 0) {
      for (size_t p = 0; p < P; ++p) {
        va[p] = work(*Ms[p]).et[1];
        vb[p] = qp[p];
      }
      dots_many(Ms, va, vb, act, hp, d1.data(), s);
      for (size_t p = 0; p < P; ++p) va[p] = pp[p];
      dots_many(Ms, va, vb, act, hp, d2.data(), s);
      for (size_t p = 0; p < P; ++p)
        if (act[p]) {
          const double beta = d2[p] != 0.0 ? -d1[p] / d2[p] : 0.0;
          axpy_cols(*Ms[p], &beta, pp[p], pv[p], Ms[p]->n, 1, s);   // p = z + beta p_prev
        }
    }
    for (size_t p = 0; p < P; ++p)
      if (act[p]) apply_level_multi(*Ms[p], 1, false, pv[p], Ms[p]->n, q[p], Ms[p]->n, 1, s);
    for (size_t p = 0; p < P; ++p) {
      va[p] = pv[p];
      vb[p] = r[p];
    }
    dots_many(Ms, va, vb, act, hp, d1.data(), s);
    for (size_t p = 0; p < P; ++p) vb[p] = q[p];
    dots_many(Ms, va, vb, act, hp, d2.data(), s);
    for (size_t p = 0; p < P; ++p)
      if (act[p]) {
        const double al = d2[p] > 0.0 ? d1[p] / d2[p] : 0.0;
        axpy_cols(*Ms[p], &al, pv[p], x[p], Ms[p]->n, 1, s);        // x += alpha p
        std::swap(pv[p], pp[p]);
        std::swap(q[p], qp[p]);
      }
  }
  H2_CUDA(cudaStreamSynchronize(s));
  const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  h2mg_status st = H2MG_OK;
  for (size_t p = 0; p < P; ++p) {
    info[p].ms_solve = ms;
    if (!info[p].converged) st = H2MG_ERR_NOT_CONVERGED;
  }
  if (nan) st = H2MG_ERR_NAN;
  return st;
}

h2mg_status solve(Matrix& M, const double* b, double* x, const h2mg_solve_opts& o, h2mg_solve_info* info,
                  cudaStream_t s) {
  h2mg_solve_info loc;
  const h2mg_status st = solve_multi(M, b, x, 1, o, &loc, s);
  if (info) *info = loc;
  return st;
}

}  // namespace h2mg
