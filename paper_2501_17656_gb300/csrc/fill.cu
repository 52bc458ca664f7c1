// fill.cu -- Chebyshev nested bases, their QR orthonormalisation, and the stored
// blocks: close blocks D, couplings S, coarse near fields P_i (all float64 math).
//
// Sec. 3.1: far blocks are U_i S_ij V_j with nested row/column bases; here the bases
// come from tensor Chebyshev interpolation on each cluster's tight box (q first-kind
// nodes per axis, k = q^dim): leaf basis U^cheb[i, a] = sqrt(w_i) L_a(x_i), transfer
// E_c[a, b] = L^P_b(xi^c_a), coupling S^cheb = k(xi_tau, xi_sigma).
// Sec. 3.3 restricts with orthogonal bases: the leaf bases are replaced by Q of
// U^cheb = Q R and each parent by Q of [R_c1 E_c1; R_c2 E_c2] = Q_P R_P, so that the
// orthonormal transfers are the two row blocks of Q_P and S = R_tau S^cheb R_sigma^T
// (diag(R) >= 0; ranks r = min(k, rows), never truncated).
// Eq. a2_str: the coarse near field of level i >= 2 is
//   P_2(c, c') = U_c^T D(c, c') U_c',   P_i(c, c') = sum_{a, a'} E'_a^T M(a, a') E'_a',
// M = P_{i-1} block if (a, a') is a non-far pair of the finer level, else its S block.
#include <algorithm>
#include <cmath>
#include <unordered_map>

#include "internal.h"

namespace h2mg {

// ----------------------------------------------------------------------------- helpers
__device__ __forceinline__ void unswz(int pos, int K, int V, int& i, int& j) {
  int LPC = K / 8, CPP = 32 / LPC, P = 8 / V;
  int sub = pos % V;
  int lane = (pos / V) % 32;
  int tk = pos / (V * 32);
  int t = tk / P, k = tk % P;
  i = 8 * (lane % LPC) + k * V + sub;
  j = t * CPP + lane / LPC;
}

__device__ __forceinline__ double load_elem(const void* pool, int fmt, int64_t idx) {
  if (fmt == FMT_F64) return ((const double*)pool)[idx];
  if (fmt == FMT_DF) {
    float2 v = ((const float2*)pool)[idx];
    return (double)v.x + (double)v.y;
  }
  return (double)((const float*)pool)[idx];
}

__device__ __forceinline__ void store_elem(void* pool, int fmt, int64_t idx, double v) {
  if (fmt == FMT_F64) {
    ((double*)pool)[idx] = v;
  } else if (fmt == FMT_DF) {
    float h = __double2float_rn(v);
    float l = __double2float_rn(v - (double)h);
    ((float2*)pool)[idx] = make_float2(h, l);
  } else {
    ((float*)pool)[idx] = __double2float_rn(v);
  }
}

// Write a K x K natural column-major block (ld K) into the pool, swizzled.
__device__ void store_block(void* pool, int fmt, int64_t blk, int K, const double* B) {
  int V = fmt == FMT_F32 ? 4 : 2;
  int64_t base = blk * K * K;
  for (int pos = threadIdx.x; pos < K * K; pos += blockDim.x) {
    int i, j;
    unswz(pos, K, V, i, j);
    store_elem(pool, fmt, base + pos, B[i + j * K]);
  }
}

// Read a swizzled K x K block into natural column-major order (transposed if asked).
__device__ void load_block(const void* pool, int fmt, int64_t blk, int K, bool trans, double* B) {
  int V = fmt == FMT_F32 ? 4 : 2;
  int64_t base = blk * K * K;
  for (int pos = threadIdx.x; pos < K * K; pos += blockDim.x) {
    int i, j;
    unswz(pos, K, V, i, j);
    double v = load_elem(pool, fmt, base + pos);
    if (trans)
      B[j + i * K] = v;
    else
      B[i + j * K] = v;
  }
}

__device__ __forceinline__ double cheb_t(int a, int q) {
  return cos((2.0 * a + 1.0) * 3.14159265358979323846 / (2.0 * q));
}

// l_b(t) on the q first-kind nodes
__device__ double lagrange1(int b, double t, int q) {
  double v = 1.0, tb = cheb_t(b, q);
  for (int c = 0; c < q; ++c)
    if (c != b) {
      double tc = cheb_t(c, q);
      v *= (t - tc) / (tb - tc);
    }
  return v;
}

// L_a(y) for the cluster whose box center/half-width are (cen, hw)
__device__ double lagrange_tensor(int a, const double* y, const double* cen, const double* hw,
                                  int dim, int q) {
  double v = 1.0;
  for (int d = 0; d < dim; ++d) {
    int ad = a % q;
    a /= q;
    v *= lagrange1(ad, (y[d] - cen[d]) / hw[d], q);
  }
  return v;
}

__device__ void box_center_half(const double* box, int j, int dim, double floor_hw, double* cen,
                                double* hw) {
  for (int d = 0; d < dim; ++d) {
    double lo = box[(int64_t)j * 2 * dim + d], hi = box[(int64_t)j * 2 * dim + dim + d];
    cen[d] = 0.5 * (lo + hi);
    hw[d] = fmax(0.5 * (hi - lo), floor_hw);
  }
}

// Block-wide sum (blockDim.x <= 1024, multiple of 32); red has >= 33 doubles.
__device__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
    red[32] = s;
  }
  __syncthreads();
  return red[32];
}

// Householder QR of the m x n column-major A (ld lda), then Q = first r = min(m, n)
// columns of H_0 ... H_{r-1} in Qm (ld ldq), with diag(R) >= 0. R is left in the
// upper triangle of A.
__device__ void cta_qr(double* A, int lda, int m, int n, double* Qm, int ldq, double* tau,
                       double* red) {
  int r = min(m, n);
  for (int j = 0; j < r; ++j) {
    double part = 0.0;
    for (int i = j + 1 + threadIdx.x; i < m; i += blockDim.x) part += A[i + j * lda] * A[i + j * lda];
    double sigma = block_sum(part, red);
    double alpha = A[j + j * lda];
    double tj = 0.0, scale = 0.0, beta = alpha;
    if (sigma > 0.0) {
      beta = -copysign(sqrt(alpha * alpha + sigma), alpha);
      tj = (beta - alpha) / beta;
      scale = 1.0 / (alpha - beta);
    }
    __syncthreads();
    if (sigma > 0.0)
      for (int i = j + 1 + threadIdx.x; i < m; i += blockDim.x) A[i + j * lda] *= scale;
    if (threadIdx.x == 0) {
      A[j + j * lda] = beta;
      tau[j] = tj;
    }
    __syncthreads();
    if (tj != 0.0)
      for (int c = j + 1 + threadIdx.x; c < n; c += blockDim.x) {
        double w = A[j + c * lda];
        for (int i = j + 1; i < m; ++i) w += A[i + j * lda] * A[i + c * lda];
        w *= tj;
        A[j + c * lda] -= w;
        for (int i = j + 1; i < m; ++i) A[i + c * lda] -= w * A[i + j * lda];
      }
    __syncthreads();
  }
  // Q = I(:, 0:r), then apply H_{r-1} .. H_0
  for (int e = threadIdx.x; e < m * r; e += blockDim.x) {
    int i = e % m, c = e / m;
    Qm[i + c * ldq] = (i == c) ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int j = r - 1; j >= 0; --j) {
    double tj = tau[j];
    if (tj != 0.0)
      for (int c = j + threadIdx.x; c < r; c += blockDim.x) {
        double w = Qm[j + c * ldq];
        for (int i = j + 1; i < m; ++i) w += A[i + j * lda] * Qm[i + c * ldq];
        w *= tj;
        Qm[j + c * ldq] -= w;
        for (int i = j + 1; i < m; ++i) Qm[i + c * ldq] -= w * A[i + j * lda];
      }
    __syncthreads();
  }
  // diag(R) >= 0
  for (int j = threadIdx.x; j < r; j += blockDim.x) {
    if (A[j + j * lda] < 0.0) {
      for (int c = j; c < n; ++c) A[j + c * lda] = -A[j + c * lda];
      for (int i = 0; i < m; ++i) Qm[i + j * ldq] = -Qm[i + j * ldq];
    }
  }
  __syncthreads();
}

// ----------------------------------------------------------------------------- nodes
__global__ void k_nodes(const double* __restrict__ box, int ell, int dim, int q, int k,
                        double floor_hw, double* __restrict__ nodes) {
  int j = blockIdx.x;
  double cen[3], hw[3];
  box_center_half(box, j, dim, floor_hw, cen, hw);
  for (int a = threadIdx.x; a < k; a += blockDim.x) {
    int aa = a;
    for (int d = 0; d < dim; ++d) {
      int ad = aa % q;
      aa /= q;
      nodes[((int64_t)j * k + a) * dim + d] = cen[d] + hw[d] * cheb_t(ad, q);
    }
  }
}

// ----------------------------------------------------------------------------- leaf QR
// One block per leaf: U^0 (n_j x k) -> Q into U (KD x KC), R into Rout (KC x KC).
// U^0 is the Chebyshev basis sqrt(w_i) L_a(x_i), or, with skeleton factors Tid
// (column-major, ld 128 per leaf, rank_id[j] columns), the leaf's interpolation matrix.
__global__ void k_leaf_qr(const double* __restrict__ X, const double* __restrict__ sw,
                          const int* __restrict__ leafoff, const double* __restrict__ box,
                          int dim, int q, int k, int KD, int KC, double floor_hw,
                          const double* __restrict__ Tid, const int* __restrict__ rank_id,
                          double* __restrict__ U, double* __restrict__ Rout) {
  extern __shared__ double sm[];
  double* A = sm;                    // KD x k
  double* Qm = A + KD * k;           // KD x KD
  double* tau = Qm + KD * KD;        // 64
  double* red = tau + 64;            // 33
  int j = blockIdx.x;
  int p0 = leafoff[j], m = leafoff[j + 1] - p0;
  if (Tid) k = rank_id[j];
  double cen[3], hw[3];
  box_center_half(box, j, dim, floor_hw, cen, hw);
  for (int e = threadIdx.x; e < m * k; e += blockDim.x) {
    int i = e % m, a = e / m;
    if (Tid) {
      A[i + a * KD] = Tid[(int64_t)j * 128 * 64 + i + a * 128];
    } else {
      const double* x = X + (int64_t)(p0 + i) * dim;
      A[i + a * KD] = sw[p0 + i] * lagrange_tensor(a, x, cen, hw, dim, q);
    }
  }
  __syncthreads();
  cta_qr(A, KD, m, k, Qm, KD, tau, red);
  int r = min(m, k);
  double* Uj = U + (int64_t)j * KD * KC;
  for (int e = threadIdx.x; e < KD * KC; e += blockDim.x) {
    int i = e % KD, c = e / KD;
    Uj[e] = (i < m && c < r) ? Qm[i + c * KD] : 0.0;
  }
  double* Rj = Rout + (int64_t)j * KC * KC;
  for (int e = threadIdx.x; e < KC * KC; e += blockDim.x) {
    int i = e % KC, c = e / KC;
    Rj[e] = (i < r && c < k && i <= c) ? A[i + c * KD] : 0.0;
  }
}

// ----------------------------------------------------------------------------- parent QR
// One block per parent p at level ell: M = [R_c1 E_c1; R_c2 E_c2] = Q R_P; the
// orthonormal transfers E'_c are the row blocks of Q (stored KC x KC, child rows).
// E_c is the Chebyshev transfer L^P_b(xi^c_a) (k x k), or, with skeleton factors
// (Tid: the parent's interpolation matrix, ld 128, rows = the children's skeletons),
// the rows of T_p that belong to child c (r_c x r_p).
__global__ void k_parent_qr(const double* __restrict__ box_p, const double* __restrict__ nodes_c,
                            const int* __restrict__ rank_c, int dim, int q, int k, int KC,
                            double floor_hw, const double* __restrict__ R_c,
                            const double* __restrict__ Tid, const int* __restrict__ rank_p,
                            double* __restrict__ E_out, double* __restrict__ R_out) {
  extern __shared__ double sm[];
  double* E = sm;                    // k x k (one child at a time)
  double* A = E + k * k;             // 2k x k, ld 2k
  double* Qm = A + 2 * k * k;        // 2k x k, ld 2k
  double* tau = Qm + 2 * k * k;      // 64
  double* red = tau + 64;            // 33
  int p = blockIdx.x;
  double cen[3], hw[3];
  box_center_half(box_p, p, dim, floor_hw, cen, hw);
  int r1 = rank_c[2 * p], r2 = rank_c[2 * p + 1];
  int m = r1 + r2, ld = 2 * k;
  const int kout = Tid ? rank_p[p] : k;   // columns: the parent's basis functions
  for (int c = 0; c < 2; ++c) {
    int child = 2 * p + c;
    int rc = c ? r2 : r1, row0 = c ? r1 : 0;
    const int kin = Tid ? rc : k;         // rows of E_c: the child's basis functions
    for (int e = threadIdx.x; e < kin * kout; e += blockDim.x) {
      int a = e % kin, b = e / kin;
      E[a + b * kin] = Tid ? Tid[(int64_t)p * 128 * 64 + row0 + a + b * 128]   // E_c[a, b] = T_p[c's a-th, b]
                           : lagrange_tensor(b, nodes_c + ((int64_t)child * k + a) * dim, cen, hw, dim, q);
    }
    __syncthreads();
    const double* Rc = R_c + (int64_t)child * KC * KC;
    for (int e = threadIdx.x; e < rc * kout; e += blockDim.x) {
      int i = e % rc, b = e / rc;
      double s = 0.0;
      for (int a = i; a < kin; ++a) s += Rc[i + a * KC] * E[a + b * kin];
      A[row0 + i + b * ld] = s;
    }
    __syncthreads();
  }
  cta_qr(A, ld, m, kout, Qm, ld, tau, red);
  k = kout;
  int rp = min(m, k);
  for (int c = 0; c < 2; ++c) {
    int child = 2 * p + c;
    int rc = c ? r2 : r1, row0 = c ? r1 : 0;
    double* Ec = E_out + (int64_t)child * KC * KC;
    for (int e = threadIdx.x; e < KC * KC; e += blockDim.x) {
      int i = e % KC, b = e / KC;
      Ec[e] = (i < rc && b < rp) ? Qm[row0 + i + b * ld] : 0.0;
    }
  }
  double* Rp = R_out + (int64_t)p * KC * KC;
  for (int e = threadIdx.x; e < KC * KC; e += blockDim.x) {
    int i = e % KC, c = e / KC;
    Rp[e] = (i < rp && c < k && i <= c) ? A[i + c * ld] : 0.0;
  }
}

void build_bases(Matrix& M) {
  if (M.tstar < 0) return;
  cudaStream_t s = M.stream;
  const int L = M.L, dim = M.dim, q = M.q, k = M.k, KD = M.KD, KC = M.KC, ts = M.tstar;
  const int nsl = M.nslots();
  // floor of the box half-widths: 1e-12 of the root extent
  std::vector<double> rb(2 * dim);
  H2_CUDA(cudaMemcpy(rb.data(), M.d_box[0], sizeof(double) * 2 * dim, cudaMemcpyDeviceToHost));
  double ext = 0.0;
  for (int d = 0; d < dim; ++d) ext = std::max(ext, rb[dim + d] - rb[d]);
  double floor_hw = 1e-12 * std::max(ext, 1e-300);
  const bool skel = M.basis == H2MG_BASIS_SKELETON;
  if (skel) {
    // skeletons, interpolation matrices, ranks and coupling points (skeleton.cu)
    build_skeletons(M);
  } else {
    // ranks (host): leaves min(k, n_j); parents min(k, r_c1 + r_c2)
    M.h_rank.assign(nsl, 0);
    std::vector<int> rk(1 << L);
    for (int j = 0; j < (1 << L); ++j) rk[j] = std::min(k, M.offsets[L][j + 1] - M.offsets[L][j]);
    for (int ell = L; ell >= ts; --ell) {
      if (ell < L) {
        std::vector<int> up(1 << ell);
        for (int p = 0; p < (1 << ell); ++p) up[p] = std::min(k, rk[2 * p] + rk[2 * p + 1]);
        rk.swap(up);
      }
      for (int j = 0; j < (1 << ell); ++j) M.h_rank[M.slot0(ell) + j] = rk[j];
    }
    M.d_rank = (int*)M.alloc(sizeof(int) * nsl);
    H2_CUDA(cudaMemcpyAsync(M.d_rank, M.h_rank.data(), sizeof(int) * nsl, cudaMemcpyHostToDevice, s));
    M.d_nodes = (double*)M.alloc(sizeof(double) * (size_t)nsl * k * dim);
    for (int ell = ts; ell <= L; ++ell) {
      { k_nodes<<<1 << ell, 128, 0, s>>>(M.d_box[ell], ell, dim, q, k, floor_hw,
                                       M.d_nodes + (size_t)M.slot0(ell) * k * dim); ::h2mg::count_launch(); }
      H2_LAUNCH_CHECK();
    }
  }
  const double* Tid = skel ? (const double*)M.tid.p : nullptr;
  const int* rid = skel ? M.d_rank : nullptr;
  M.d_U = (double*)M.alloc(sizeof(double) * (size_t)(1 << L) * KD * KC);
  M.d_R = (double*)M.alloc(sizeof(double) * (size_t)nsl * KC * KC);
  M.d_E = (double*)M.alloc(sizeof(double) * (size_t)nsl * KC * KC);
  {
    size_t sm = sizeof(double) * ((size_t)KD * k + KD * KD + 64 + 33);
    H2_CUDA(cudaFuncSetAttribute(k_leaf_qr, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    { k_leaf_qr<<<1 << L, 128, sm, s>>>(M.d_X, M.d_sw, M.d_leafoff, M.d_box[L], dim, q, k, KD, KC,
                                       floor_hw, Tid ? Tid + (size_t)M.slot0(L) * 128 * 64 : nullptr,
                                       rid ? rid + M.slot0(L) : nullptr, M.d_U,
                                       M.d_R + (size_t)M.slot0(L) * KC * KC); ::h2mg::count_launch(); }
    H2_LAUNCH_CHECK();
  }
  {
    size_t sm = sizeof(double) * ((size_t)k * k + 4 * k * k + 64 + 33);
    H2_CUDA(cudaFuncSetAttribute(k_parent_qr, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    for (int ell = L - 1; ell >= ts; --ell) {
      { k_parent_qr<<<1 << ell, 128, sm, s>>>(
          M.d_box[ell], M.d_nodes + (size_t)M.slot0(ell + 1) * k * dim, M.d_rank + M.slot0(ell + 1),
          dim, q, k, KC, floor_hw, M.d_R + (size_t)M.slot0(ell + 1) * KC * KC,
          Tid ? Tid + (size_t)M.slot0(ell) * 128 * 64 : nullptr, rid ? rid + M.slot0(ell) : nullptr,
          M.d_E + (size_t)M.slot0(ell + 1) * KC * KC, M.d_R + (size_t)M.slot0(ell) * KC * KC); ::h2mg::count_launch(); }
      H2_LAUNCH_CHECK();
    }
  }
  H2_CUDA(cudaStreamSynchronize(s));
  if (skel) M.free_owned(M.tid.p);   // the interpolation matrices live on in U, E and R
  M.tid = DevBuf{};
}

// ----------------------------------------------------------------------------- blocks
// S = R_t k(xi_t, xi_s) R_s^T for far pairs (t, s) (slots), written swizzled.
// Coupling points: k per slot (Chebyshev nodes, unit weights), or, with cnt / nw given,
// the cnt[slot] skeleton points of each slot with their sqrt(w).
__global__ void k_fill_S(const int* __restrict__ pt, const int* __restrict__ ps,
                         const double* __restrict__ nodes, const double* __restrict__ R, int k,
                         int KC, int dim, KernelParams kp, const int* __restrict__ cnt,
                         const double* __restrict__ nw, void* __restrict__ pool, int fmt) {
  extern __shared__ double sm[];
  double* Sc = sm;              // KC x KC
  double* T = Sc + KC * KC;     // KC x KC
  int64_t b = blockIdx.x;
  int t = pt[b], s = ps[b];
  const int kt = cnt ? cnt[t] : k, ks = cnt ? cnt[s] : k;
  for (int e = threadIdx.x; e < KC * KC; e += blockDim.x) {
    int a = e % KC, c = e / KC;
    double v = 0.0;
    if (a < kt && c < ks) {
      v = kernel_eval(kp, nodes + ((int64_t)t * k + a) * dim, nodes + ((int64_t)s * k + c) * dim, dim);
      if (nw) v *= nw[(int64_t)t * k + a] * nw[(int64_t)s * k + c];
    }
    Sc[e] = v;
  }
  __syncthreads();
  const double* Rt = R + (int64_t)t * KC * KC;
  const double* Rs = R + (int64_t)s * KC * KC;
  // T = Sc R_s^T : T[a][c] = sum_{b >= c} Sc[a][b] R_s[c][b]
  for (int e = threadIdx.x; e < KC * KC; e += blockDim.x) {
    int a = e % KC, c = e / KC;
    double v = 0.0;
    for (int bb = c; bb < KC; ++bb) v += Sc[a + bb * KC] * Rs[c + bb * KC];
    T[e] = v;
  }
  __syncthreads();
  // S = R_t T : S[r][c] = sum_{a >= r} R_t[r][a] T[a][c]
  for (int e = threadIdx.x; e < KC * KC; e += blockDim.x) {
    int r = e % KC, c = e / KC;
    double v = 0.0;
    for (int a = r; a < KC; ++a) v += Rt[r + a * KC] * T[a + c * KC];
    Sc[e] = v;
  }
  __syncthreads();
  store_block(pool, fmt, b, KC, Sc);
}

// D block (t, s) of leaves: sqrt(w_i) k(x_i, x_j) sqrt(w_j), A_ii on the diagonal.
__device__ double d_entry(int i, int j, int t, int s, const int* leafoff, const double* X,
                          const double* sw, const double* dg, int dim, const KernelParams& kp) {
  int nt = leafoff[t + 1] - leafoff[t], ns = leafoff[s + 1] - leafoff[s];
  if (i >= nt || j >= ns) return 0.0;
  int pi = leafoff[t] + i, pj = leafoff[s] + j;
  if (pi == pj) return dg[pi];
  return sw[pi] * kernel_eval(kp, X + (int64_t)pi * dim, X + (int64_t)pj * dim, dim) * sw[pj];
}

__global__ void k_fill_D(const int* __restrict__ pt, const int* __restrict__ ps,
                         const int* __restrict__ leafoff, const double* __restrict__ X,
                         const double* __restrict__ sw, const double* __restrict__ dg, int dim,
                         int KD, KernelParams kp, void* __restrict__ pool, int fmt) {
  int64_t b = blockIdx.x;
  int t = pt[b], s = ps[b];
  int V = fmt == FMT_F32 ? 4 : 2;
  for (int pos = threadIdx.x; pos < KD * KD; pos += blockDim.x) {
    int i, j;
    unswz(pos, KD, V, i, j);
    store_elem(pool, fmt, b * KD * KD + pos, d_entry(i, j, t, s, leafoff, X, sw, dg, dim, kp));
  }
}

// P_2 = U_t^T D(t, s) U_s with D recomputed in float64.
__global__ void k_fill_P2(const int* __restrict__ pt, const int* __restrict__ ps,
                          const int* __restrict__ leafoff, const double* __restrict__ X,
                          const double* __restrict__ sw, const double* __restrict__ dg, int dim,
                          int KD, int KC, KernelParams kp, const double* __restrict__ U,
                          void* __restrict__ pool, int fmt) {
  extern __shared__ double sm[];
  double* D = sm;                              // KD x KD (then KC x KC)
  double* T = D + max(KD * KD, KC * KC);       // KD x KC
  int64_t b = blockIdx.x;
  int t = pt[b], s = ps[b];
  for (int e = threadIdx.x; e < KD * KD; e += blockDim.x)
    D[e] = d_entry(e % KD, e / KD, t, s, leafoff, X, sw, dg, dim, kp);
  __syncthreads();
  const double* Ut = U + (int64_t)t * KD * KC;
  const double* Us = U + (int64_t)s * KD * KC;
  for (int e = threadIdx.x; e < KD * KC; e += blockDim.x) {
    int i = e % KD, c = e / KD;
    double v = 0.0;
    for (int jj = 0; jj < KD; ++jj) v += D[i + jj * KD] * Us[jj + c * KD];
    T[e] = v;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < KC * KC; e += blockDim.x) {
    int r = e % KC, c = e / KC;
    double v = 0.0;
    for (int i = 0; i < KD; ++i) v += Ut[i + r * KD] * T[i + c * KD];
    D[e] = v;   // reuse
  }
  __syncthreads();
  store_block(pool, fmt, b, KC, D);
}

// P_i (i >= 3) from the four child blocks (references precomputed on the host).
struct ChildRef {
  int pool;      // 0: P_{i-1} pool, 1: S pool
  int trans;     // read the transposed block
  int64_t blk;   // block index in that pool
};

__global__ void k_fill_Pi(const int* __restrict__ pt, const int* __restrict__ ps,
                          const ChildRef* __restrict__ ref, const void* __restrict__ poolPf,
                          const void* __restrict__ poolS, int fmt, const double* __restrict__ E,
                          int KC, void* __restrict__ pool) {
  extern __shared__ double sm[];
  double* Mb = sm;              // KC x KC
  double* T = Mb + KC * KC;
  double* acc = T + KC * KC;
  int64_t b = blockIdx.x;
  int c = pt[b], cp = ps[b];    // fine-level slot indices of the children are 2c+x (relative)
  for (int e = threadIdx.x; e < KC * KC; e += blockDim.x) acc[e] = 0.0;
  for (int q4 = 0; q4 < 4; ++q4) {
    ChildRef R = ref[b * 4 + q4];
    int a = 2 * c + (q4 >> 1), ap = 2 * cp + (q4 & 1);
    __syncthreads();
    load_block(R.pool ? poolS : poolPf, fmt, R.blk, KC, R.trans != 0, Mb);
    __syncthreads();
    const double* Ea = E + (int64_t)a * KC * KC;
    const double* Eap = E + (int64_t)ap * KC * KC;
    // T = M E'_ap
    for (int e = threadIdx.x; e < KC * KC; e += blockDim.x) {
      int i = e % KC, jj = e / KC;
      double v = 0.0;
      for (int l = 0; l < KC; ++l) v += Mb[i + l * KC] * Eap[l + jj * KC];
      T[e] = v;
    }
    __syncthreads();
    // acc += E'_a^T T
    for (int e = threadIdx.x; e < KC * KC; e += blockDim.x) {
      int r = e % KC, jj = e / KC;
      double v = 0.0;
      for (int l = 0; l < KC; ++l) v += Ea[l + r * KC] * T[l + jj * KC];
      acc[e] += v;
    }
  }
  __syncthreads();
  store_block(pool, fmt, b, KC, acc);
}

// Re-store a pool in another format (the swizzle depends on the element width).
__global__ void k_convert_pool(const void* __restrict__ src, int fsrc, void* __restrict__ dst,
                               int fdst, int K) {
  int64_t b = blockIdx.x;
  int Vs = fsrc == FMT_F32 ? 4 : 2, Vd = fdst == FMT_F32 ? 4 : 2;
  for (int pos = threadIdx.x; pos < K * K; pos += blockDim.x) {
    int i, j;
    unswz(pos, K, Vd, i, j);
    double v = load_elem(src, fsrc, b * K * K + swz(i, j, K, Vs));
    store_elem(dst, fdst, b * K * K + pos, v);
  }
}

__global__ void k_to_f32(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = __double2float_rn(a[i]);
}

// ----------------------------------------------------------------------------- host side
static void upload_pairs(Matrix& M, const std::vector<int>& t, const std::vector<int>& s, int** dt,
                         int** ds) {
  size_t n = std::max<size_t>(t.size(), 1);
  *dt = (int*)M.alloc(sizeof(int) * n);
  *ds = (int*)M.alloc(sizeof(int) * n);
  if (!t.empty()) {
    H2_CUDA(cudaMemcpyAsync(*dt, t.data(), sizeof(int) * t.size(), cudaMemcpyHostToDevice, M.stream));
    H2_CUDA(cudaMemcpyAsync(*ds, s.data(), sizeof(int) * s.size(), cudaMemcpyHostToDevice, M.stream));
  }
}

// Launch a grid of up to 2^31-1 blocks in chunks of 65535 * 1024 (plenty).
template <class F>
static void chunked(int64_t nb, F launch) {
  const int64_t CH = 1 << 20;
  for (int64_t b0 = 0; b0 < nb; b0 += CH) launch(b0, (int)std::min(CH, nb - b0));
}

static size_t pool_bytes(int64_t nblk, int K, int fmt) { return (size_t)nblk * K * K * fmt_bytes(fmt); }

void build_blocks(Matrix& M, const Matrix* base) {
  (void)base;
  cudaStream_t s = M.stream;
  const int L = M.L, KD = M.KD, KC = M.KC, dim = M.dim, k = M.k;
  // ---- close pairs (upper) -> D
  std::vector<int> dt, ds;
  const HostCSR& N = M.inadm[L];
  for (int t = 0; t < (1 << L); ++t)
    for (int e = N.rowptr[t]; e < N.rowptr[t + 1]; ++e)
      if (N.col[e] >= t) {
        dt.push_back(t);
        ds.push_back(N.col[e]);
      }
  M.nD = (int64_t)dt.size();
  int *d_dt, *d_ds;
  upload_pairs(M, dt, ds, &d_dt, &d_ds);
  M.poolD.bytes = pool_bytes(M.nD, KD, M.fmt);
  M.poolD.p = M.alloc(M.poolD.bytes);
  chunked(M.nD, [&](int64_t b0, int nb) {
    { k_fill_D<<<nb, 256, 0, s>>>(d_dt + b0, d_ds + b0, M.d_leafoff, M.d_X, M.d_sw, M.d_dg, dim, KD,
                                M.kp, (char*)M.poolD.p + pool_bytes(b0, KD, M.fmt), M.fmt); ::h2mg::count_launch(); }
    H2_LAUNCH_CHECK();
  });
  if (M.tstar < 0) {
    H2_CUDA(cudaStreamSynchronize(s));
    return;
  }
  // ---- far pairs (upper) of levels t*..L -> S, level by level
  std::vector<int> st, ss;
  M.s_level_base.assign(L + 2, 0);
  for (int ell = M.tstar; ell <= L; ++ell) {
    M.s_level_base[ell] = (int64_t)st.size();
    const HostCSR& F = M.far[ell];
    for (int t = 0; t < (1 << ell); ++t)
      for (int e = F.rowptr[t]; e < F.rowptr[t + 1]; ++e)
        if (F.col[e] > t) {
          st.push_back(M.slot0(ell) + t);
          ss.push_back(M.slot0(ell) + F.col[e]);
        }
  }
  M.s_level_base[L + 1] = (int64_t)st.size();
  M.nS = (int64_t)st.size();
  int *d_st, *d_ss;
  upload_pairs(M, st, ss, &d_st, &d_ss);
  M.poolS.bytes = pool_bytes(M.nS, KC, M.fmt);
  M.poolS.p = M.alloc(M.poolS.bytes);
  size_t smS = sizeof(double) * 2 * KC * KC;
  H2_CUDA(cudaFuncSetAttribute(k_fill_S, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smS));
  chunked(M.nS, [&](int64_t b0, int nb) {
    const bool sk = M.basis == H2MG_BASIS_SKELETON;
    { k_fill_S<<<nb, 256, smS, s>>>(d_st + b0, d_ss + b0, M.d_nodes, M.d_R, sk ? KC : k, KC, dim, M.kp,
                                  sk ? M.d_rank : nullptr, sk ? M.d_nsw : nullptr,
                                  (char*)M.poolS.p + pool_bytes(b0, KC, M.fmt), M.fmt); ::h2mg::count_launch(); }
    H2_LAUNCH_CHECK();
  });
  H2_CUDA(cudaStreamSynchronize(s));
}

// Index of the upper entry (t, s) of a full CSR list restricted to s >= t, or -1.
static int64_t upper_index(const HostCSR& C, const std::vector<int64_t>& ubase, int t, int s,
                           bool strict) {
  auto b = C.col.begin() + C.rowptr[t], e = C.col.begin() + C.rowptr[t + 1];
  auto it = std::lower_bound(b, e, s);
  if (it == e || *it != s) return -1;
  auto first = std::lower_bound(b, e, strict ? t + 1 : t);
  return ubase[t] + (it - first);
}

static std::vector<int64_t> upper_base(const HostCSR& C, int nrows, bool strict) {
  std::vector<int64_t> ub(nrows + 1, 0);
  for (int t = 0; t < nrows; ++t) {
    int cnt = 0;
    for (int e = C.rowptr[t]; e < C.rowptr[t + 1]; ++e) cnt += strict ? (C.col[e] > t) : (C.col[e] >= t);
    ub[t + 1] = ub[t] + cnt;
  }
  return ub;
}

void build_coarse_near(Matrix& M) {
  if (M.tstar < 0 || M.lev < 2) return;
  cudaStream_t s = M.stream;
  const int L = M.L, KD = M.KD, KC = M.KC, dim = M.dim;
  M.poolP.assign(M.lev + 1, {});
  M.nP.assign(M.lev + 1, 0);
  // ---- P_2 on the close leaf pairs (same upper list as D)
  {
    std::vector<int> dt, ds;
    const HostCSR& N = M.inadm[L];
    for (int t = 0; t < (1 << L); ++t)
      for (int e = N.rowptr[t]; e < N.rowptr[t + 1]; ++e)
        if (N.col[e] >= t) {
          dt.push_back(t);
          ds.push_back(N.col[e]);
        }
    int *d_t, *d_s;
    upload_pairs(M, dt, ds, &d_t, &d_s);
    M.nP[2] = (int64_t)dt.size();
    M.poolP[2].bytes = pool_bytes(M.nP[2], KC, M.fmt);
    M.poolP[2].p = M.alloc(M.poolP[2].bytes);
    size_t sm = sizeof(double) * ((size_t)std::max(KD * KD, KC * KC) + KD * KC);
    H2_CUDA(cudaFuncSetAttribute(k_fill_P2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    chunked(M.nP[2], [&](int64_t b0, int nb) {
      { k_fill_P2<<<nb, 256, sm, s>>>(d_t + b0, d_s + b0, M.d_leafoff, M.d_X, M.d_sw, M.d_dg, dim, KD,
                                    KC, M.kp, M.d_U, (char*)M.poolP[2].p + pool_bytes(b0, KC, M.fmt),
                                    M.fmt); ::h2mg::count_launch(); }
      H2_LAUNCH_CHECK();
    });
  }
  // ---- P_i, i >= 3, level by level
  size_t sm = sizeof(double) * 3 * KC * KC;
  H2_CUDA(cudaFuncSetAttribute(k_fill_Pi, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  for (int i = 3; i <= M.lev; ++i) {
    int mc = L - i + 2, mf = mc + 1;
    const HostCSR& Ic = M.inadm[mc];
    const HostCSR& If = M.inadm[mf];
    const HostCSR& Ff = M.far[mf];
    auto ubI = upper_base(If, 1 << mf, false);
    auto ubF = upper_base(Ff, 1 << mf, true);
    std::vector<int> pt, ps;
    std::vector<ChildRef> refs;
    for (int c = 0; c < (1 << mc); ++c)
      for (int e = Ic.rowptr[c]; e < Ic.rowptr[c + 1]; ++e) {
        int cp = Ic.col[e];
        if (cp < c) continue;
        pt.push_back(c);
        ps.push_back(cp);
        for (int q4 = 0; q4 < 4; ++q4) {
          int a = 2 * c + (q4 >> 1), ap = 2 * cp + (q4 & 1);
          int lo = std::min(a, ap), hi = std::max(a, ap);
          ChildRef R{0, a > ap ? 1 : 0, -1};
          int64_t idx = upper_index(If, ubI, lo, hi, false);
          if (idx >= 0) {
            R.pool = 0;
            R.blk = idx;
          } else {
            idx = upper_index(Ff, ubF, lo, hi, true);
            H2_REQUIRE(idx >= 0, H2MG_ERR_CUDA, "internal: child pair missing from the partition");
            R.pool = 1;
            R.blk = M.s_level_base[mf] + idx;
          }
          refs.push_back(R);
        }
      }
    int *d_t, *d_s;
    upload_pairs(M, pt, ps, &d_t, &d_s);
    ChildRef* d_ref = (ChildRef*)M.alloc(sizeof(ChildRef) * std::max<size_t>(refs.size(), 1));
    if (!refs.empty())
      H2_CUDA(cudaMemcpyAsync(d_ref, refs.data(), sizeof(ChildRef) * refs.size(), cudaMemcpyHostToDevice, s));
    M.nP[i] = (int64_t)pt.size();
    M.poolP[i].bytes = pool_bytes(M.nP[i], KC, M.fmt);
    M.poolP[i].p = M.alloc(M.poolP[i].bytes);
    const double* Ef = M.d_E + (size_t)M.slot0(mf) * KC * KC;
    chunked(M.nP[i], [&](int64_t b0, int nb) {
      { k_fill_Pi<<<nb, 256, sm, s>>>(d_t + b0, d_s + b0, d_ref + b0 * 4, M.poolP[i - 1].p, M.poolS.p,
                                    M.fmt, Ef, KC, (char*)M.poolP[i].p + pool_bytes(b0, KC, M.fmt)); ::h2mg::count_launch(); }
      H2_LAUNCH_CHECK();
    });
    H2_CUDA(cudaStreamSynchronize(s));
  }
  H2_CUDA(cudaStreamSynchronize(s));
}

void build_f32_copies(Matrix& M) {
  if (!M.with_f32) return;
  cudaStream_t s = M.stream;
  auto conv = [&](const DevBuf& src, DevBuf& dst, int64_t nblk, int K) {
    dst.bytes = pool_bytes(nblk, K, FMT_F32);
    dst.p = M.alloc(dst.bytes);
    chunked(nblk, [&](int64_t b0, int nb) {
      { k_convert_pool<<<nb, 256, 0, s>>>((const char*)src.p + pool_bytes(b0, K, M.fmt), M.fmt,
                                        (char*)dst.p + pool_bytes(b0, K, FMT_F32), FMT_F32, K); ::h2mg::count_launch(); }
      H2_LAUNCH_CHECK();
    });
  };
  conv(M.poolD, M.poolD32, M.nD, M.KD);
  if (M.tstar >= 0) {
    conv(M.poolS, M.poolS32, M.nS, M.KC);
    M.poolP32.assign(M.poolP.size(), {});
    for (size_t i = 2; i < M.poolP.size(); ++i) conv(M.poolP[i], M.poolP32[i], M.nP[i], M.KC);
    int64_t nu = (int64_t)(1 << M.L) * M.KD * M.KC, ne = (int64_t)M.nslots() * M.KC * M.KC;
    M.d_U32 = (float*)M.alloc(sizeof(float) * nu);
    M.d_E32 = (float*)M.alloc(sizeof(float) * ne);
    { k_to_f32<<<ceil_div(nu, 256), 256, 0, s>>>(M.d_U, M.d_U32, nu); ::h2mg::count_launch(); }
    H2_LAUNCH_CHECK();
    { k_to_f32<<<ceil_div(ne, 256), 256, 0, s>>>(M.d_E, M.d_E32, ne); ::h2mg::count_launch(); }
    H2_LAUNCH_CHECK();
  }
  H2_CUDA(cudaStreamSynchronize(s));
}

}  // namespace h2mg
