// dense.cu -- the coarsest operator A_l as a dense matrix, its Cholesky factor and
// the coarse solve e_l = dir_sol(A_l, r_l) (Sec. 3.3, Algorithm 1).
//
// A_l acts on the coefficients of tree level m = m(l). Its coupling part is the H2
// chain of levels t*..m expanded densely: G_{t*} holds the far blocks of level t*,
// G_{ell+1} = T_ell G_ell T_ell^T + (far blocks of level ell+1) with T_ell the
// block-diagonal orthonormal transfers, and A_l = G_m + P_l. For l = 1 (no far
// field, or a forced single level) A_1 = D + U_1 G_L U_1^T on the point slots.
// Padded slots (beyond a cluster's rank or a leaf's size) get a unit diagonal so
// the factor exists; they are zero in every right-hand side.
#include <algorithm>
#include <cmath>

#include "internal.h"

namespace h2mg {

__device__ void unswz_d(int pos, int K, int V, int& i, int& j) {
  int LPC = K / 8, CPP = 32 / LPC, P = 8 / V;
  int sub = pos % V;
  int lane = (pos / V) % 32;
  int tk = pos / (V * 32);
  int t = tk / P, k = tk % P;
  i = 8 * (lane % LPC) + k * V + sub;
  j = t * CPP + lane / LPC;
}

__device__ __forceinline__ double load_elem_d(const void* pool, int fmt, int64_t idx) {
  if (fmt == FMT_F64) return ((const double*)pool)[idx];
  if (fmt == FMT_DF) {
    float2 v = ((const float2*)pool)[idx];
    return (double)v.x + (double)v.y;
  }
  return (double)((const float*)pool)[idx];
}

// dense[t*K + i, s*K + j] += B_ts[i, j] (and the transpose for t != s)
__global__ void k_scatter(const int* __restrict__ pt, const int* __restrict__ ps,
                          const void* __restrict__ pool, int fmt, int K, double* __restrict__ G,
                          int64_t n) {
  int64_t b = blockIdx.x;
  int t = pt[b], s = ps[b];
  int V = fmt == FMT_F32 ? 4 : 2;
  for (int pos = threadIdx.x; pos < K * K; pos += blockDim.x) {
    int i, j;
    unswz_d(pos, K, V, i, j);
    double v = load_elem_d(pool, fmt, b * K * K + pos);
    int64_t r = (int64_t)t * K + i, c = (int64_t)s * K + j;
    G[r + c * n] += v;
    if (t != s) G[c + r * n] += v;
  }
}

// out block (a, a') = B_a G(p(a), p(a')) B_a'^T, B_a of size Ra x C (column-major),
// G of order nc = 2^ell * C, out of order no = 2^(ell+1) * Ra.
__global__ void k_expand(const double* __restrict__ G, int64_t nc, const double* __restrict__ B,
                         int Ra, int C, int ncl_out, int shift, double* __restrict__ out, int64_t no) {
  extern __shared__ double sm[];
  double* Gb = sm;            // C x C
  double* T = Gb + C * C;     // C x Ra
  int a = blockIdx.x % ncl_out, ap = blockIdx.x / ncl_out;
  int pa = a >> shift, pap = ap >> shift;   // shift 1: parent cluster; 0: same cluster
  for (int e = threadIdx.x; e < C * C; e += blockDim.x) {
    int i = e % C, j = e / C;
    Gb[e] = G[((int64_t)pa * C + i) + ((int64_t)pap * C + j) * nc];
  }
  __syncthreads();
  const double* Ba = B + (int64_t)a * Ra * C;
  const double* Bap = B + (int64_t)ap * Ra * C;
  // T[b][j] = sum_c Gb[b][c] Bap[j][c]
  for (int e = threadIdx.x; e < C * Ra; e += blockDim.x) {
    int bb = e % C, j = e / C;
    double v = 0.0;
    for (int c = 0; c < C; ++c) v += Gb[bb + c * C] * Bap[j + c * Ra];
    T[e] = v;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < Ra * Ra; e += blockDim.x) {
    int i = e % Ra, j = e / Ra;
    double v = 0.0;
    for (int bb = 0; bb < C; ++bb) v += Ba[i + bb * Ra] * T[bb + j * C];
    out[((int64_t)a * Ra + i) + ((int64_t)ap * Ra + j) * no] = v;
  }
}

__global__ void k_pad_diag(double* __restrict__ A, int64_t n, const unsigned char* __restrict__ valid) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && !valid[i]) A[i + i * n] = 1.0;
}

// ----------------------------------------------------------------------------- Cholesky
constexpr int NB = 32;

__global__ void k_potrf_diag(double* __restrict__ A, int64_t n, int k0, int nb, int* __restrict__ flag) {
  __shared__ double S[NB * NB];
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
    int i = e % nb, j = e / nb;
    S[e] = A[(k0 + i) + (int64_t)(k0 + j) * n];
  }
  __syncthreads();
  for (int j = 0; j < nb; ++j) {
    double d = S[j + j * nb];
    if (!(d > 0.0)) {
      if (threadIdx.x == 0) atomicOr(flag, 1);
      d = 1.0;
    }
    double ljj = sqrt(d);
    __syncthreads();
    if (threadIdx.x == 0) S[j + j * nb] = ljj;
    for (int i = j + 1 + threadIdx.x; i < nb; i += blockDim.x) S[i + j * nb] /= ljj;
    __syncthreads();
    for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
      int i = e % nb, c = e / nb;
      if (c > j && i >= c) S[i + c * nb] -= S[i + j * nb] * S[c + j * nb];
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
    int i = e % nb, j = e / nb;
    if (i >= j) A[(k0 + i) + (int64_t)(k0 + j) * n] = S[e];
  }
}

// Rows below the diagonal block: L21 = A21 L11^{-T} (one thread per row).
__global__ void k_trsm_panel(double* __restrict__ A, int64_t n, int k0, int nb) {
  __shared__ double L11[NB * NB];
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
    int i = e % nb, j = e / nb;
    L11[e] = A[(k0 + i) + (int64_t)(k0 + j) * n];
  }
  __syncthreads();
  int64_t i = (int64_t)k0 + nb + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int j = 0; j < nb; ++j) {
    double v = A[i + (int64_t)(k0 + j) * n];
    for (int t = 0; t < j; ++t) v -= A[i + (int64_t)(k0 + t) * n] * L11[j + t * nb];
    A[i + (int64_t)(k0 + j) * n] = v / L11[j + j * nb];
  }
}

// Trailing update of the lower triangle: A22 -= L21 L21^T, 64 x 64 tiles.
__global__ void k_syrk_update(double* __restrict__ A, int64_t n, int k0, int nb, int tiles) {
  int bi = blockIdx.x % tiles, bj = blockIdx.x / tiles;
  if (bj > bi) return;
  __shared__ double Li[64 * NB], Lj[64 * NB];
  int64_t r0 = (int64_t)k0 + nb + (int64_t)bi * 64, c0 = (int64_t)k0 + nb + (int64_t)bj * 64;
  for (int e = threadIdx.x; e < 64 * nb; e += blockDim.x) {
    int i = e % 64, t = e / 64;
    Li[e] = (r0 + i < n) ? A[(r0 + i) + (int64_t)(k0 + t) * n] : 0.0;
    Lj[e] = (c0 + i < n) ? A[(c0 + i) + (int64_t)(k0 + t) * n] : 0.0;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < 64 * 64; e += blockDim.x) {
    int i = e % 64, j = e / 64;
    int64_t r = r0 + i, c = c0 + j;
    if (r < n && c < n && r >= c) {
      double v = 0.0;
      for (int t = 0; t < nb; ++t) v += Li[i + t * 64] * Lj[j + t * 64];
      A[r + c * n] -= v;
    }
  }
}

// ----------------------------------------------------------------------------- inverse
// A_l^{-1} from the Cholesky factor, by substitution on the identity, all columns at
// once: L Y = I (forward, block row by block row), then L^T X = Y (backward). Each
// step solves the NB x NB diagonal block for every column (one thread per column),
// then updates the remaining rows with a 64 x 64-tiled product.
__global__ void k_inv_diag(const double* __restrict__ L, int64_t n, int k0, int nb, int fwd,
                           double* __restrict__ B) {
  __shared__ double Lk[NB * NB];
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
    int i = e % nb, j = e / nb;
    Lk[e] = L[(k0 + i) + (int64_t)(k0 + j) * n];
  }
  __syncthreads();
  int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  double v[NB];
  for (int i = 0; i < nb; ++i) v[i] = B[(k0 + i) + c * n];
  if (fwd) {
    for (int i = 0; i < nb; ++i) {
      double t = v[i];
      for (int j = 0; j < i; ++j) t -= Lk[i + j * nb] * v[j];
      v[i] = t / Lk[i + i * nb];
    }
  } else {
    for (int i = nb - 1; i >= 0; --i) {
      double t = v[i];
      for (int j = i + 1; j < nb; ++j) t -= Lk[j + i * nb] * v[j];
      v[i] = t / Lk[i + i * nb];
    }
  }
  for (int i = 0; i < nb; ++i) B[(k0 + i) + c * n] = v[i];
}

// fwd: B[i, c] -= sum_t L[i, k0+t] B[k0+t, c] for i >= k0+nb;
// bwd: B[i, c] -= sum_t L[k0+t, i] B[k0+t, c] for i < k0.
__global__ void k_inv_update(const double* __restrict__ L, int64_t n, int k0, int nb, int fwd, int row0,
                             int rows, double* __restrict__ B) {
  __shared__ double Lp[64 * NB], Bb[NB * 64];
  int rt = blockIdx.x, ct = blockIdx.y;
  int64_t r0 = row0 + (int64_t)rt * 64, c0 = (int64_t)ct * 64;
  for (int e = threadIdx.x; e < 64 * nb; e += blockDim.x) {
    int i = e % 64, t = e / 64;
    int64_t r = r0 + i;
    double v = 0.0;
    if (r < row0 + rows) v = fwd ? L[r + (int64_t)(k0 + t) * n] : L[(k0 + t) + r * n];
    Lp[e] = v;
    int tt = e % nb, cc = e / nb;
    Bb[e] = (c0 + cc < n) ? B[(k0 + tt) + (c0 + cc) * n] : 0.0;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < 64 * 64; e += blockDim.x) {
    int i = e % 64, j = e / 64;
    int64_t r = r0 + i, c = c0 + j;
    if (r < row0 + rows && c < n) {
      double s = 0.0;
      for (int t = 0; t < nb; ++t) s += Lp[i + t * 64] * Bb[t + j * nb];
      B[r + c * n] -= s;
    }
  }
}

__global__ void k_identity(double* __restrict__ B, int64_t n) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n * n) B[e] = (e % n == e / n) ? 1.0 : 0.0;
}

// e[i] = sum_j Ainv[j, i] r[j]: one warp per output, reading column i (contiguous).
__global__ void k_symv_cols(const double* __restrict__ Ainv, int64_t n, const double* __restrict__ r,
                            double* __restrict__ e) {
  int64_t i = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  int lane = threadIdx.x & 31;
  if (i >= n) return;
  const double* col = Ainv + i * n;
  double s = 0.0;
  for (int64_t j = lane; j < n; j += 32) s = fma(col[j], r[j], s);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) e[i] = s;
}

// E[:, c] = A^{-1} R[:, c] for NR columns (leading dimension n): one warp per output
// row reads that column of the symmetric inverse once for all NR right-hand sides.
template <int NR>
__global__ void k_symv_multi(const double* __restrict__ Ainv, int64_t n, const double* __restrict__ r,
                             double* __restrict__ e) {
  int64_t i = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  int lane = threadIdx.x & 31;
  if (i >= n) return;
  const double* col = Ainv + i * n;
  double s[NR];
#pragma unroll
  for (int c = 0; c < NR; ++c) s[c] = 0.0;
  for (int64_t j = lane; j < n; j += 32) {
    const double a = col[j];
#pragma unroll
    for (int c = 0; c < NR; ++c) s[c] = fma(a, r[c * n + j], s[c]);
  }
#pragma unroll
  for (int c = 0; c < NR; ++c) {
    for (int o = 16; o > 0; o >>= 1) s[c] += __shfl_xor_sync(0xffffffffu, s[c], o);
    if (lane == 0) e[c * n + i] = s[c];
  }
}

static void build_inverse(Matrix& M) {
  cudaStream_t s = M.stream;
  int64_t n = M.nl;
  double* B = (double*)M.alloc(sizeof(double) * n * n);
  { k_identity<<<ceil_div(n * n, 256), 256, 0, s>>>(B, n); ::h2mg::count_launch(); }
  H2_LAUNCH_CHECK();
  int cgrid = ceil_div(n, 128);
  for (int k0 = 0; k0 < n; k0 += NB) {
    int nb = (int)std::min<int64_t>(NB, n - k0);
    { k_inv_diag<<<cgrid, 128, 0, s>>>(M.d_Al, n, k0, nb, 1, B); ::h2mg::count_launch(); }
    H2_LAUNCH_CHECK();
    int64_t rem = n - k0 - nb;
    if (rem > 0) {
      dim3 grid(ceil_div(rem, 64), ceil_div(n, 64));
      { k_inv_update<<<grid, 256, 0, s>>>(M.d_Al, n, k0, nb, 1, k0 + nb, (int)rem, B); ::h2mg::count_launch(); }
      H2_LAUNCH_CHECK();
    }
  }
  int last = (int)((n - 1) / NB) * NB;
  for (int k0 = last; k0 >= 0; k0 -= NB) {
    int nb = (int)std::min<int64_t>(NB, n - k0);
    { k_inv_diag<<<cgrid, 128, 0, s>>>(M.d_Al, n, k0, nb, 0, B); ::h2mg::count_launch(); }
    H2_LAUNCH_CHECK();
    if (k0 > 0) {
      dim3 grid(ceil_div(k0, 64), ceil_div(n, 64));
      { k_inv_update<<<grid, 256, 0, s>>>(M.d_Al, n, k0, nb, 0, 0, k0, B); ::h2mg::count_launch(); }
      H2_LAUNCH_CHECK();
    }
  }
  H2_CUDA(cudaStreamSynchronize(s));
  M.d_Ainv = B;
}

static void upload_i32(Matrix& M, const std::vector<int>& v, int** d) {
  *d = (int*)M.alloc(sizeof(int) * std::max<size_t>(v.size(), 1));
  if (!v.empty()) H2_CUDA(cudaMemcpyAsync(*d, v.data(), sizeof(int) * v.size(), cudaMemcpyHostToDevice, M.stream));
}

// Scatter the upper entries of a full level list (strict: far lists) from a pool.
static void scatter_level(Matrix& M, const HostCSR& C, int ncl, bool strict, const void* pool,
                          int64_t blk0, int K, double* G, int64_t n) {
  std::vector<int> pt, ps;
  for (int t = 0; t < ncl; ++t)
    for (int e = C.rowptr[t]; e < C.rowptr[t + 1]; ++e)
      if (strict ? C.col[e] > t : C.col[e] >= t) {
        pt.push_back(t);
        ps.push_back(C.col[e]);
      }
  if (pt.empty()) return;
  int *dt, *ds;
  upload_i32(M, pt, &dt);
  upload_i32(M, ps, &ds);
  const char* base = (const char*)pool + (size_t)blk0 * K * K * fmt_bytes(M.fmt);
  { k_scatter<<<(int)pt.size(), 256, 0, M.stream>>>(dt, ds, base, M.fmt, K, G, n); ::h2mg::count_launch(); }
  H2_LAUNCH_CHECK();
}

void build_dense_coarse(Matrix& M) {
  cudaStream_t s = M.stream;
  const int L = M.L, KC = M.KC, KD = M.KD;
  const int l = M.lev;
  double* G = nullptr;
  int64_t ng = 0;
  int mtop = (l == 1) ? L : L - l + 2;   // tree level whose coefficients the chain reaches
  if (M.tstar >= 0) {
    int ts = M.tstar;
    ng = (int64_t)(1 << ts) * KC;
    G = (double*)M.alloc(sizeof(double) * ng * ng);
    scatter_level(M, M.far[ts], 1 << ts, true, M.poolS.p, M.s_level_base[ts], KC, G, ng);
    size_t sm = sizeof(double) * 2 * KC * KC;
    H2_CUDA(cudaFuncSetAttribute(k_expand, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)std::max<size_t>(sm, sizeof(double) * (KC * KC + KC * KD))));
    for (int ell = ts; ell < mtop; ++ell) {
      int64_t nn = (int64_t)(1 << (ell + 1)) * KC;
      double* G2 = (double*)M.alloc(sizeof(double) * nn * nn);
      int ncl = 1 << (ell + 1);
      { k_expand<<<ncl * ncl, 256, sm, s>>>(G, ng, M.d_E + (size_t)M.slot0(ell + 1) * KC * KC, KC, KC, ncl,
                                          1, G2, nn); ::h2mg::count_launch(); }
      H2_LAUNCH_CHECK();
      scatter_level(M, M.far[ell + 1], ncl, true, M.poolS.p, M.s_level_base[ell + 1], KC, G2, nn);
      H2_CUDA(cudaStreamSynchronize(s));
      cudaFree(G);   // intermediate levels are released right away
      M.owned.erase(std::remove_if(M.owned.begin(), M.owned.end(), [&](const DevBuf& d) { return d.p == G; }),
                    M.owned.end());
      G = G2;
      ng = nn;
    }
  }
  std::vector<unsigned char> valid;
  if (l >= 2) {
    // A_l = G_m + P_l
    int m = mtop;
    M.nl = (int)ng;
    scatter_level(M, M.inadm[m], 1 << m, false, M.poolP[l].p, 0, KC, G, ng);
    valid.assign(ng, 0);
    for (int j = 0; j < (1 << m); ++j)
      for (int a = 0; a < M.h_rank[M.slot0(m) + j]; ++a) valid[(size_t)j * KC + a] = 1;
    M.d_Al = G;
  } else {
    // A_1 = D + U G_L U^T on the padded point slots
    int64_t np = (int64_t)(1 << L) * KD;
    H2_REQUIRE(np <= 16384, H2MG_ERR_UNSUPPORTED, "a single-level (dense) hierarchy needs n <= 16384");
    double* A1 = (double*)M.alloc(sizeof(double) * np * np);
    if (M.tstar >= 0) {
      int ncl = 1 << L;
      size_t sm = sizeof(double) * (KC * KC + KC * KD);
      { k_expand<<<ncl * ncl, 256, sm, s>>>(G, ng, M.d_U, KD, KC, ncl, 0, A1, np); ::h2mg::count_launch(); }
      H2_LAUNCH_CHECK();
    }
    M.nl = (int)np;
    valid.assign(np, 0);
    for (int j = 0; j < (1 << L); ++j)
      for (int i = 0; i < M.offsets[L][j + 1] - M.offsets[L][j]; ++i) valid[(size_t)j * KD + i] = 1;
    M.d_Al = A1;
    scatter_level(M, M.inadm[L], 1 << L, false, M.poolD.p, 0, KD, A1, np);
  }
  unsigned char* dv = (unsigned char*)M.alloc(valid.size());
  H2_CUDA(cudaMemcpyAsync(dv, valid.data(), valid.size(), cudaMemcpyHostToDevice, s));
  { k_pad_diag<<<ceil_div(M.nl, 256), 256, 0, s>>>(M.d_Al, M.nl, dv); ::h2mg::count_launch(); }
  H2_LAUNCH_CHECK();
  // Cholesky (lower), pivot check into d_flag
  H2_CUDA(cudaMemsetAsync(M.d_flag, 0, sizeof(int), s));
  int64_t n = M.nl;
  for (int k0 = 0; k0 < n; k0 += NB) {
    int nb = (int)std::min<int64_t>(NB, n - k0);
    { k_potrf_diag<<<1, 256, 0, s>>>(M.d_Al, n, k0, nb, M.d_flag); ::h2mg::count_launch(); }
    H2_LAUNCH_CHECK();
    int64_t rem = n - k0 - nb;
    if (rem > 0) {
      { k_trsm_panel<<<ceil_div(rem, 128), 128, 0, s>>>(M.d_Al, n, k0, nb); ::h2mg::count_launch(); }
      H2_LAUNCH_CHECK();
      int tiles = ceil_div(rem, 64);
      { k_syrk_update<<<tiles * tiles, 256, 0, s>>>(M.d_Al, n, k0, nb, tiles); ::h2mg::count_launch(); }
      H2_LAUNCH_CHECK();
    }
  }
  int flag = 0;
  H2_CUDA(cudaMemcpyAsync(&flag, M.d_flag, sizeof(int), cudaMemcpyDeviceToHost, s));
  H2_CUDA(cudaStreamSynchronize(s));
  M.coarse_ok = (flag == 0);
  if (M.coarse_ok) build_inverse(M);
  M.wcoarse.bytes = sizeof(double) * 3 * (size_t)M.nl;
  M.wcoarse.p = M.alloc(M.wcoarse.bytes);
}

__global__ void k_to_slots(const double* __restrict__ v, const int* __restrict__ slot_of, int64_t n,
                           double* __restrict__ out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[slot_of[i]] = v[i];
}
__global__ void k_from_slots(const double* __restrict__ v, const int* __restrict__ slot_of, int64_t n,
                             double* __restrict__ out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = v[slot_of[i]];
}

// e = A_l^{-1} r, with A_l^{-1} formed from the Cholesky factor at build time: one
// warp per output reads one column of the (symmetric) inverse. For l = 1 the vectors
// are in user point order and are mapped to and from the padded point slots.
void coarse_solve(Matrix& M, const double* r, double* e, cudaStream_t s) {
  int64_t n = M.nl;
  double* w = (double*)M.wcoarse.p;
  double* x = w + n;
  const double* rin = r;
  double* eout = e;
  if (M.lev == 1) {
    H2_CUDA(cudaMemsetAsync(w, 0, sizeof(double) * n, s));
    { k_to_slots<<<ceil_div(M.n, 256), 256, 0, s>>>(r, M.d_slot_of, M.n, w); ::h2mg::count_launch(); }
    H2_LAUNCH_CHECK();
    rin = w;
    eout = x;
  } else if (r == e) {
    H2_CUDA(cudaMemcpyAsync(w, r, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    rin = w;
  }
  { k_symv_cols<<<ceil_div(n, 8), 256, 0, s>>>(M.d_Ainv, n, rin, eout); ::h2mg::count_launch(); }
  H2_LAUNCH_CHECK();
  if (M.lev == 1) {
    { k_from_slots<<<ceil_div(M.n, 256), 256, 0, s>>>(x, M.d_slot_of, M.n, e); ::h2mg::count_launch(); }
    H2_LAUNCH_CHECK();
  }
}

// The coarse solve for nr columns of the coarsest level (leading dimension nl); r and
// e must not overlap. Level l = 1 (the whole matrix is dense) goes column by column.
void coarse_solve_multi(Matrix& M, const double* r, double* e, int nr, cudaStream_t s) {
  const int64_t n = M.nl;
  if (M.lev == 1) {
    for (int c = 0; c < nr; ++c) coarse_solve(M, r + c * M.n, e + c * M.n, s);
    return;
  }
  const int g = ceil_div(n, 8);
  switch (nr) {
    case 1: { k_symv_multi<1><<<g, 256, 0, s>>>(M.d_Ainv, n, r, e); ::h2mg::count_launch(); } break;
    case 2: { k_symv_multi<2><<<g, 256, 0, s>>>(M.d_Ainv, n, r, e); ::h2mg::count_launch(); } break;
    case 3: { k_symv_multi<3><<<g, 256, 0, s>>>(M.d_Ainv, n, r, e); ::h2mg::count_launch(); } break;
    case 4: { k_symv_multi<4><<<g, 256, 0, s>>>(M.d_Ainv, n, r, e); ::h2mg::count_launch(); } break;
    default: throw Error{H2MG_ERR_INVALID_ARG, "too many columns for one coarse solve"};
  }
  H2_LAUNCH_CHECK();
}

}  // namespace h2mg
