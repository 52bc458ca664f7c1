// skeleton.cu -- nested cluster bases by recursive skeletonization (interpolative
// decompositions), the tolerance-driven alternative to Chebyshev interpolation.
//
// The paper's H2 matrices come from an algebraic construction to a relative accuracy
// eps with adaptive ranks (Sec. 4.1, "relative accuracy 1e-9"). Here every cluster
// tau gets a skeleton, a subset of its points whose matrix rows interpolate the
// cluster's far-field rows:
//     A(X_tau, F_tau) ~= T_tau A(skel_tau, F_tau),   T_tau[skel_tau, :] = I.
// Skeletons are nested: a leaf chooses among its points, a parent among the union of
// its children's skeletons (the candidates, first child first). The factors play the
// roles of the Chebyshev ones -- leaf basis U = T_leaf, transfer E_c = the rows of
// T_parent belonging to child c's skeleton, coupling S^0 = A(skel_tau, skel_sigma) --
// and the QR chain of fill.cu orthonormalises them unchanged.
//
// Per cluster tau at tree level ell (levels L down to t*, one launch per level):
//  1. the far-field sample F_tau: the candidates of every far partner of tau at
//     level ell, then, for every far partner sigma' of tau's parent, the candidates
//     of sigma''s two children concatenated and thinned to every s-th entry from the
//     first, s = ceil(count / 128);
//  2. R0 = the R factor of W = A(F_tau, candidates): the sampled rows are generated
//     in chunks of 32 and folded into an upper-triangular R in shared memory by
//     Householder reflections that touch only row j of R and the chunk (a
//     tall-skinny QR; W itself is never stored);
//  3. greedy column-pivoted Householder QR of R0 (the column of largest remaining
//     norm; columns within a relative 1e-10 of the largest squared norm are tied and
//     the lowest index wins), stopped at rank_max, at min(rows, candidates), or once
//     the best remaining norm is <= tol * the first pivot's norm;
//  4. T[pivot a] = e_a for the r pivots and T[pivot r + b] = (R11^{-1} R12)[:, b].
// A cluster with an empty sample keeps its first min(candidates, rank_max)
// candidates with T = [I; 0].
#include <algorithm>
#include <cmath>

#include "internal.h"

namespace h2mg {

constexpr int SK_CAND = 128;        // candidates of a cluster at most (two skeletons of <= 64)
constexpr int SK_CHUNK = 32;        // sampled rows folded into R at a time (one per lane)
constexpr int SK_SAMPLE_CAP = 128;  // points kept per far partner of the parent
constexpr double SK_TIE = 1e-10;    // relative tie band of the pivot choice

// Sum over the 32 lanes of a warp.
__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide max / min helpers (blockDim.x == 256); red has >= 8 entries.
__device__ double block_max(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double m = red[0];
  for (int i = 1; i < 8; ++i) m = fmax(m, red[i]);
  __syncthreads();
  return m;
}
__device__ int block_min_int(int v, int* red) {
  for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  int m = red[0];
  for (int i = 1; i < 8; ++i) m = min(m, red[i]);
  __syncthreads();
  return m;
}

// One CTA (256 threads) per cluster of the level.
//   cand   [ncl][SK_CAND]: candidate tree positions, ncand[ncl] of them
//   samp   sampled tree positions of all clusters, cluster c at samp[soff[c] .. soff[c+1])
//   out:   skel[ncl][64] (tree positions, pivot order), rank[ncl], T[ncl][SK_CAND x 64]
//          (rows = candidates in their original order, column-major, ld SK_CAND)
__global__ void __launch_bounds__(256, 1) k_skeletonize(const int* __restrict__ cand, const int* __restrict__ ncand,
                                                       const int* __restrict__ samp, const int64_t* __restrict__ soff,
                                                       const double* __restrict__ X, const double* __restrict__ sw,
                                                       int dim, KernelParams kp, double tol, int rank_max,
                                                       int* __restrict__ skel, int* __restrict__ rank_out,
                                                       double* __restrict__ Tout) {
  extern __shared__ double sm[];
  double* R = sm;                                  // SK_CAND x SK_CAND, column-major, ld SK_CAND
  double* C = R + SK_CAND * SK_CAND;               // SK_CHUNK x SK_CAND, column-major, ld SK_CHUNK
  double* cx = C + SK_CHUNK * SK_CAND;             // candidate coordinates [SK_CAND][3]
  double* cw = cx + SK_CAND * 3;                   // candidate sqrt(w)
  double* nrm = cw + SK_CAND;                      // column norms (pivoting)
  double* red = nrm + SK_CAND;                     // 8 reduction slots
  double* bcast = red + 8;                         // 4 broadcast slots
  int* piv = (int*)(bcast + 4);                    // SK_CAND
  int* ired = piv + SK_CAND;                       // 8
  const int c = blockIdx.x;
  const int nc = ncand[c];
  const int* cd = cand + (int64_t)c * SK_CAND;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t s0 = soff[c], s1 = soff[c + 1];
  const int64_t m = s1 - s0;
  for (int i = threadIdx.x; i < nc; i += blockDim.x) {
    const int p = cd[i];
    for (int d = 0; d < dim; ++d) cx[i * 3 + d] = X[(int64_t)p * dim + d];
    cw[i] = sw[p];
    piv[i] = i;
  }
  for (int i = threadIdx.x; i < SK_CAND * SK_CAND; i += blockDim.x) R[i] = 0.0;
  __syncthreads();
  int r = 0;
  if (m > 0 && nc > 0) {
    // ---- 2. tall-skinny QR of the sampled rows, SK_CHUNK rows at a time
    for (int64_t q0 = 0; q0 < m; q0 += SK_CHUNK) {
      for (int e = threadIdx.x; e < SK_CHUNK * nc; e += blockDim.x) {
        const int i = e % SK_CHUNK, k = e / SK_CHUNK;
        double v = 0.0;
        if (q0 + i < m) {
          const int f = samp[s0 + q0 + i];
          v = sw[f] * kernel_eval(kp, X + (int64_t)f * dim, cx + k * 3, dim) * cw[k];
        }
        C[i + k * SK_CHUNK] = v;
      }
      __syncthreads();
      for (int j = 0; j < nc; ++j) {
        const double cij = C[lane + j * SK_CHUNK];
        const double sigma = warp_sum(cij * cij);
        const double alpha = R[j + j * SK_CAND];
        if (sigma > 0.0) {
          const double beta = -copysign(sqrt(alpha * alpha + sigma), alpha);
          const double tau = (beta - alpha) / beta;
          const double vi = cij / (alpha - beta);
          for (int k = j + 1 + w; k < nc; k += 8) {
            const double ck = C[lane + k * SK_CHUNK];
            const double wk = tau * (R[j + k * SK_CAND] + warp_sum(vi * ck));
            if (lane == 0) R[j + k * SK_CAND] -= wk;
            C[lane + k * SK_CHUNK] = ck - wk * vi;
          }
          __syncthreads();
          if (threadIdx.x == 0) R[j + j * SK_CAND] = beta;
        } else {
          __syncthreads();
        }
      }
      __syncthreads();
    }
    // ---- 3. greedy column-pivoted Householder QR of R0 (rows: min(m, nc))
    const int rows = (int)std::min<int64_t>(m, nc);
    const int kmax = min(rank_max, min(rows, nc));
    double first = 0.0;
    for (int j = 0; j < kmax; ++j) {
      for (int k = j + threadIdx.x; k < nc; k += blockDim.x) {
        double s = 0.0;
        for (int i = j; i < nc; ++i) s = fma(R[i + k * SK_CAND], R[i + k * SK_CAND], s);
        nrm[k] = s;
      }
      __syncthreads();
      double mv = -1.0;
      for (int k = j + threadIdx.x; k < nc; k += blockDim.x) mv = fmax(mv, nrm[k]);
      const double big = block_max(mv, red);
      if (j == 0) {
        first = sqrt(big);
        if (first == 0.0) break;
      } else if (sqrt(big) <= tol * first) {
        break;
      }
      int cand_k = 1 << 30;
      for (int k = j + threadIdx.x; k < nc; k += blockDim.x)
        if (nrm[k] >= big * (1.0 - SK_TIE)) cand_k = min(cand_k, k);
      const int p = block_min_int(cand_k, ired);
      if (p != j) {
        for (int i = threadIdx.x; i < nc; i += blockDim.x) {
          const double t = R[i + j * SK_CAND];
          R[i + j * SK_CAND] = R[i + p * SK_CAND];
          R[i + p * SK_CAND] = t;
        }
        if (threadIdx.x == 0) {
          const int t = piv[j];
          piv[j] = piv[p];
          piv[p] = t;
        }
        __syncthreads();
      }
      // reflector of R[j:, j]
      if (threadIdx.x == 0) {
        const double alpha = R[j + j * SK_CAND];
        double sigma = 0.0;
        for (int i = j + 1; i < nc; ++i) sigma = fma(R[i + j * SK_CAND], R[i + j * SK_CAND], sigma);
        double beta = alpha, tau = 0.0, scale = 0.0;
        if (sigma > 0.0) {
          beta = -copysign(sqrt(alpha * alpha + sigma), alpha);
          tau = (beta - alpha) / beta;
          scale = 1.0 / (alpha - beta);
        }
        bcast[0] = beta;
        bcast[1] = tau;
        bcast[2] = scale;
      }
      __syncthreads();
      const double beta = bcast[0], tau = bcast[1], scale = bcast[2];
      if (tau != 0.0) {
        for (int i = j + 1 + threadIdx.x; i < nc; i += blockDim.x) R[i + j * SK_CAND] *= scale;
        __syncthreads();
        for (int k = j + 1 + threadIdx.x; k < nc; k += blockDim.x) {
          double wk = R[j + k * SK_CAND];
          for (int i = j + 1; i < nc; ++i) wk = fma(R[i + j * SK_CAND], R[i + k * SK_CAND], wk);
          wk *= tau;
          R[j + k * SK_CAND] -= wk;
          for (int i = j + 1; i < nc; ++i) R[i + k * SK_CAND] = fma(-wk, R[i + j * SK_CAND], R[i + k * SK_CAND]);
        }
        __syncthreads();
        if (threadIdx.x == 0) R[j + j * SK_CAND] = beta;
        for (int i = j + 1 + threadIdx.x; i < nc; i += blockDim.x) R[i + j * SK_CAND] = 0.0;
      }
      __syncthreads();
      r = j + 1;
    }
    r = max(r, 1);
    // ---- 4. R11^{-1} R12 by back substitution, one thread per column of R12
    if (R[0] != 0.0) {
      for (int b = r + threadIdx.x; b < nc; b += blockDim.x) {
        for (int a = r - 1; a >= 0; --a) {
          double v = R[a + b * SK_CAND];
          for (int a2 = a + 1; a2 < r; ++a2) v = fma(-R[a + a2 * SK_CAND], R[a2 + b * SK_CAND], v);
          R[a + b * SK_CAND] = v / R[a + a * SK_CAND];
        }
      }
    } else {
      for (int b = r + threadIdx.x; b < nc; b += blockDim.x)
        for (int a = 0; a < r; ++a) R[a + b * SK_CAND] = 0.0;
    }
    __syncthreads();
  } else {
    r = min(nc, rank_max);   // empty sample: the first candidates, T = [I; 0]
  }
  // ---- outputs
  double* Tc = Tout + (int64_t)c * SK_CAND * 64;
  for (int e = threadIdx.x; e < SK_CAND * 64; e += blockDim.x) Tc[e] = 0.0;
  __syncthreads();
  const bool id = (m > 0 && nc > 0);
  for (int e = threadIdx.x; e < nc * r; e += blockDim.x) {
    const int k = e % nc, a = e / nc;   // pivot position k, column a
    double v;
    if (k < r) v = (k == a) ? 1.0 : 0.0;
    else v = id ? R[a + k * SK_CAND] : 0.0;
    Tc[piv[k] + a * SK_CAND] = v;
  }
  for (int a = threadIdx.x; a < 64; a += blockDim.x) skel[(int64_t)c * 64 + a] = a < r ? cd[piv[a]] : -1;
  if (threadIdx.x == 0) rank_out[c] = r;
}

// Candidates of the clusters of level ell (< L): the skeleton of child 2j, then that
// of child 2j + 1 (ranks rk of level ell + 1).
__global__ void k_skel_cand(const int* __restrict__ skel_child, const int* __restrict__ rk_child, int ncl,
                            int* __restrict__ cand, int* __restrict__ ncand) {
  const int j = blockIdx.x;
  if (j >= ncl) return;
  const int r1 = rk_child[2 * j], r2 = rk_child[2 * j + 1];
  for (int i = threadIdx.x; i < r1 + r2; i += blockDim.x)
    cand[(int64_t)j * SK_CAND + i] =
        i < r1 ? skel_child[(int64_t)(2 * j) * 64 + i] : skel_child[(int64_t)(2 * j + 1) * 64 + i - r1];
  if (threadIdx.x == 0) ncand[j] = r1 + r2;
}

// Candidates of the leaves: their points in tree order.
__global__ void k_skel_cand_leaf(const int* __restrict__ leafoff, int* __restrict__ cand, int* __restrict__ ncand) {
  const int j = blockIdx.x;
  const int p0 = leafoff[j], nl = leafoff[j + 1] - p0;
  for (int i = threadIdx.x; i < nl; i += blockDim.x) cand[(int64_t)j * SK_CAND + i] = p0 + i;
  if (threadIdx.x == 0) ncand[j] = nl;
}

// Sample positions of every cluster, from a list of (destination offset, source
// cluster, kind) segments: kind 0 = all candidates of cluster src; kind s >= 1 = the
// candidates of clusters 2 src and 2 src + 1 concatenated, every s-th from the first.
struct SampleSeg {
  int64_t dst;
  int src;
  int kind;
};
__global__ void k_skel_samples(const SampleSeg* __restrict__ seg, int nseg, const int* __restrict__ cand,
                               const int* __restrict__ ncand, int* __restrict__ samp) {
  const int g = blockIdx.x;
  if (g >= nseg) return;
  const SampleSeg S = seg[g];
  if (S.kind == 0) {
    const int nn = ncand[S.src];
    for (int i = threadIdx.x; i < nn; i += blockDim.x) samp[S.dst + i] = cand[(int64_t)S.src * SK_CAND + i];
  } else {
    const int a = 2 * S.src, b = 2 * S.src + 1;
    const int na = ncand[a], nb = ncand[b];
    const int cnt = (na + nb + S.kind - 1) / S.kind;
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
      const int k = i * S.kind;
      samp[S.dst + i] = k < na ? cand[(int64_t)a * SK_CAND + k] : cand[(int64_t)b * SK_CAND + k - na];
    }
  }
}

// Skeleton coordinates and sqrt(w) of every slot (the coupling points of k_fill_S).
__global__ void k_skel_nodes(const int* __restrict__ skel, const int* __restrict__ rank, int nsl, int KC, int dim,
                             const double* __restrict__ X, const double* __restrict__ sw, double* __restrict__ nodes,
                             double* __restrict__ nsw) {
  const int t = blockIdx.x;
  if (t >= nsl) return;
  const int r = rank[t];
  for (int a = threadIdx.x; a < KC; a += blockDim.x) {
    const int p = a < r ? skel[(int64_t)t * 64 + a] : -1;
    for (int d = 0; d < dim; ++d) nodes[((int64_t)t * KC + a) * dim + d] = p >= 0 ? X[(int64_t)p * dim + d] : 0.0;
    nsw[(int64_t)t * KC + a] = p >= 0 ? sw[p] : 0.0;
  }
}

size_t skeleton_smem_bytes() {
  return sizeof(double) * ((size_t)SK_CAND * SK_CAND + SK_CHUNK * SK_CAND + SK_CAND * 3 + SK_CAND + SK_CAND + 8 + 4) +
         sizeof(int) * (SK_CAND + 8);
}

// Skeletons of every cluster at levels t*..L, bottom-up, into M.d_skel (slot-indexed,
// 64 per slot), M.d_Tid (slot-indexed, SK_CAND x 64) and M.h_rank / M.d_rank.
void build_skeletons(Matrix& M) {
  cudaStream_t s = M.stream;
  const int L = M.L, ts = M.tstar;
  const int nsl = M.nslots();
  M.d_skel = (int*)M.alloc(sizeof(int) * (size_t)nsl * 64);
  M.tid.bytes = sizeof(double) * (size_t)nsl * SK_CAND * 64;
  M.tid.p = M.alloc(M.tid.bytes);
  M.h_rank.assign(nsl, 0);
  M.d_rank = (int*)M.alloc(sizeof(int) * nsl);
  const size_t smem = skeleton_smem_bytes();
  H2_CUDA(cudaFuncSetAttribute(k_skeletonize, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  // candidates of two consecutive levels (this one and the one below)
  std::vector<int> ncand_h;                      // of level ell
  int* d_cand = (int*)M.alloc(sizeof(int) * ((size_t)1 << L) * SK_CAND);
  int* d_ncand = (int*)M.alloc(sizeof(int) * ((size_t)1 << L));
  std::vector<int> partners_own, partners_par;
  for (int ell = L; ell >= ts; --ell) {
    const int ncl = 1 << ell;
    if (ell == L) {
      { k_skel_cand_leaf<<<ncl, 64, 0, s>>>(M.d_leafoff, d_cand, d_ncand); ::h2mg::count_launch(); }
      H2_LAUNCH_CHECK();
      ncand_h.assign(ncl, 0);
      for (int j = 0; j < ncl; ++j) ncand_h[j] = M.offsets[L][j + 1] - M.offsets[L][j];
    } else {
      { k_skel_cand<<<ncl, 128, 0, s>>>(M.d_skel + (size_t)M.slot0(ell + 1) * 64, M.d_rank + M.slot0(ell + 1), ncl,
                                        d_cand, d_ncand); ::h2mg::count_launch(); }
      H2_LAUNCH_CHECK();
      ncand_h.assign(ncl, 0);
      for (int j = 0; j < ncl; ++j)
        ncand_h[j] = M.h_rank[M.slot0(ell + 1) + 2 * j] + M.h_rank[M.slot0(ell + 1) + 2 * j + 1];
    }
    // sample segments: own far partners, then the parent's far partners (thinned)
    std::vector<SampleSeg> segs;
    std::vector<int64_t> soff(ncl + 1, 0);
    const HostCSR& F = M.far[ell];
    const HostCSR* Fp = (ell - 1 >= ts) ? &M.far[ell - 1] : nullptr;
    int64_t tot = 0;
    for (int j = 0; j < ncl; ++j) {
      soff[j] = tot;
      for (int e = F.rowptr[j]; e < F.rowptr[j + 1]; ++e) {
        const int sg = F.col[e];
        segs.push_back({tot, sg, 0});
        tot += ncand_h[sg];
      }
      if (Fp) {
        const int pj = j >> 1;
        for (int e = Fp->rowptr[pj]; e < Fp->rowptr[pj + 1]; ++e) {
          const int sg = Fp->col[e];
          const int cnt = ncand_h[2 * sg] + ncand_h[2 * sg + 1];
          const int step = std::max(1, (cnt + SK_SAMPLE_CAP - 1) / SK_SAMPLE_CAP);
          segs.push_back({tot, sg, step});
          tot += (cnt + step - 1) / step;
        }
      }
    }
    soff[ncl] = tot;
    int* d_samp = (int*)M.alloc(sizeof(int) * std::max<int64_t>(tot, 1));
    int64_t* d_soff = (int64_t*)M.alloc(sizeof(int64_t) * (ncl + 1));
    SampleSeg* d_seg = (SampleSeg*)M.alloc(sizeof(SampleSeg) * std::max<size_t>(segs.size(), 1));
    H2_CUDA(cudaMemcpyAsync(d_soff, soff.data(), sizeof(int64_t) * (ncl + 1), cudaMemcpyHostToDevice, s));
    if (!segs.empty()) {
      H2_CUDA(cudaMemcpyAsync(d_seg, segs.data(), sizeof(SampleSeg) * segs.size(), cudaMemcpyHostToDevice, s));
      const int64_t CH = 1 << 20;
      for (int64_t g0 = 0; g0 < (int64_t)segs.size(); g0 += CH) {
        const int ng = (int)std::min<int64_t>(CH, (int64_t)segs.size() - g0);
        { k_skel_samples<<<ng, 128, 0, s>>>(d_seg + g0, ng, d_cand, d_ncand, d_samp); ::h2mg::count_launch(); }
        H2_LAUNCH_CHECK();
      }
    }
    { k_skeletonize<<<ncl, 256, smem, s>>>(d_cand, d_ncand, d_samp, d_soff, M.d_X, M.d_sw, M.dim, M.kp, M.basis_tol,
                                          M.k, M.d_skel + (size_t)M.slot0(ell) * 64, M.d_rank + M.slot0(ell),
                                          (double*)M.tid.p + (size_t)M.slot0(ell) * SK_CAND * 64);
      ::h2mg::count_launch(); }
    H2_LAUNCH_CHECK();
    H2_CUDA(cudaMemcpyAsync(M.h_rank.data() + M.slot0(ell), M.d_rank + M.slot0(ell), sizeof(int) * ncl,
                            cudaMemcpyDeviceToHost, s));
    H2_CUDA(cudaStreamSynchronize(s));
    M.free_owned(d_samp);
    M.free_owned(d_soff);
    M.free_owned(d_seg);
  }
  M.free_owned(d_cand);
  M.free_owned(d_ncand);
  // coupling points: skeleton coordinates and sqrt(w), KC per slot
  M.d_nodes = (double*)M.alloc(sizeof(double) * (size_t)nsl * M.KC * M.dim);
  M.d_nsw = (double*)M.alloc(sizeof(double) * (size_t)nsl * M.KC);
  { k_skel_nodes<<<nsl, 64, 0, s>>>(M.d_skel, M.d_rank, nsl, M.KC, M.dim, M.d_X, M.d_sw, M.d_nodes, M.d_nsw);
    ::h2mg::count_launch(); }
  H2_LAUNCH_CHECK();
  H2_CUDA(cudaStreamSynchronize(s));
}

}  // namespace h2mg
