// tree.cu -- cluster tree (KD bisection at the median) and the block partition into
// close and far pairs, level by level (Sec. 3.1: close blocks D_ij, far blocks U_i S_ij V_j).
//
// Tree: every cluster above depth L = ceil(log2(n / leaf)) is split along the axis of
// largest tight-box extent (ties: lowest axis); its points are ordered by
// (coordinate, original index) and the first ceil(n/2) form the left child. Each
// level is one stable LSD radix sort of the original indices by the key
// (cluster, coordinate), starting from index order, so ties in the coordinate fall
// back to the original index.
//
// Partition: a pair of clusters is far when the boxes are apart and
// max(diam) <= eta * dist; the candidate pairs of level ell are the child pairs of
// the non-far pairs of level ell-1 (dual traversal from (root, root)), produced
// row by row so that every row's column list is sorted.
#include <cmath>

#include "internal.h"

namespace h2mg {

// ----------------------------------------------------------------------------- boxes
// One block per cluster: tight box of its points and its split axis.
__global__ void k_boxes(const double* __restrict__ X, const int* __restrict__ ord,
                        const int* __restrict__ off, int dim, double* __restrict__ box,
                        int* __restrict__ axis) {
  int j = blockIdx.x;
  int a = off[j], b = off[j + 1];
  __shared__ double slo[3][256], shi[3][256];
  double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int p = a + threadIdx.x; p < b; p += blockDim.x) {
    int i = ord[p];
    for (int d = 0; d < dim; ++d) {
      double v = X[(int64_t)i * dim + d];
      lo[d] = fmin(lo[d], v);
      hi[d] = fmax(hi[d], v);
    }
  }
  for (int d = 0; d < dim; ++d) {
    slo[d][threadIdx.x] = lo[d];
    shi[d][threadIdx.x] = hi[d];
  }
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s)
      for (int d = 0; d < dim; ++d) {
        slo[d][threadIdx.x] = fmin(slo[d][threadIdx.x], slo[d][threadIdx.x + s]);
        shi[d][threadIdx.x] = fmax(shi[d][threadIdx.x], shi[d][threadIdx.x + s]);
      }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    int best = 0;
    double ext = -1.0;
    for (int d = 0; d < dim; ++d) {
      box[(int64_t)j * 2 * dim + d] = slo[d][0];
      box[(int64_t)j * 2 * dim + dim + d] = shi[d][0];
      double e = __dsub_rn(shi[d][0], slo[d][0]);
      if (e > ext) {
        ext = e;
        best = d;
      }
    }
    if (axis) axis[j] = best;
  }
}

__global__ void k_seg_of(const int* __restrict__ ord, const int* __restrict__ off,
                         int* __restrict__ seg_of) {
  int j = blockIdx.x;
  for (int p = off[j] + threadIdx.x; p < off[j + 1]; p += blockDim.x) seg_of[ord[p]] = j;
}

// Order-preserving map of a double to uint64 (-0.0 treated as +0.0).
__device__ __forceinline__ uint64_t order_key(double v) {
  if (v == 0.0) v = 0.0;
  uint64_t b = (uint64_t)__double_as_longlong(v);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

__global__ void k_coord_keys(const double* __restrict__ X, int n, int dim,
                             const int* __restrict__ seg_of, const int* __restrict__ axis,
                             uint64_t* __restrict__ key, int* __restrict__ val) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  key[i] = order_key(X[(int64_t)i * dim + axis[seg_of[i]]]);
  val[i] = i;
}

__global__ void k_seg_keys(const int* __restrict__ val, const int* __restrict__ seg_of, int n,
                           uint64_t* __restrict__ key) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < n) key[p] = (uint64_t)seg_of[val[p]];
}

__global__ void k_finite(const double* __restrict__ v, int64_t n, int* __restrict__ flag) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && !isfinite(v[i])) atomicOr(flag, 1);
}

__global__ void k_tree_out(const double* __restrict__ X, const int* __restrict__ ord, int n,
                           int dim, const int* __restrict__ leafoff, int L, int KD,
                           double* __restrict__ Xt, int* __restrict__ slot_of) {
  int leaf = blockIdx.x;
  for (int p = leafoff[leaf] + threadIdx.x; p < leafoff[leaf + 1]; p += blockDim.x) {
    int i = ord[p];
    for (int d = 0; d < dim; ++d) Xt[(int64_t)p * dim + d] = X[(int64_t)i * dim + d];
    slot_of[i] = leaf * KD + (p - leafoff[leaf]);
  }
}

void build_tree(Matrix& M, const double* d_pts) {
  cudaStream_t s = M.stream;
  const int n = (int)M.n, dim = M.dim;
  // depth: smallest L with ceil(n / 2^L) <= leaf
  int L = 0;
  while (((int64_t)n + (1ll << L) - 1) >> L > M.leaf) ++L;
  M.L = L;
  // finite coordinates
  {
    int* flag = M.d_flag;
    H2_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), s));
    int64_t tot = (int64_t)n * dim;
    { k_finite<<<ceil_div(tot, 256), 256, 0, s>>>(d_pts, tot, flag); ::h2mg::count_launch(); }
    H2_LAUNCH_CHECK();
    int h = 0;
    H2_CUDA(cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    H2_CUDA(cudaStreamSynchronize(s));
    H2_REQUIRE(h == 0, H2MG_ERR_INVALID_ARG, "points contain NaN or Inf");
  }
  // host offsets of every level (ceil / floor halves)
  M.offsets.assign(L + 1, {});
  M.offsets[0] = {0, n};
  for (int ell = 0; ell < L; ++ell) {
    const auto& o = M.offsets[ell];
    std::vector<int> nx(1, 0);
    for (size_t j = 0; j + 1 < o.size(); ++j) {
      int sz = o[j + 1] - o[j];
      nx.push_back(o[j] + (sz + 1) / 2);
      nx.push_back(o[j + 1]);
    }
    M.offsets[ell + 1] = nx;
  }
  int maxleaf = 0;
  for (size_t j = 0; j + 1 < M.offsets[L].size(); ++j)
    maxleaf = std::max(maxleaf, M.offsets[L][j + 1] - M.offsets[L][j]);
  M.KD = maxleaf <= 16 ? 16 : maxleaf <= 32 ? 32 : 64;

  int* ord = (int*)M.alloc(sizeof(int) * n);
  {
    std::vector<int> id(n);
    for (int i = 0; i < n; ++i) id[i] = i;
    H2_CUDA(cudaMemcpyAsync(ord, id.data(), sizeof(int) * n, cudaMemcpyHostToDevice, s));
  }
  int* seg_of = (int*)M.alloc(sizeof(int) * n);
  uint64_t* key = (uint64_t*)M.alloc(sizeof(uint64_t) * n);
  int* d_off = (int*)M.alloc(sizeof(int) * ((1 << L) + 1));
  int* d_axis = (int*)M.alloc(sizeof(int) * (1 << L));
  M.d_box.assign(L + 1, nullptr);
  for (int ell = 0; ell <= L; ++ell) {
    int ncl = 1 << ell;
    M.d_box[ell] = (double*)M.alloc(sizeof(double) * 2 * dim * ncl);
    H2_CUDA(cudaMemcpyAsync(d_off, M.offsets[ell].data(), sizeof(int) * (ncl + 1),
                            cudaMemcpyHostToDevice, s));
    { k_boxes<<<ncl, 256, 0, s>>>(d_pts, ord, d_off, dim, M.d_box[ell], d_axis); ::h2mg::count_launch(); }
    H2_LAUNCH_CHECK();
    if (ell == L) break;
    { k_seg_of<<<ncl, 256, 0, s>>>(ord, d_off, seg_of); ::h2mg::count_launch(); }
    H2_LAUNCH_CHECK();
    { k_coord_keys<<<ceil_div(n, 256), 256, 0, s>>>(d_pts, n, dim, seg_of, d_axis, key, ord); ::h2mg::count_launch(); }
    H2_LAUNCH_CHECK();
    radix_sort_u64(key, ord, n, 64, M, s);            // by coordinate, ties by index
    if (ell > 0) {
      { k_seg_keys<<<ceil_div(n, 256), 256, 0, s>>>(ord, seg_of, n, key); ::h2mg::count_launch(); }
      H2_LAUNCH_CHECK();
      radix_sort_u64(key, ord, n, ell, M, s);         // by cluster (stable)
    }
  }
  M.d_perm = ord;
  M.d_leafoff = (int*)M.alloc(sizeof(int) * ((1 << L) + 1));
  H2_CUDA(cudaMemcpyAsync(M.d_leafoff, M.offsets[L].data(), sizeof(int) * ((1 << L) + 1),
                          cudaMemcpyHostToDevice, s));
  M.d_X = (double*)M.alloc(sizeof(double) * (size_t)n * dim);
  M.d_slot_of = (int*)M.alloc(sizeof(int) * n);
  { k_tree_out<<<1 << L, 128, 0, s>>>(d_pts, ord, n, dim, M.d_leafoff, L, M.KD, M.d_X, M.d_slot_of); ::h2mg::count_launch(); }
  H2_LAUNCH_CHECK();
  H2_CUDA(cudaStreamSynchronize(s));
}

// ----------------------------------------------------------------------------- partition
__device__ __forceinline__ bool admissible_pair(const double* bt, const double* bs, int dim,
                                                double eta) {
  // diam = |hi - lo|, dist = |max(0, lo_s - hi_t, lo_t - hi_s)|, summed in axis order
  double dt = 0.0, ds = 0.0, g2 = 0.0;
  for (int d = 0; d < dim; ++d) {
    double et = __dsub_rn(bt[dim + d], bt[d]);
    double es = __dsub_rn(bs[dim + d], bs[d]);
    dt = __dadd_rn(dt, __dmul_rn(et, et));
    ds = __dadd_rn(ds, __dmul_rn(es, es));
    double g = fmax(0.0, fmax(__dsub_rn(bs[d], bt[dim + d]), __dsub_rn(bt[d], bs[dim + d])));
    g2 = __dadd_rn(g2, __dmul_rn(g, g));
  }
  double dist = __dsqrt_rn(g2);
  double diam = fmax(__dsqrt_rn(dt), __dsqrt_rn(ds));
  return dist > 0.0 && diam <= __dmul_rn(eta, dist);
}

// pass 0: count, pass 1: write. Row t of level ell expands the non-far row t/2 of ell-1.
__global__ void k_partition(int nrows, const int* __restrict__ prow, const int* __restrict__ pcol,
                            const double* __restrict__ box, int dim, double eta, int pass,
                            int* __restrict__ far_cnt, int* __restrict__ in_cnt,
                            int* __restrict__ far_col, int* __restrict__ in_col) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nrows) return;
  int p = t >> 1;
  int nf = 0, ni = 0;
  int of = pass ? far_cnt[t] : 0, oi = pass ? in_cnt[t] : 0;
  const double* bt = box + (int64_t)t * 2 * dim;
  for (int e = prow[p]; e < prow[p + 1]; ++e) {
    int sp = pcol[e];
    for (int c = 0; c < 2; ++c) {
      int sidx = 2 * sp + c;
      bool adm = admissible_pair(bt, box + (int64_t)sidx * 2 * dim, dim, eta);
      if (adm) {
        if (pass) far_col[of + nf] = sidx;
        ++nf;
      } else {
        if (pass) in_col[oi + ni] = sidx;
        ++ni;
      }
    }
  }
  if (!pass) {
    far_cnt[t] = nf;
    in_cnt[t] = ni;
  }
}

void build_partition(Matrix& M) {
  cudaStream_t s = M.stream;
  const int L = M.L, dim = M.dim;
  M.far.assign(L + 1, {});
  M.inadm.assign(L + 1, {});
  // level 0: the root pair (dist = 0) is never far
  M.far[0].rowptr = {0, 0};
  M.inadm[0].rowptr = {0, 1};
  M.inadm[0].col = {0};
  int* prow = (int*)M.alloc(sizeof(int) * 2);
  int* pcol = (int*)M.alloc(sizeof(int) * 1);
  {
    int h[2] = {0, 1}, z = 0;
    H2_CUDA(cudaMemcpyAsync(prow, h, sizeof(h), cudaMemcpyHostToDevice, s));
    H2_CUDA(cudaMemcpyAsync(pcol, &z, sizeof(int), cudaMemcpyHostToDevice, s));
  }
  for (int ell = 1; ell <= L; ++ell) {
    int nrows = 1 << ell;
    int* fc = (int*)M.alloc(sizeof(int) * (nrows + 1));
    int* ic = (int*)M.alloc(sizeof(int) * (nrows + 1));
    { k_partition<<<ceil_div(nrows, 128), 128, 0, s>>>(nrows, prow, pcol, M.d_box[ell], dim, M.eta, 0,
                                                     fc, ic, nullptr, nullptr); ::h2mg::count_launch(); }
    H2_LAUNCH_CHECK();
    exclusive_scan_i32(fc, fc, nrows, s, M);
    exclusive_scan_i32(ic, ic, nrows, s, M);
    int nf = 0, ni = 0;
    H2_CUDA(cudaMemcpyAsync(&nf, fc + nrows, sizeof(int), cudaMemcpyDeviceToHost, s));
    H2_CUDA(cudaMemcpyAsync(&ni, ic + nrows, sizeof(int), cudaMemcpyDeviceToHost, s));
    H2_CUDA(cudaStreamSynchronize(s));
    int* fcol = (int*)M.alloc(sizeof(int) * std::max(nf, 1));
    int* icol = (int*)M.alloc(sizeof(int) * std::max(ni, 1));
    { k_partition<<<ceil_div(nrows, 128), 128, 0, s>>>(nrows, prow, pcol, M.d_box[ell], dim, M.eta, 1,
                                                     fc, ic, fcol, icol); ::h2mg::count_launch(); }
    H2_LAUNCH_CHECK();
    HostCSR& F = M.far[ell];
    HostCSR& I = M.inadm[ell];
    F.rowptr.resize(nrows + 1);
    I.rowptr.resize(nrows + 1);
    F.col.resize(nf);
    I.col.resize(ni);
    H2_CUDA(cudaMemcpyAsync(F.rowptr.data(), fc, sizeof(int) * (nrows + 1), cudaMemcpyDeviceToHost, s));
    H2_CUDA(cudaMemcpyAsync(I.rowptr.data(), ic, sizeof(int) * (nrows + 1), cudaMemcpyDeviceToHost, s));
    if (nf) H2_CUDA(cudaMemcpyAsync(F.col.data(), fcol, sizeof(int) * nf, cudaMemcpyDeviceToHost, s));
    if (ni) H2_CUDA(cudaMemcpyAsync(I.col.data(), icol, sizeof(int) * ni, cudaMemcpyDeviceToHost, s));
    H2_CUDA(cudaStreamSynchronize(s));
    prow = ic;
    pcol = icol;
  }
  M.tstar = -1;
  for (int ell = 0; ell <= L; ++ell)
    if (M.far[ell].nnz() > 0) {
      M.tstar = ell;
      break;
    }
  M.lev_nat = M.tstar < 0 ? 1 : L - M.tstar + 1;
}

}  // namespace h2mg
