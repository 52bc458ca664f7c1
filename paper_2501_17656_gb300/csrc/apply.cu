// apply.cu -- the level-synchronous H2 matrix-vector product of every multigrid level.
//
// Sec. 3.1: y = D x + U_1 (S_1 x_1 + U_2 (... (S_{l-1} x_l + U_l S_l x_l) ...)) with
// x_i = V_i x_{i-1} (upward pass) and y_{i-1} = D_i x_{i-1} + U_i y_i (downward pass).
// For multigrid level i >= 2 the operator A_i (eq. a2_str) has the same shape on the
// coefficients of tree level m(i), with P_i in place of D and the identity as the
// basis of level m(i).
//
// GPU layout: one symmetric block-sparse product (k_bsgemv) covers the close blocks
// or every coupling level at once: one CTA per block row, each warp streams whole
// K x K blocks (swizzled so that every warp load is one contiguous 512 B segment),
// and each block is used twice -- y_t += B x_s for its row and, for s != t, the
// transposed product B^T x_t for its column, both added atomically into a zeroed row
// buffer. The upward pass (k_up_leaf, k_up_multi) forms the cluster coefficients of
// every level; the downward pass (k_down_multi) adds the transfer from the parent to
// each level's row results and writes the finest level out (k_leaf_final at i = 1).
//
// Arithmetic per block format: F64 (DFMA), DF (double-float on the FP32 pipes: the
// error-free products/sums of Dekker and Knuth), F32 (FP32 FMA). Vectors inside the
// product are in the same format; the multigrid vectors outside are float64.
#include <algorithm>

#include "internal.h"

namespace h2mg {

// ----------------------------------------------------------------------------- arithmetic
template <int FMT>
struct Ar;

template <>
struct Ar<FMT_F64> {
  static constexpr int V = 2;
  using yo_t = double;       // type of the atomically accumulated row outputs
  __device__ static yo_t to_yo(double a) { return a; }
  __device__ static void atomic_add(yo_t* p, double a) { atomicAdd(p, a); }
  __device__ static double from_yo(yo_t v) { return v; }
  using vec_t = double;
  using mel_t = double;
  using acc_t = double;
  using ld_t = double2;
  __device__ static acc_t zero() { return 0.0; }
  __device__ static void decode(const ld_t& v, mel_t* m) {
    m[0] = v.x;
    m[1] = v.y;
  }
  __device__ static void fma(acc_t& a, mel_t m, vec_t x) { a = ::fma(m, x, a); }
  __device__ static void add(acc_t& a, acc_t b) { a += b; }
  __device__ static void norm(acc_t&) {}
  __device__ static acc_t shfl(acc_t a, int m) { return __shfl_xor_sync(0xffffffffu, a, m); }
  __device__ static vec_t out(acc_t a) { return a; }
  __device__ static double to_d(vec_t v) { return v; }
  __device__ static vec_t from_d(double v) { return v; }
};

template <>
struct Ar<FMT_DF> {
  static constexpr int V = 2;
  using yo_t = double;
  __device__ static yo_t to_yo(float2 a) { return (double)a.x + (double)a.y; }
  __device__ static void atomic_add(yo_t* p, float2 a) { atomicAdd(p, to_yo(a)); }
  __device__ static float2 from_yo(yo_t v) { return from_d(v); }
  using vec_t = float2;
  using mel_t = float2;
  using acc_t = float2;
  using ld_t = float4;
  __device__ static acc_t zero() { return make_float2(0.f, 0.f); }
  __device__ static void decode(const ld_t& v, mel_t* m) {
    m[0] = make_float2(v.x, v.y);
    m[1] = make_float2(v.z, v.w);
  }
  __device__ static void fma(acc_t& a, mel_t m, vec_t x) { df_fma(a.x, a.y, m.x, m.y, x.x, x.y); }
  __device__ static void add(acc_t& a, acc_t b) { df_add(a.x, a.y, b.x, b.y); }
  __device__ static void norm(acc_t& a) { df_norm(a.x, a.y); }
  __device__ static acc_t shfl(acc_t a, int m) {
    return make_float2(__shfl_xor_sync(0xffffffffu, a.x, m), __shfl_xor_sync(0xffffffffu, a.y, m));
  }
  __device__ static vec_t out(acc_t a) {
    df_norm(a.x, a.y);
    return a;
  }
  __device__ static double to_d(vec_t v) { return (double)v.x + (double)v.y; }
  __device__ static vec_t from_d(double v) {
    df2 d = df_from_double(v);
    return make_float2(d.hi, d.lo);
  }
};

template <>
struct Ar<FMT_F32> {
  static constexpr int V = 4;
  using yo_t = float;
  __device__ static yo_t to_yo(float a) { return a; }
  __device__ static void atomic_add(yo_t* p, float a) { atomicAdd(p, a); }
  __device__ static float from_yo(yo_t v) { return v; }
  using vec_t = float;
  using mel_t = float;
  using acc_t = float;
  using ld_t = float4;
  __device__ static acc_t zero() { return 0.f; }
  __device__ static void decode(const ld_t& v, mel_t* m) {
    m[0] = v.x;
    m[1] = v.y;
    m[2] = v.z;
    m[3] = v.w;
  }
  __device__ static void fma(acc_t& a, mel_t m, vec_t x) { a = fmaf(m, x, a); }
  __device__ static void add(acc_t& a, acc_t b) { a += b; }
  __device__ static void norm(acc_t&) {}
  __device__ static acc_t shfl(acc_t a, int m) { return __shfl_xor_sync(0xffffffffu, a, m); }
  __device__ static vec_t out(acc_t a) { return a; }
  __device__ static double to_d(vec_t v) { return (double)v; }
  __device__ static vec_t from_d(double v) { return __double2float_rn(v); }
};

// Float64 blocks, double-double vectors and sums (the extended-precision residual).
template <>
struct Ar<FMT_DD> {
  static constexpr int V = 2;
  using yo_t = double2;
  __device__ static yo_t to_yo(double2 a) { return a; }
  __device__ static void atomic_add(yo_t* p, double2 a) { dd_atomic_add(p, a); }
  __device__ static double2 from_yo(yo_t v) { return v; }
  using vec_t = double2;
  using mel_t = double;
  using acc_t = double2;
  using ld_t = double2;
  __device__ static acc_t zero() { return make_double2(0.0, 0.0); }
  __device__ static void decode(const ld_t& v, mel_t* m) {
    m[0] = v.x;
    m[1] = v.y;
  }
  __device__ static void fma(acc_t& a, mel_t m, vec_t x) { dd_fma(a.x, a.y, m, x.x, x.y); }
  __device__ static void add(acc_t& a, acc_t b) { dd_add(a.x, a.y, b.x, b.y); }
  __device__ static void norm(acc_t& a) { dd_norm(a.x, a.y); }
  __device__ static acc_t shfl(acc_t a, int m) {
    return make_double2(__shfl_xor_sync(0xffffffffu, a.x, m), __shfl_xor_sync(0xffffffffu, a.y, m));
  }
  __device__ static vec_t out(acc_t a) {
    dd_norm(a.x, a.y);
    return a;
  }
  __device__ static double to_d(vec_t v) { return v.x + v.y; }
  __device__ static vec_t from_d(double v) { return make_double2(v, 0.0); }
};

// NR consecutive elements from shared memory, as one vector load where the row is 8
// or 16 bytes (rows are aligned to their size).
template <class T, int NR>
__device__ __forceinline__ void load_row(const T* p, T* out) {
  if constexpr (sizeof(T) * NR == 16) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    memcpy(out, &v, 16);
  } else if constexpr (sizeof(T) * NR == 8) {
    const float2 v = *reinterpret_cast<const float2*>(p);
    memcpy(out, &v, 8);
  } else {
#pragma unroll
    for (int j = 0; j < NR; ++j) out[j] = p[j];
  }
}

// ----------------------------------------------------------------------------- block GEMV
// One CTA (8 warps) per block row t of a symmetric upper-stored block operator:
// yrow[t] += sum_e B_e x_col(e) and, for every off-diagonal entry e = (t, s),
// yrow[s] += B_e^T x_t. All contributions are atomic adds (FP64 for the F64 and DF
// copies, FP32 for the F32 copy) into a row buffer zeroed before the launch, so the
// summation order, and the last bits of a sum, may differ from run to run. When the
// operator has few rows, each row is split over `split` CTAs (strided entries).
// NR right-hand sides share every block read: vectors are interleaved, element
// (slot, coefficient, column j) at ((slot * K + coefficient) * NR + j).
// CTAs per SM the register allocation must allow: the FP32 products are HBM-bound and
// need the occupancy; the float64 / double-float ones are ALU-bound.
template <int FMT, int NR>
constexpr int bsgemv_min_ctas() {
  return FMT == FMT_F32 ? (NR >= 4 ? 2 : (NR == 2 ? 3 : 4)) : 2;
}

// Asks the memory system to bring `bytes` (a multiple of 16, 16-byte aligned) from
// global memory into L2 without waiting: the next block a warp will read streams in
// while it works on the current one.
__device__ __forceinline__ void prefetch_l2_bulk(const void* p, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

template <int K, int FMT, int NR>
__global__ void __launch_bounds__(256, bsgemv_min_ctas<FMT, NR>()) k_bsgemv(const int* __restrict__ rowptr,
                                                const int* __restrict__ col,
                                                const void* const* __restrict__ blk,
                                                const typename Ar<FMT>::vec_t* __restrict__ x,
                                                typename Ar<FMT>::yo_t* __restrict__ yrow, int split) {
  using A = Ar<FMT>;
  using vec_t = typename A::vec_t;
  using mel_t = typename A::mel_t;
  using acc_t = typename A::acc_t;
  using ld_t = typename A::ld_t;
  constexpr int LPC = K / 8, CPP = 32 / LPC, T = K * K / 256;
  constexpr int CH = T < LPC ? T : LPC;
  constexpr int V = A::V, P = 8 / V;
  __shared__ acc_t red[8][K * NR];
  // x of the block row (input of the transposed products), one padding row after
  // every 8 rows so that the 8 row groups of a warp read distinct banks
  __shared__ __align__(16) vec_t sxt[(K + K / 8) * NR];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int row = blockIdx.x / split, part = blockIdx.x % split;
  const int rb = 8 * (lane % LPC), cl = lane / LPC;
  for (int i = threadIdx.x; i < K * NR; i += blockDim.x) {
    const int r = i / NR;
    sxt[(r + r / 8) * NR + i % NR] = x[(int64_t)row * K * NR + i];
  }
  __syncthreads();
  const vec_t* xt = sxt + (rb + rb / 8) * NR;   // rows rb..rb+7 of this lane
  acc_t ya[8][NR];
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int j = 0; j < NR; ++j) ya[r][j] = A::zero();
  const int e0 = rowptr[row], e1 = rowptr[row + 1];
  constexpr unsigned kBlockBytes = K * K / V * (unsigned)sizeof(ld_t);   // one stored block
  for (int e = e0 + part * 8 + w; e < e1; e += 8 * split) {
    const int s = col[e];
    const ld_t* B = (const ld_t*)blk[e];
    // with one column the loads of 32 warps per SM already cover the DRAM latency, and
    // prefetched blocks would be evicted from L2 before use; with several columns
    // (fewer resident warps) the prefetch keeps the stream going
    if constexpr (NR >= 2)
      if (lane == 0 && e + 8 * split < e1) prefetch_l2_bulk(blk[e + 8 * split], kBlockBytes);
    const vec_t* xs = x + (int64_t)s * K * NR;
    const bool off = (s != row);
#pragma unroll 1
    for (int ch = 0; ch < T / CH; ++ch) {
      acc_t zc[CH][NR];
#pragma unroll
      for (int tt = 0; tt < CH; ++tt) {
        const int t = ch * CH + tt;
        mel_t m[8];
#pragma unroll
        for (int k = 0; k < P; ++k) {
          ld_t v = __ldcs(B + (t * P + k) * 32 + lane);
          A::decode(v, m + k * V);
        }
#pragma unroll
        for (int j = 0; j < NR; ++j) {
          const vec_t xv = xs[(cl + CPP * t) * NR + j];
#pragma unroll
          for (int r = 0; r < 8; ++r) A::fma(ya[r][j], m[r], xv);
          acc_t zz = A::zero();
#pragma unroll
          for (int r = 0; r < 8; ++r) A::fma(zz, m[r], xt[r * NR + j]);
          zc[tt][j] = zz;
        }
        if ((t & 3) == 3) {
#pragma unroll
          for (int r = 0; r < 8; ++r)
#pragma unroll
            for (int j = 0; j < NR; ++j) A::norm(ya[r][j]);
        }
      }
      if (off) {
        // reduce the CH partial columns over the LPC lanes that share them
#pragma unroll
        for (int j = 0; j < NR; ++j) {
          if (CH == LPC) {
#pragma unroll
            for (int h = CH / 2; h >= 1; h >>= 1) {
              const bool up = (lane & h) != 0;
#pragma unroll
              for (int q = 0; q < h; ++q) {
                acc_t send = up ? zc[q][j] : zc[q + h][j];
                acc_t keep = up ? zc[q + h][j] : zc[q][j];
                A::add(keep, A::shfl(send, h));
                zc[q][j] = keep;
              }
            }
            const int tt = lane & (CH - 1);
            A::atomic_add(yrow + ((int64_t)s * K + cl + CPP * (ch * CH + tt)) * NR + j, A::out(zc[0][j]));
          } else {
#pragma unroll
            for (int h = LPC / 2; h >= 1; h >>= 1) A::add(zc[0][j], A::shfl(zc[0][j], h));
            if ((lane % LPC) == 0)
              A::atomic_add(yrow + ((int64_t)s * K + cl + CPP * (ch * CH)) * NR + j, A::out(zc[0][j]));
          }
        }
      }
    }
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
      for (int j = 0; j < NR; ++j) A::norm(ya[r][j]);
  }
  // rows: sum over the lanes that share them, then over the warps
#pragma unroll
  for (int h = LPC; h < 32; h <<= 1)
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
      for (int j = 0; j < NR; ++j) A::add(ya[r][j], A::shfl(ya[r][j], h));
  if (lane < LPC)
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
      for (int j = 0; j < NR; ++j) red[w][(rb + r) * NR + j] = ya[r][j];
  __syncthreads();
  for (int i = threadIdx.x; i < K * NR; i += blockDim.x) {
    acc_t s = red[0][i];
#pragma unroll
    for (int ww = 1; ww < 8; ++ww) A::add(s, red[ww][i]);
    A::atomic_add(yrow + (int64_t)row * K * NR + i, A::out(s));
  }
}

// ----------------------------------------------------------------------------- passes
// point vectors (float64, user order, column j at x + j*ldx) -> padded tree slots
template <int FMT, int NR>
__global__ void k_pts_in(const double* __restrict__ x, int64_t ldx, const int* __restrict__ slot_of, int64_t n,
                         typename Ar<FMT>::vec_t* __restrict__ xp) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t sl = slot_of[i];
#pragma unroll
  for (int j = 0; j < NR; ++j) xp[sl * NR + j] = Ar<FMT>::from_d(x[i + j * ldx]);
}

// coefficient vectors (float64, KC per cluster, column j at x + j*ldx) -> interleaved
template <int FMT, int NR>
__global__ void k_coef_in(const double* __restrict__ x, int64_t ldx, int64_t n,
                          typename Ar<FMT>::vec_t* __restrict__ xc) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
#pragma unroll
  for (int j = 0; j < NR; ++j) xc[i * NR + j] = Ar<FMT>::from_d(x[i + j * ldx]);
}

// x_hat(leaf l)[b] = sum_i U_l[i, b] x_l[i]   (UT = U^T, KC x KD column-major)
template <int FMT, class BT, int NR>
__global__ void k_up_leaf(const BT* __restrict__ UT, int KD, int KC,
                          const typename Ar<FMT>::vec_t* __restrict__ xp,
                          typename Ar<FMT>::vec_t* __restrict__ xc) {
  int l = blockIdx.x;
  const BT* Ul = UT + (int64_t)l * KD * KC;
  if constexpr (FMT == FMT_DD) {   // double-double coefficients
    __shared__ double2 xd[64 * NR];
    for (int i = threadIdx.x; i < KD * NR; i += blockDim.x) xd[i] = xp[(int64_t)l * KD * NR + i];
    __syncthreads();
    for (int b = threadIdx.x; b < KC; b += blockDim.x) {
      double2 acc[NR];
#pragma unroll
      for (int j = 0; j < NR; ++j) acc[j] = make_double2(0.0, 0.0);
      for (int i = 0; i < KD; ++i) {
        const double u = (double)Ul[b + i * KC];
#pragma unroll
        for (int j = 0; j < NR; ++j) dd_fma(acc[j].x, acc[j].y, u, xd[i * NR + j].x, xd[i * NR + j].y);
      }
#pragma unroll
      for (int j = 0; j < NR; ++j) {
        dd_norm(acc[j].x, acc[j].y);
        xc[((int64_t)l * KC + b) * NR + j] = acc[j];
      }
    }
  } else {
    __shared__ double xs[64 * NR];
    for (int i = threadIdx.x; i < KD * NR; i += blockDim.x) xs[i] = Ar<FMT>::to_d(xp[(int64_t)l * KD * NR + i]);
    __syncthreads();
    for (int b = threadIdx.x; b < KC; b += blockDim.x) {
      double acc[NR];
#pragma unroll
      for (int j = 0; j < NR; ++j) acc[j] = 0.0;
      for (int i = 0; i < KD; ++i) {
        double u = (double)Ul[b + i * KC];
#pragma unroll
        for (int j = 0; j < NR; ++j) acc[j] += u * xs[i * NR + j];
      }
#pragma unroll
      for (int j = 0; j < NR; ++j) xc[((int64_t)l * KC + b) * NR + j] = Ar<FMT>::from_d(acc[j]);
    }
  }
}

// Transfer passes as block products. Every orthonormal transfer E'_c (K x K, rows =
// child coefficients, columns = parent coefficients) is stored swizzled like the
// blocks of k_bsgemv, and one warp streams one transfer with the same lane layout:
// the upward pass uses the transposed product E'_c^T x_c (reduce-scatter over the
// lanes that share a column), the downward pass the row product E'_c y_parent.
//
// One launch covers up to 3 (upward) or 4 (downward) consecutive tree levels: a CTA
// owns a subtree (8 clusters of the bottom level going up; one cluster of the top
// level and its descendants going down), keeps the intermediate coefficients in
// shared memory and writes every level's coefficients to global memory, since the
// coupling products and the next launch read them.

// v = E'^T x over the TPW tiles starting at tile t0 of one K x K transfer at B
// (warp-wide; x: K*NR values, any address space). A tile covers CPP whole columns of
// E', so the tiles of one transfer can be split over several warps, each writing the
// outputs of its own columns.
template <int K, int FMT, int NR, int TPW>
__device__ __forceinline__ void warp_transfer_t(const void* __restrict__ Bv, const typename Ar<FMT>::vec_t* x,
                                                typename Ar<FMT>::acc_t* v, int t0) {
  using A = Ar<FMT>;
  using vec_t = typename A::vec_t;
  using mel_t = typename A::mel_t;
  using acc_t = typename A::acc_t;
  using ld_t = typename A::ld_t;
  constexpr int LPC = K / 8, CPP = 32 / LPC;
  constexpr int CH = TPW < LPC ? TPW : LPC;
  constexpr int V = A::V, P = 8 / V;
  const int lane = threadIdx.x & 31;
  const int rb = 8 * (lane % LPC), cl = lane / LPC;
  vec_t xt[8][NR];
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int j = 0; j < NR; ++j) xt[r][j] = x[(rb + r) * NR + j];
  const ld_t* B = (const ld_t*)Bv;
#pragma unroll 1
  for (int ch = 0; ch < TPW / CH; ++ch) {
    acc_t zc[CH][NR];
#pragma unroll
    for (int tt = 0; tt < CH; ++tt) {
      const int t = t0 + ch * CH + tt;
      mel_t m[8];
#pragma unroll
      for (int k = 0; k < P; ++k) {
        ld_t q = __ldg(B + (t * P + k) * 32 + lane);
        A::decode(q, m + k * V);
      }
#pragma unroll
      for (int j = 0; j < NR; ++j) {
        acc_t zz = A::zero();
#pragma unroll
        for (int r = 0; r < 8; ++r) A::fma(zz, m[r], xt[r][j]);
        zc[tt][j] = zz;
      }
    }
#pragma unroll
    for (int j = 0; j < NR; ++j) {
      // butterfly over the CH tiles (lane keeps tile lane & (CH-1)), then the rest of
      // the LPC lanes that share a column
#pragma unroll
      for (int h = CH / 2; h >= 1; h >>= 1) {
        const bool up = (lane & h) != 0;
#pragma unroll
        for (int q = 0; q < h; ++q) {
          acc_t send = up ? zc[q][j] : zc[q + h][j];
          acc_t keep = up ? zc[q + h][j] : zc[q][j];
          A::add(keep, A::shfl(send, h));
          zc[q][j] = keep;
        }
      }
#pragma unroll
      for (int h = CH; h < LPC; h <<= 1) A::add(zc[0][j], A::shfl(zc[0][j], h));
      if ((lane % LPC) < CH) v[(cl + CPP * (t0 + ch * CH + (lane & (CH - 1)))) * NR + j] = zc[0][j];
    }
  }
}

// Splits one transfer's T tiles over `wpb` warps (a power of two): warp `sub` takes
// T / wpb consecutive tiles (warps beyond T do nothing).
template <int K, int FMT, int NR>
__device__ __forceinline__ void warp_transfer_t_part(const void* B, const typename Ar<FMT>::vec_t* x,
                                                     typename Ar<FMT>::acc_t* v, int wpb, int sub) {
  constexpr int T = K * K / 256;
  const int w = wpb < T ? wpb : T;
  if (sub >= w) return;
  const int tpw = T / w;
  if constexpr (T >= 16) if (tpw == 16) { warp_transfer_t<K, FMT, NR, 16>(B, x, v, 0); return; }
  if constexpr (T >= 8) if (tpw == 8) { warp_transfer_t<K, FMT, NR, 8>(B, x, v, sub * 8); return; }
  if constexpr (T >= 4) if (tpw == 4) { warp_transfer_t<K, FMT, NR, 4>(B, x, v, sub * 4); return; }
  if constexpr (T >= 2) if (tpw == 2) { warp_transfer_t<K, FMT, NR, 2>(B, x, v, sub * 2); return; }
  warp_transfer_t<K, FMT, NR, 1>(B, x, v, sub);
}

// s = rows of E' y over the tiles [t0, t1) of one K x K transfer at B (warp-wide;
// y: K*NR values, any address space); partial sums over those tiles' columns.
template <int K, int FMT, int NR>
__device__ __forceinline__ void warp_transfer(const void* __restrict__ Bv, const typename Ar<FMT>::vec_t* y,
                                              typename Ar<FMT>::acc_t* s, int t0, int t1) {
  using A = Ar<FMT>;
  using vec_t = typename A::vec_t;
  using mel_t = typename A::mel_t;
  using acc_t = typename A::acc_t;
  using ld_t = typename A::ld_t;
  constexpr int LPC = K / 8, CPP = 32 / LPC;
  constexpr int V = A::V, P = 8 / V;
  const int lane = threadIdx.x & 31;
  const int rb = 8 * (lane % LPC), cl = lane / LPC;
  acc_t ya[8][NR];
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int j = 0; j < NR; ++j) ya[r][j] = A::zero();
  const ld_t* B = (const ld_t*)Bv;
#pragma unroll 4
  for (int t = t0; t < t1; ++t) {
    mel_t m[8];
#pragma unroll
    for (int k = 0; k < P; ++k) {
      ld_t q = __ldg(B + (t * P + k) * 32 + lane);
      A::decode(q, m + k * V);
    }
#pragma unroll
    for (int j = 0; j < NR; ++j) {
      const vec_t xv = y[(cl + CPP * t) * NR + j];
#pragma unroll
      for (int r = 0; r < 8; ++r) A::fma(ya[r][j], m[r], xv);
    }
  }
#pragma unroll
  for (int h = LPC; h < 32; h <<= 1)
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
      for (int j = 0; j < NR; ++j) A::add(ya[r][j], A::shfl(ya[r][j], h));
  if (lane < LPC)
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
      for (int j = 0; j < NR; ++j) s[(rb + r) * NR + j] = ya[r][j];
}

// Levels of one pass launch: step k works on tree level `lev[k]`.
struct PassLevels {
  const void* E[4];   // transfer pool of the (child) clusters of step k (nullptr: top level, no parent)
  void* out[4];       // up: parent coefficients of step k; down: coefficients of step k's clusters
  int slot[4];        // down: first slot of step k's level (row buffer index)
  int n[4];           // clusters of step k's level
};

// Upward pass over `steps` levels: step k maps the children (level lc - k) of this
// CTA's subtree to their parents. x_bottom: coefficients of level lc. At step k the
// 8 >> k children of the CTA share its 8 warps (1 << k warps per transfer).
template <int K, int FMT, int NR>
__global__ void __launch_bounds__(256) k_up_multi(PassLevels pl, int steps,
                                                  const typename Ar<FMT>::vec_t* __restrict__ xbottom) {
  using A = Ar<FMT>;
  using vec_t = typename A::vec_t;
  using acc_t = typename A::acc_t;
  constexpr size_t kBlk = (size_t)K * K * (FMT == FMT_F32 ? 4 : 8);
  __shared__ acc_t v[8][K * NR];
  __shared__ vec_t xin[4][K * NR];
  const int w = threadIdx.x >> 5;
  for (int k = 0; k < steps; ++k) {
    const int per = 8 >> k;                 // children of this CTA at step k
    const int b = w >> k, sub = w & ((1 << k) - 1);
    const int c = blockIdx.x * per + b;     // child index within its level
    if (c < pl.n[k]) {
      const vec_t* x = (k == 0) ? xbottom + (int64_t)c * K * NR : xin[b];
      warp_transfer_t_part<K, FMT, NR>((const char*)pl.E[k] + (size_t)c * kBlk, x, v[b], 1 << k, sub);
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < (per / 2) * K * NR; idx += blockDim.x) {
      const int pb = idx / (K * NR), i = idx % (K * NR);
      const int c0 = blockIdx.x * per + 2 * pb;
      if (c0 < pl.n[k]) {
        acc_t t = v[2 * pb][i];
        A::add(t, v[2 * pb + 1][i]);
        const vec_t o = A::out(t);
        ((vec_t*)pl.out[k])[(int64_t)(c0 >> 1) * K * NR + i] = o;
        xin[pb][i] = o;
      }
    }
    __syncthreads();
  }
}

// Downward pass over `steps` levels from this CTA's top cluster (level lt): step k
// forms y_c = yrow_c + E'_c y_parent(c) for the 2^k descendants at level lt + k
// (no transfer term at the coupling top level), the CTA's 8 warps sharing each
// transfer's tiles (8 >> k warps per transfer). ypar: coefficients of level lt - 1.
// On the last step of the last launch the result goes to yout (float64, column j at
// yout + j * ldo) instead of the coefficient buffer, when yout is given.
template <int K, int FMT, int NR>
__global__ void __launch_bounds__(256) k_down_multi(PassLevels pl, int steps,
                                                    const typename Ar<FMT>::yo_t* __restrict__ yrow,
                                                    const typename Ar<FMT>::vec_t* __restrict__ ypar,
                                                    double* __restrict__ yout, int64_t ldo) {
  using A = Ar<FMT>;
  using vec_t = typename A::vec_t;
  using acc_t = typename A::acc_t;
  constexpr size_t kBlk = (size_t)K * K * (FMT == FMT_F32 ? 4 : 8);
  constexpr int T = K * K / 256;
  __shared__ acc_t sv[8][K * NR];
  __shared__ vec_t ys[8][K * NR];
  const int w = threadIdx.x >> 5;
  for (int k = 0; k < steps; ++k) {
    const int per = 1 << k;                       // clusters of this CTA at step k
    const int wpb = 8 >> k;                       // warps per transfer
    const int wpe = wpb < T ? wpb : T;            // of which hold tiles
    const int b = w / wpb, sub = w % wpb;
    const int c = blockIdx.x * per + b;           // cluster index within its level
    if (pl.E[k] && c < pl.n[k] && sub < wpe) {
      const vec_t* yp = (k == 0) ? ypar + (int64_t)(c >> 1) * K * NR : ys[b >> 1];
      const int tpw = T / wpe;
      warp_transfer<K, FMT, NR>((const char*)pl.E[k] + (size_t)c * kBlk, yp, sv[w], sub * tpw, (sub + 1) * tpw);
    }
    __syncthreads();   // every parent value and partial of this step is in place
    const bool last = (k == steps - 1) && yout;
    for (int idx = threadIdx.x; idx < per * K * NR; idx += blockDim.x) {
      const int bb = idx / (K * NR), i = idx % (K * NR);
      const int cc = blockIdx.x * per + bb;
      if (cc >= pl.n[k]) continue;
      acc_t acc = A::from_yo(yrow[(int64_t)(pl.slot[k] + cc) * K * NR + i]);
      if (pl.E[k])
        for (int q = 0; q < wpe; ++q) A::add(acc, sv[bb * wpb + q][i]);
      const vec_t o = A::out(acc);
      if (last) {
        const int a = i / NR, j = i % NR;
        yout[(int64_t)cc * K + a + j * ldo] = A::to_d(o);
      } else {
        ((vec_t*)pl.out[k])[(int64_t)cc * K * NR + i] = o;
        ys[bb][i] = o;
      }
    }
    __syncthreads();
  }
}

// natural column-major K x K blocks (float64) -> swizzled blocks in a format
__global__ void k_swizzle_blocks(const double* __restrict__ in, int K, void* __restrict__ out, int fmt) {
  int64_t b = blockIdx.x;
  int V = fmt == FMT_F32 ? 4 : 2, LPC = K / 8, CPP = 32 / LPC, P = 8 / V;
  for (int pos = threadIdx.x; pos < K * K; pos += blockDim.x) {
    int sub = pos % V, ln = (pos / V) % 32, tk = pos / (V * 32);
    int t = tk / P, k = tk % P;
    int i = 8 * (ln % LPC) + k * V + sub, j = t * CPP + ln / LPC;
    double v = in[b * K * K + i + (int64_t)j * K];
    int64_t idx = b * K * K + pos;
    if (fmt == FMT_F64) {
      ((double*)out)[idx] = v;
    } else if (fmt == FMT_DF) {
      float h = __double2float_rn(v);
      ((float2*)out)[idx] = make_float2(h, __double2float_rn(v - (double)h));
    } else {
      ((float*)out)[idx] = __double2float_rn(v);
    }
  }
}

// y(point) = yrowD + U y_hat(leaf), scattered to user order (column j at y + j*ldy).
template <int FMT, class BT, int NR>
__global__ void k_leaf_final(int KD, int KC, const typename Ar<FMT>::yo_t* __restrict__ yrow,
                             const BT* __restrict__ U, const typename Ar<FMT>::vec_t* __restrict__ yleaf,
                             const int* __restrict__ leafoff, const int* __restrict__ perm,
                             double* __restrict__ y, int64_t ldy) {
  using A = Ar<FMT>;
  int l = blockIdx.x;
  int p0 = leafoff[l], nl = leafoff[l + 1] - p0;
  if constexpr (FMT == FMT_DD) {   // double-double sums, rounded to float64 on output
    __shared__ double2 pd[64 * NR];
    if (U)
      for (int i = threadIdx.x; i < KC * NR; i += blockDim.x) pd[i] = yleaf[(int64_t)l * KC * NR + i];
    __syncthreads();
    for (int i = threadIdx.x; i < nl; i += blockDim.x) {
      double2 v[NR];
#pragma unroll
      for (int j = 0; j < NR; ++j) v[j] = yrow[((int64_t)l * KD + i) * NR + j];
      if (U) {
        const BT* Ul = U + (int64_t)l * KD * KC;
        for (int b = 0; b < KC; ++b) {
          const double u = (double)Ul[i + b * KD];
#pragma unroll
          for (int j = 0; j < NR; ++j) dd_fma(v[j].x, v[j].y, u, pd[b * NR + j].x, pd[b * NR + j].y);
        }
      }
      const int64_t o = perm[p0 + i];
#pragma unroll
      for (int j = 0; j < NR; ++j) y[o + j * ldy] = v[j].x + v[j].y;
    }
  } else {
    __shared__ double ps[64 * NR];
    if (U)
      for (int i = threadIdx.x; i < KC * NR; i += blockDim.x) ps[i] = A::to_d(yleaf[(int64_t)l * KC * NR + i]);
    __syncthreads();
    for (int i = threadIdx.x; i < nl; i += blockDim.x) {
      double v[NR];
#pragma unroll
      for (int j = 0; j < NR; ++j) v[j] = (double)yrow[((int64_t)l * KD + i) * NR + j];
      if (U) {
        const BT* Ul = U + (int64_t)l * KD * KC;
        for (int b = 0; b < KC; ++b) {
          double u = (double)Ul[i + b * KD];
#pragma unroll
          for (int j = 0; j < NR; ++j) v[j] += u * ps[b * NR + j];
        }
      }
      const int64_t o = perm[p0 + i];
#pragma unroll
      for (int j = 0; j < NR; ++j) y[o + j * ldy] = v[j];
    }
  }
}

__global__ void k_transpose_blocks(const double* __restrict__ in, int R, int C, double* __restrict__ out) {
  // per block: in R x C column-major -> out C x R column-major
  int64_t b = blockIdx.x;
  for (int e = threadIdx.x; e < R * C; e += blockDim.x) {
    int i = e % R, j = e / R;
    out[b * R * C + j + (int64_t)i * C] = in[b * R * C + e];
  }
}
__global__ void k_transpose_blocks32(const float* __restrict__ in, int R, int C, float* __restrict__ out) {
  int64_t b = blockIdx.x;
  for (int e = threadIdx.x; e < R * C; e += blockDim.x) {
    int i = e % R, j = e / R;
    out[b * R * C + j + (int64_t)i * C] = in[b * R * C + e];
  }
}

// ----------------------------------------------------------------------------- host
struct OpHost {
  std::vector<int> rowptr, col;
  std::vector<int64_t> blk;     // block index in the pool of the entry
  std::vector<int> pool;        // 0: D/S pool, 1: P pool
  std::vector<int> rowof;
};

static int64_t upper_pos(const HostCSR& C, int t, int s, bool strict) {
  auto b = C.col.begin() + C.rowptr[t], e = C.col.begin() + C.rowptr[t + 1];
  auto it = std::lower_bound(b, e, s);
  if (it == e || *it != s) return -1;
  auto first = std::lower_bound(b, e, strict ? t + 1 : t);
  return it - first;
}

static std::vector<int64_t> ubase(const HostCSR& C, int nrows, bool strict) {
  std::vector<int64_t> ub(nrows + 1, 0);
  for (int t = 0; t < nrows; ++t) {
    int cnt = 0;
    for (int e = C.rowptr[t]; e < C.rowptr[t + 1]; ++e) cnt += strict ? (C.col[e] > t) : (C.col[e] >= t);
    ub[t + 1] = ub[t] + cnt;
  }
  return ub;
}

static SymOp upload_op(Matrix& M, const OpHost& H, int K, const void* pool0, const void* pool1,
                       const void* pool0_32, const void* pool1_32) {
  SymOp op;
  op.K = K;
  op.nrows = (int)H.rowptr.size() - 1;
  op.nnz = (int)H.col.size();
  cudaStream_t s = M.stream;
  auto up = [&](const void* src, size_t bytes) {
    void* d = M.alloc(std::max<size_t>(bytes, 8));
    if (bytes) H2_CUDA(cudaMemcpyAsync(d, src, bytes, cudaMemcpyHostToDevice, s));
    return d;
  };
  op.rowptr = (int*)up(H.rowptr.data(), sizeof(int) * H.rowptr.size());
  op.col = (int*)up(H.col.data(), sizeof(int) * H.col.size());
  std::vector<const void*> p(op.nnz), p32(op.nnz);
  size_t b64 = (size_t)K * K * fmt_bytes(M.fmt), b32 = (size_t)K * K * 4;
  for (int e = 0; e < op.nnz; ++e) {
    p[e] = (const char*)(H.pool[e] ? pool1 : pool0) + H.blk[e] * b64;
    const void* q = H.pool[e] ? pool1_32 : pool0_32;
    p32[e] = q ? (const char*)q + H.blk[e] * b32 : nullptr;
  }
  op.blk = (const void**)up(p.data(), sizeof(void*) * p.size());
  op.blk32 = (const void**)up(p32.data(), sizeof(void*) * p32.size());
  int64_t noff = 0;
  for (int t = 0; t < op.nrows; ++t)
    for (int e = H.rowptr[t]; e < H.rowptr[t + 1]; ++e) noff += (H.col[e] != t);
  op.noff = noff;
  return op;
}

// Coupling rows of levels t*..top (+ the P_i blocks of level top when i >= 2).
static OpHost coupling_rows(const Matrix& M, int top, int i) {
  OpHost H;
  H.rowptr.push_back(0);
  for (int ell = M.tstar; ell <= top; ++ell) {
    const HostCSR& F = M.far[ell];
    auto ubF = ubase(F, 1 << ell, true);
    const HostCSR* Ip = (i >= 2 && ell == top) ? &M.inadm[ell] : nullptr;
    std::vector<int64_t> ubI;
    if (Ip) ubI = ubase(*Ip, 1 << ell, false);
    for (int t = 0; t < (1 << ell); ++t) {
      // merge far (strict upper) and close (upper incl. diagonal) columns
      std::vector<std::pair<int, std::pair<int, int64_t>>> ent;
      for (int e = F.rowptr[t]; e < F.rowptr[t + 1]; ++e)
        if (F.col[e] > t)
          ent.push_back({F.col[e], {0, M.s_level_base[ell] + ubF[t] + upper_pos(F, t, F.col[e], true)}});
      if (Ip)
        for (int e = Ip->rowptr[t]; e < Ip->rowptr[t + 1]; ++e)
          if (Ip->col[e] >= t) ent.push_back({Ip->col[e], {1, ubI[t] + upper_pos(*Ip, t, Ip->col[e], false)}});
      std::sort(ent.begin(), ent.end());
      for (auto& en : ent) {
        H.col.push_back(M.slot0(ell) + en.first);
        H.pool.push_back(en.second.first);
        H.blk.push_back(en.second.second);
      }
      H.rowptr.push_back((int)H.col.size());
    }
  }
  return H;
}

void setup_operators(Matrix& M) {
  cudaStream_t s = M.stream;
  const int L = M.L;
  // close part of level 1
  {
    OpHost H;
    const HostCSR& N = M.inadm[L];
    H.rowptr.push_back(0);
    int64_t b = 0;
    for (int t = 0; t < (1 << L); ++t) {
      for (int e = N.rowptr[t]; e < N.rowptr[t + 1]; ++e)
        if (N.col[e] >= t) {
          H.col.push_back(N.col[e]);
          H.blk.push_back(b++);
          H.pool.push_back(0);
        }
      H.rowptr.push_back((int)H.col.size());
    }
    M.opD = upload_op(M, H, M.KD, M.poolD.p, nullptr, M.poolD32.p, nullptr);
  }
  M.opC.assign(M.lev + 1, SymOp{});
  if (M.tstar >= 0) {
    for (int i = 1; i <= M.lev; ++i) {
      if (M.apply_only && i > 1) break;
      int top = (i == 1) ? L : L - i + 2;
      OpHost H = coupling_rows(M, top, i);
      const void* pP = (i >= 2) ? M.poolP[i].p : nullptr;
      const void* pP32 = (i >= 2 && M.with_f32) ? M.poolP32[i].p : nullptr;
      M.opC[i] = upload_op(M, H, M.KC, M.poolS.p, pP, M.with_f32 ? M.poolS32.p : nullptr, pP32);
    }
    // transposed copies of the transfers and leaf bases (coalesced upward pass) and the
    // swizzled transfer pools; a sibling matrix already has its base's
    size_t nu = (size_t)(1 << L), ne = (size_t)M.nslots();
    if (!M.d_UT) {
      double* UT = (double*)M.alloc(sizeof(double) * nu * M.KD * M.KC);
      double* ET = (double*)M.alloc(sizeof(double) * ne * M.KC * M.KC);
      { k_transpose_blocks<<<(int)nu, 256, 0, s>>>(M.d_U, M.KD, M.KC, UT); ::h2mg::count_launch(); }
      H2_LAUNCH_CHECK();
      { k_transpose_blocks<<<(int)ne, 256, 0, s>>>(M.d_E, M.KC, M.KC, ET); ::h2mg::count_launch(); }
      H2_LAUNCH_CHECK();
      M.d_UT = UT;
      M.d_ET = ET;
      M.poolE.bytes = ne * M.KC * M.KC * fmt_bytes(M.fmt);
      M.poolE.p = M.alloc(M.poolE.bytes);
      { k_swizzle_blocks<<<(int)ne, 256, 0, s>>>(M.d_E, M.KC, M.poolE.p, M.fmt); ::h2mg::count_launch(); }
      H2_LAUNCH_CHECK();
    }
    if (M.with_f32) {
      M.poolE32.bytes = ne * M.KC * M.KC * 4;
      M.poolE32.p = M.alloc(M.poolE32.bytes);
      { k_swizzle_blocks<<<(int)ne, 256, 0, s>>>(M.d_E, M.KC, M.poolE32.p, FMT_F32); ::h2mg::count_launch(); }
      H2_LAUNCH_CHECK();
      float* UT32 = (float*)M.alloc(sizeof(float) * nu * M.KD * M.KC);
      float* ET32 = (float*)M.alloc(sizeof(float) * ne * M.KC * M.KC);
      { k_transpose_blocks32<<<(int)nu, 256, 0, s>>>(M.d_U32, M.KD, M.KC, UT32); ::h2mg::count_launch(); }
      H2_LAUNCH_CHECK();
      { k_transpose_blocks32<<<(int)ne, 256, 0, s>>>(M.d_E32, M.KC, M.KC, ET32); ::h2mg::count_launch(); }
      H2_LAUNCH_CHECK();
      M.d_UT32 = UT32;
      M.d_ET32 = ET32;
    }
  }
  // product workspaces hold up to NRMAX interleaved columns
  size_t ncoef = (size_t)std::max(M.nslots(), 1) * M.KC * NRMAX;
  size_t npts = (size_t)(1 << L) * M.KD * NRMAX;
  M.wx.p = M.alloc(8 * ncoef);
  M.wyrow.p = M.alloc(8 * ncoef);
  M.wyc.p = M.alloc(8 * ncoef);
  M.wxp.p = M.alloc(8 * npts);
  M.wyp.p = M.alloc(8 * npts);
  H2_CUDA(cudaStreamSynchronize(s));
}

template <int FMT, int NR>
static void launch_bsgemv(Matrix& M, const SymOp& op, bool f32, const void* x, void* yrow, cudaStream_t s,
                          int force_split = 0) {
  using vt = typename Ar<FMT>::vec_t;
  using yt = typename Ar<FMT>::yo_t;
  if (op.nrows == 0) return;
  H2_CUDA(cudaMemsetAsync(yrow, 0, sizeof(yt) * (size_t)op.nrows * op.K * NR, s));
  // CTAs per block row: the autotuner's choice, else enough CTAs to fill the GPU when
  // the operator has few block rows
  const int tuned = op.split[FMT == FMT_DD ? FMT_F64 : FMT][nr_index(NR)];
  const int split = force_split > 0 ? force_split : (tuned > 0 ? tuned : split_heuristic(op.nrows));
  const int grid = op.nrows * split;
  const void* const* blk = f32 ? op.blk32 : op.blk;
  Profile& P = M.prof;
  const bool rec = P.on && (!P.f32_only || FMT == FMT_F32);
  if (rec && P.cap_ev) {
    // inside a graph capture: the records become event nodes of the graph
    H2_REQUIRE(2 * P.cap_next + 2 <= P.cap_ev->size(), H2MG_ERR_UNSUPPORTED, "graph profiling events exhausted");
    H2_CUDA(cudaEventRecordWithFlags((*P.cap_ev)[2 * P.cap_next], s, cudaEventRecordExternal));
  } else if (rec) {
    if (P.used * 2 + 2 > P.ev.size()) {
      for (int i = 0; i < 64; ++i) {
        cudaEvent_t e;
        H2_CUDA(cudaEventCreate(&e));
        P.ev.push_back(e);
      }
    }
    H2_CUDA(cudaEventRecord(P.ev[2 * P.used], s));
  }
  switch (op.K) {
    case 16:
      { k_bsgemv<16, FMT, NR><<<grid, 256, 0, s>>>(op.rowptr, op.col, blk, (const vt*)x, (yt*)yrow, split); ::h2mg::count_launch(); }
      break;
    case 32:
      { k_bsgemv<32, FMT, NR><<<grid, 256, 0, s>>>(op.rowptr, op.col, blk, (const vt*)x, (yt*)yrow, split); ::h2mg::count_launch(); }
      break;
    case 64:
      { k_bsgemv<64, FMT, NR><<<grid, 256, 0, s>>>(op.rowptr, op.col, blk, (const vt*)x, (yt*)yrow, split); ::h2mg::count_launch(); }
      break;
    default:
      throw Error{H2MG_ERR_UNSUPPORTED, "block size not supported"};
  }
  H2_LAUNCH_CHECK();
  if (rec && P.cap_ev) {
    H2_CUDA(cudaEventRecordWithFlags((*P.cap_ev)[2 * P.cap_next + 1], s, cudaEventRecordExternal));
    P.cap_next++;
    P.cap_bytes->push_back((double)op.bytes(FMT == FMT_F32 ? 4 : 8, sizeof(vt) * NR));
  } else if (rec) {
    H2_CUDA(cudaEventRecord(P.ev[2 * P.used + 1], s));
    P.used++;
    P.bytes.push_back((double)op.bytes(FMT == FMT_F32 ? 4 : 8, sizeof(vt) * NR));
  }
}

// Upward pass from tree level `lb` (coefficients at xc + cslot(lb)) to level `ltop`:
// children of level l + 1 -> parents of level l, up to 3 levels per launch.
template <int FMT, int NR>
static void pass_up(const Matrix& M, const char* epool, size_t eb, void* xc, int lb, int ltop, cudaStream_t s) {
  using vt = typename Ar<FMT>::vec_t;
  const int KC = M.KC;
  auto cslot = [&](int ell) { return (vt*)xc + (size_t)M.slot0(ell) * KC * NR; };
  for (int lc = lb; lc > ltop;) {
    const int steps = std::min(3, lc - ltop);
    PassLevels pl{};
    for (int k = 0; k < steps; ++k) {
      pl.E[k] = epool + (size_t)M.slot0(lc - k) * KC * KC * eb;
      pl.out[k] = cslot(lc - k - 1);
      pl.n[k] = 1 << (lc - k);
    }
    const int grid = ceil_div(1 << lc, 8);
    switch (KC) {
      case 16: { k_up_multi<16, FMT, NR><<<grid, 256, 0, s>>>(pl, steps, cslot(lc)); ::h2mg::count_launch(); } break;
      case 32: { k_up_multi<32, FMT, NR><<<grid, 256, 0, s>>>(pl, steps, cslot(lc)); ::h2mg::count_launch(); } break;
      default: { k_up_multi<64, FMT, NR><<<grid, 256, 0, s>>>(pl, steps, cslot(lc)); ::h2mg::count_launch(); } break;
    }
    H2_LAUNCH_CHECK();
    lc -= steps;
  }
}

// Downward pass from the coupling top level ts to level `lbot`, up to 4 levels per
// launch; the last level goes to yout (when given) instead of the coefficient buffer.
template <int FMT, int NR>
static void pass_down(const Matrix& M, const char* epool, size_t eb, const void* yrow, void* yc, int ts, int lbot,
                      double* yout, int64_t ldo, cudaStream_t s) {
  using vt = typename Ar<FMT>::vec_t;
  using yt = typename Ar<FMT>::yo_t;
  const int KC = M.KC;
  auto cslot = [&](int ell) { return (vt*)yc + (size_t)M.slot0(ell) * KC * NR; };
  for (int lt = ts; lt <= lbot;) {
    const int steps = std::min(4, lbot - lt + 1);
    PassLevels pl{};
    for (int k = 0; k < steps; ++k) {
      const int ell = lt + k;
      pl.E[k] = ell > ts ? epool + (size_t)M.slot0(ell) * KC * KC * eb : nullptr;
      pl.out[k] = cslot(ell);
      pl.slot[k] = M.slot0(ell);
      pl.n[k] = 1 << ell;
    }
    const vt* ypar = lt > ts ? cslot(lt - 1) : nullptr;
    double* yo = (lt + steps - 1 == lbot) ? yout : nullptr;
    const int grid = 1 << lt;
    switch (KC) {
      case 16: { k_down_multi<16, FMT, NR><<<grid, 256, 0, s>>>(pl, steps, (const yt*)yrow, ypar, yo, ldo); ::h2mg::count_launch(); } break;
      case 32: { k_down_multi<32, FMT, NR><<<grid, 256, 0, s>>>(pl, steps, (const yt*)yrow, ypar, yo, ldo); ::h2mg::count_launch(); } break;
      default: { k_down_multi<64, FMT, NR><<<grid, 256, 0, s>>>(pl, steps, (const yt*)yrow, ypar, yo, ldo); ::h2mg::count_launch(); } break;
    }
    H2_LAUNCH_CHECK();
    lt += steps;
  }
}

// y = A_i x for NR columns (x, y column-major with leading dimensions ldx, ldy).
template <int FMT, class BT, int NR>
static void apply_impl(Matrix& M, int i, const double* x, int64_t ldx, double* y, int64_t ldy, cudaStream_t s,
                       const BT* U, const BT* UT, const ApplyWork* ws = nullptr) {
  using vt = typename Ar<FMT>::vec_t;
  using yt = typename Ar<FMT>::yo_t;
  const int L = M.L, KC = M.KC, KD = M.KD, ts = M.tstar;
  const bool f32 = (FMT == FMT_F32);
  vt* xc = (vt*)(ws ? ws->xc : M.wx.p);
  yt* yr = (yt*)(ws ? ws->yr : M.wyrow.p);
  vt* yc = (vt*)(ws ? ws->yc : M.wyc.p);
  const char* epool = (const char*)(FMT == FMT_F32 ? M.poolE32.p : M.poolE.p);
  const size_t eb = FMT == FMT_F32 ? 4 : 8;
  auto cslot = [&](int ell) { return (size_t)M.slot0(ell) * KC * NR; };   // first element of a level
  if (i == 1) {
    vt* xp = (vt*)(ws ? ws->xp : M.wxp.p);
    yt* yp = (yt*)(ws ? ws->yp : M.wyp.p);
    // padded slots must read as zero: the buffer is shared by every format and column
    // count, so whatever an earlier product left there (possibly the halves of float64
    // values, which as floats can be NaN) is cleared first
    H2_CUDA(cudaMemsetAsync(xp, 0, sizeof(vt) * (size_t)(1 << L) * KD * NR, s));
    { k_pts_in<FMT, NR><<<ceil_div(M.n, 256), 256, 0, s>>>(x, ldx, M.d_slot_of, M.n, xp); ::h2mg::count_launch(); }
    H2_LAUNCH_CHECK();
    if (ts >= 0) {
      { k_up_leaf<FMT, BT, NR><<<1 << L, std::max(KC, 32), 0, s>>>(UT, KD, KC, xp, xc + cslot(L)); ::h2mg::count_launch(); }
      H2_LAUNCH_CHECK();
      pass_up<FMT, NR>(M, epool, eb, xc, L, ts, s);
    }
    launch_bsgemv<FMT, NR>(M, M.opD, f32, xp, yp, s);
    if (ts >= 0) {
      launch_bsgemv<FMT, NR>(M, M.opC[1], f32, xc, yr, s);
      pass_down<FMT, NR>(M, epool, eb, yr, yc, ts, L, nullptr, 0, s);
    }
    { k_leaf_final<FMT, BT, NR><<<1 << L, std::max(KD, 32), 0, s>>>(
        KD, KC, yp, ts >= 0 ? U : nullptr, ts >= 0 ? yc + cslot(L) : nullptr, M.d_leafoff, M.d_perm, y, ldy);
      ::h2mg::count_launch(); }
    H2_LAUNCH_CHECK();
    return;
  }
  const int m = L - i + 2;
  const int64_t nm = (int64_t)(1 << m) * KC;
  { k_coef_in<FMT, NR><<<ceil_div(nm, 256), 256, 0, s>>>(x, ldx, nm, xc + cslot(m)); ::h2mg::count_launch(); }
  H2_LAUNCH_CHECK();
  pass_up<FMT, NR>(M, epool, eb, xc, m, ts, s);
  launch_bsgemv<FMT, NR>(M, M.opC[i], f32, xc, yr, s);
  pass_down<FMT, NR>(M, epool, eb, yr, yc, ts, m, y, ldy, s);
}

template <int FMT, class BT>
static void apply_cols(Matrix& M, int i, const double* x, int64_t ldx, double* y, int64_t ldy, int nr,
                       cudaStream_t s, const BT* U, const BT* UT) {
  int c = 0;
  while (c < nr) {
    int left = nr - c;
    if constexpr (FMT == FMT_F32) {
      if (left >= 4) {
        apply_impl<FMT, BT, 4>(M, i, x + c * ldx, ldx, y + c * ldy, ldy, s, U, UT);
        c += 4;
        continue;
      }
    }
    if (left >= 2) {
      apply_impl<FMT, BT, 2>(M, i, x + c * ldx, ldx, y + c * ldy, ldy, s, U, UT);
      c += 2;
    } else {
      apply_impl<FMT, BT, 1>(M, i, x + c * ldx, ldx, y + c * ldy, ldy, s, U, UT);
      c += 1;
    }
  }
}

// Y = A_i X for nr columns; columns go through the block products NR at a time
// (4 for the FP32 copy, 2 for float64 / double-float), each block read once per group.
void apply_level_multi(Matrix& M, int i, bool f32, const double* x, int64_t ldx, double* y, int64_t ldy, int nr,
                       cudaStream_t s) {
  if (f32) {
    H2_REQUIRE(M.with_f32, H2MG_ERR_INVALID_ARG, "matrix was built without an FP32 copy");
    apply_cols<FMT_F32, float>(M, i, x, ldx, y, ldy, nr, s, M.d_U32, M.d_UT32);
  } else if (M.fmt == FMT_DF) {
    apply_cols<FMT_DF, double>(M, i, x, ldx, y, ldy, nr, s, M.d_U, M.d_UT);
  } else {
    apply_cols<FMT_F64, double>(M, i, x, ldx, y, ldy, nr, s, M.d_U, M.d_UT);
  }
}

void apply_level(Matrix& M, int i, bool f32, const double* x, double* y, cudaStream_t s) {
  int64_t n = level_size(M, i);
  apply_level_multi(M, i, f32, x, n, y, n, 1, s);
}

// y = A x at level 1 from the float64 blocks with double-double vectors and sums (one
// column): the outer residual b - A x of a solve whose x is much larger than b, where
// the float64 sum would round at the level of the residual itself.
void apply_level1_dd(Matrix& M, const double* x, double* y, cudaStream_t s) {
  H2_REQUIRE(M.fmt == FMT_F64, H2MG_ERR_INVALID_ARG, "the double-double product needs float64 storage");
  apply_impl<FMT_DD, double, 1>(M, 1, x, M.n, y, M.n, s, M.d_U, M.d_UT);
}

// Level-1 product in the primary format with caller-supplied workspace (the
// handle's own buffers are not touched).
void apply_level1_ws(Matrix& M, const double* x, double* y, cudaStream_t s, const ApplyWork& ws) {
  if (M.fmt == FMT_DF)
    apply_impl<FMT_DF, double, 1>(M, 1, x, M.n, y, M.n, s, M.d_U, M.d_UT, &ws);
  else
    apply_impl<FMT_F64, double, 1>(M, 1, x, M.n, y, M.n, s, M.d_U, M.d_UT, &ws);
}

// Bytes of each workspace region of the level-1 product.
void apply_level1_ws_sizes(const Matrix& M, size_t* coef, size_t* pts) {
  *coef = 8 * (size_t)std::max(M.nslots(), 1) * M.KC;
  *pts = 8 * (size_t)(1 << M.L) * M.KD;
}

// ----------------------------------------------------------------------------- autotuner
// Times `reps` launches of one block product with row split `split` on the handle's
// workspaces (contents irrelevant: only the launch time is wanted).
template <int FMT, int NR>
static float time_product(Matrix& M, SymOp& op, bool pts, int split, int reps, cudaStream_t s, cudaEvent_t e0,
                          cudaEvent_t e1) {
  const bool f32 = FMT == FMT_F32;
  void* x = pts ? M.wxp.p : M.wx.p;
  void* y = pts ? M.wyp.p : M.wyrow.p;
  launch_bsgemv<FMT, NR>(M, op, f32, x, y, s, split);   // warm-up
  H2_CUDA(cudaEventRecord(e0, s));
  for (int r = 0; r < reps; ++r) launch_bsgemv<FMT, NR>(M, op, f32, x, y, s, split);
  H2_CUDA(cudaEventRecord(e1, s));
  H2_CUDA(cudaEventSynchronize(e1));
  float ms = 0.f;
  H2_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  return ms / reps;
}

template <int FMT, int NR>
static void tune_one(Matrix& M, SymOp& op, bool pts, int opi, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1,
                     std::vector<double>& rep) {
  if (op.nrows == 0 || op.nnz == 0) return;
  const int heur = split_heuristic(op.nrows);
  const int cands[] = {1, 2, 4, 8, 16, 32, 64};
  const float base = time_product<FMT, NR>(M, op, pts, heur, 3, s, e0, e1);
  float best = base;
  int bs = heur;
  for (int c : cands) {
    if (c == heur || (int64_t)op.nrows * c > (1 << 22)) continue;
    if (c > 1 && op.nnz < op.nrows * c) continue;       // more CTAs than blocks: idle CTAs
    const float t = time_product<FMT, NR>(M, op, pts, c, 3, s, e0, e1);
    if (t < best) {
      best = t;
      bs = c;
    }
  }
  op.split[FMT][nr_index(NR)] = bs;
  rep.insert(rep.end(), {(double)opi, (double)NR, (double)base, (double)best});
}

// Every operator of the hierarchy (index 0 = the close part of level 1, i = the
// coupling operator of level i), in the primary format for 1 and 2 columns and, with
// an FP32 copy, in FP32 for 1, 2 and 4 columns.
int autotune_products(Matrix& M, cudaStream_t s, double* out, int cap) {
  H2_REQUIRE(!M.prof.on, H2MG_ERR_INVALID_ARG, "stop h2mg_profile before tuning");
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  H2_CUDA(cudaEventCreate(&e0));
  H2_CUDA(cudaEventCreate(&e1));
  std::vector<double> rep;
  try {
    for (int oi = 0; oi < (int)M.opC.size(); ++oi) {
      SymOp& op = oi == 0 ? M.opD : M.opC[oi];
      const bool pts = oi == 0;
      if (M.fmt == FMT_DF) {
        tune_one<FMT_DF, 1>(M, op, pts, oi, s, e0, e1, rep);
        tune_one<FMT_DF, 2>(M, op, pts, oi, s, e0, e1, rep);
      } else {
        tune_one<FMT_F64, 1>(M, op, pts, oi, s, e0, e1, rep);
        tune_one<FMT_F64, 2>(M, op, pts, oi, s, e0, e1, rep);
      }
      if (M.with_f32 && op.blk32) {
        tune_one<FMT_F32, 1>(M, op, pts, oi, s, e0, e1, rep);
        tune_one<FMT_F32, 2>(M, op, pts, oi, s, e0, e1, rep);
        tune_one<FMT_F32, 4>(M, op, pts, oi, s, e0, e1, rep);
      }
    }
  } catch (...) {
    best_effort(cudaEventDestroy(e0), "cudaEventDestroy (tune)");
    best_effort(cudaEventDestroy(e1), "cudaEventDestroy (tune)");
    throw;
  }
  best_effort(cudaEventDestroy(e0), "cudaEventDestroy (tune)");
  best_effort(cudaEventDestroy(e1), "cudaEventDestroy (tune)");
  const int n = (int)rep.size() / 4;
  if (out)
    for (int k = 0; k < std::min(n, cap); ++k)
      for (int j = 0; j < 4; ++j) out[4 * k + j] = rep[4 * k + j];
  return n;
}

// Algorithmic bytes of one A_i apply in the primary format: every stored block once,
// the transfers (and leaf bases at i = 1) twice, the input and output vectors once.
int64_t apply_bytes(const Matrix& M, int i) {
  int64_t eb = fmt_bytes(M.fmt);
  int64_t bytes = 0;
  if (i == 1) {
    bytes += (int64_t)M.opD.nnz * M.KD * M.KD * eb + 2 * 8 * M.n;
    if (M.tstar >= 0) {
      bytes += (int64_t)M.opC[1].nnz * M.KC * M.KC * eb;
      bytes += 2 * 8 * ((int64_t)(1 << M.L) * M.KD * M.KC);
      for (int ell = M.tstar + 1; ell <= M.L; ++ell) bytes += 2 * 8 * ((int64_t)(1 << ell) * M.KC * M.KC);
    }
    return bytes;
  }
  int m = M.L - i + 2;
  bytes += (int64_t)M.opC[i].nnz * M.KC * M.KC * eb + 2 * 8 * ((int64_t)(1 << m) * M.KC);
  for (int ell = M.tstar + 1; ell <= m; ++ell) bytes += 2 * 8 * ((int64_t)(1 << ell) * M.KC * M.KC);
  return bytes;
}

}  // namespace h2mg
