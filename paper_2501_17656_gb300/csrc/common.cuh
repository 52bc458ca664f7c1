// common.cuh -- shared device/host helpers of the H2-MG library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string>

#include "../../include/h2mg.h"

namespace h2mg {

// ----------------------------------------------------------------------------- errors
struct Error {
  h2mg_status status;
  std::string msg;
};

void set_error(const std::string& msg);
void count_launch();   // every kernel launch of the library is counted (h2mg_launch_count)
void add_launches(int64_t k);
void best_effort(cudaError_t e, const char* what);   // unchecked release: report under H2MG_DEBUG, clear   // kernels run by a graph replay (negative: undo capture-time counts)

#define H2_CUDA(call)                                                                   \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess) {                                                            \
      throw ::h2mg::Error{e_ == cudaErrorMemoryAllocation ? H2MG_ERR_OOM : H2MG_ERR_CUDA, \
                          std::string(#call) + ": " + cudaGetErrorString(e_)};          \
    }                                                                                   \
  } while (0)

#define H2_LAUNCH_CHECK() H2_CUDA(cudaGetLastError())

#define H2_REQUIRE(cond, code, text)                                                    \
  do {                                                                                  \
    if (!(cond)) throw ::h2mg::Error{code, std::string(text)};                          \
  } while (0)

inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// ----------------------------------------------------------------------------- kernels
// k(x, y) off the diagonal; see h2mg_kernel_kind. Evaluated in float64.
struct KernelParams {
  int kind;
  double length;
  double nugget;
  int degree;
};

__host__ __device__ inline double kernel_eval(const KernelParams& kp, const double* x,
                                              const double* y, int dim) {
  if (kp.kind == H2MG_K_POLY) {
    double dot = 0.0;
    for (int d = 0; d < dim; ++d) dot = fma(x[d], y[d], dot);
    double b = 1.0 + dot, p = 1.0;
    for (int e = 0; e < kp.degree; ++e) p *= b;
    return p;
  }
  double r2 = 0.0;
  for (int d = 0; d < dim; ++d) {
    double t = x[d] - y[d];
    r2 = fma(t, t, r2);
  }
  switch (kp.kind) {
    case H2MG_K_GAUSSIAN:
      return exp(-r2 / (kp.length * kp.length));
    case H2MG_K_EXPONENTIAL:
      return exp(-sqrt(r2) / kp.length);
    case H2MG_K_MATERN32: {
      double u = 1.7320508075688772 * sqrt(r2) / kp.length;
      return (1.0 + u) * exp(-u);
    }
    case H2MG_K_DMATERN32_DL: {
      double u = 1.7320508075688772 * sqrt(r2) / kp.length;
      return (3.0 * r2 / (kp.length * kp.length * kp.length)) * exp(-u);
    }
    case H2MG_K_LAPLACE_SL:
      return 1.0 / (12.566370614359172 * sqrt(r2));
    default:
      return 0.0;
  }
}

// k(x, x): value at zero distance (POLY depends on x; LAPLACE_SL is singular).
__host__ __device__ inline double kernel_self(const KernelParams& kp, const double* x, int dim) {
  switch (kp.kind) {
    case H2MG_K_GAUSSIAN:
    case H2MG_K_EXPONENTIAL:
    case H2MG_K_MATERN32:
      return 1.0;
    case H2MG_K_DMATERN32_DL:
      return 0.0;
    case H2MG_K_POLY: {
      double dot = 0.0;
      for (int d = 0; d < dim; ++d) dot = fma(x[d], x[d], dot);
      double b = 1.0 + dot, p = 1.0;
      for (int e = 0; e < kp.degree; ++e) p *= b;
      return p;
    }
    default:
      return 0.0;
  }
}

// ----------------------------------------------------------------------------- double-float
// A double-float value hi + lo with |lo| <= ulp(hi)/2 after normalisation. Products
// and sums use the error-free transformations of Dekker (two-product via FMA) and
// Knuth (two-sum); accumulators are kept unnormalised ("sloppy" sum) and
// normalised once when read out.
struct df2 {
  float hi, lo;
};

__device__ __forceinline__ df2 df_from_double(double v) {
  float h = __double2float_rn(v);
  float l = __double2float_rn(v - (double)h);
  return {h, l};
}
__device__ __forceinline__ double df_to_double(df2 a) { return (double)a.hi + (double)a.lo; }

// acc += m * x  (all double-float)
__device__ __forceinline__ void df_fma(float& ah, float& al, float mh, float ml, float xh, float xl) {
  float p = mh * xh;
  float e = fmaf(mh, xh, -p);
  e = fmaf(mh, xl, e);
  e = fmaf(ml, xh, e);
  float s = ah + p;
  float bb = s - ah;
  float err = (ah - (s - bb)) + (p - bb);
  ah = s;
  al = al + (err + e);
}
// a += b (double-float, unnormalised accumulators)
__device__ __forceinline__ void df_add(float& ah, float& al, float bh, float bl) {
  float s = ah + bh;
  float bb = s - ah;
  float err = (ah - (s - bb)) + (bh - bb);
  ah = s;
  al = al + (err + bl);
}
__device__ __forceinline__ void df_norm(float& ah, float& al) {
  float s = ah + al;
  al = al - (s - ah);
  ah = s;
}

// ----------------------------------------------------------------------------- block layout
// Every K x K block (K in {16, 32, 64}) of D, S and P_i is stored in the order in
// which the block-GEMV warp reads it: lane l owns rows 8*(l % LPC) .. +7 of the
// columns (l / LPC) + CPP * t, t = 0 .. K*K/256 - 1 (LPC = K/8 lanes per column,
// CPP = 32/LPC columns per pass). Each pass is read with P = 8/V 16-byte loads per
// lane, V = elements per 16 bytes, so every warp load is one contiguous 512-byte
// segment. swz(i, j) is the storage position of entry (row i, column j).
__host__ __device__ inline int64_t swz(int i, int j, int K, int V) {
  int LPC = K / 8, CPP = 32 / LPC;
  int t = j / CPP;
  int lane = (j % CPP) * LPC + i / 8;
  int ii = i % 8;
  int P = 8 / V;
  int k = ii / V, sub = ii % V;
  return ((int64_t)(t * P + k) * 32 + lane) * V + sub;
}

// Element formats of stored blocks. FMT_DD is not a storage format: float64 blocks
// read by a product whose vectors and sums are double-double (the extended-precision
// outer residual).
enum Fmt { FMT_F64 = 0, FMT_DF = 1, FMT_F32 = 2, FMT_DD = 3 };
inline int fmt_bytes(int fmt) { return fmt == FMT_F32 ? 4 : 8; }
inline int fmt_vec(int fmt) { return fmt == FMT_F32 ? 4 : 2; }

// ----------------------------------------------------------------------------- double-double
// A value hi + lo of two doubles: Dekker's product (exact through FMA) and Knuth's
// two-sum give a ~106-bit accumulation; accumulators are kept unnormalised and
// normalised when read out, like the double-float ones above.
__device__ __forceinline__ void dd_fma(double& ah, double& al, double m, double xh, double xl) {
  const double p = m * xh;
  double e = fma(m, xh, -p);
  e = fma(m, xl, e);
  const double s = ah + p;
  const double bb = s - ah;
  const double err = (ah - (s - bb)) + (p - bb);
  ah = s;
  al = al + (err + e);
}
__device__ __forceinline__ void dd_add(double& ah, double& al, double bh, double bl) {
  const double s = ah + bh;
  const double bb = s - ah;
  const double err = (ah - (s - bb)) + (bh - bb);
  ah = s;
  al = al + (err + bl);
}
__device__ __forceinline__ void dd_norm(double& ah, double& al) {
  const double s = ah + al;
  al = al - (s - ah);
  ah = s;
}
// *p += v in double-double with two atomics: the hardware rounds old + v.x exactly as
// two-sum's sum does, so the rounding error of this add is recovered from the returned
// old value and added to the low word with v.y.
__device__ __forceinline__ void dd_atomic_add(double2* p, double2 v) {
  const double old = atomicAdd(&p->x, v.x);
  const double s = old + v.x;
  const double bb = s - old;
  const double err = (old - (s - bb)) + (v.x - bb);
  atomicAdd(&p->y, err + v.y);
}

}  // namespace h2mg
