// capi.cu -- the extern "C" entry points declared in include/h2mg.h.
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <string>

#include "internal.h"

namespace h2mg {

static thread_local std::string g_last_error;
void set_error(const std::string& msg) { g_last_error = msg; }

static std::atomic<int64_t> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void add_launches(int64_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

void* Matrix::alloc(size_t bytes) {
  void* p = nullptr;
  if (bytes == 0) bytes = 8;
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    throw Error{e == cudaErrorMemoryAllocation ? H2MG_ERR_OOM : H2MG_ERR_CUDA,
                "cudaMalloc(" + std::to_string(bytes) + " B): " + cudaGetErrorString(e)};
  }
  owned.push_back({p, bytes});
  e = cudaMemsetAsync(p, 0, bytes, stream);
  if (e != cudaSuccess) throw Error{H2MG_ERR_CUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e)};
  return p;
}

void Matrix::free_owned(void* p) {
  if (!p) return;
  for (auto& d : owned)
    if (d.p == p) {
      // queued work of the handle's stream may still use it
      best_effort(cudaStreamSynchronize(stream), "cudaStreamSynchronize (free)");
      best_effort(cudaFree(d.p), "cudaFree (build scratch)");
      d.p = nullptr;
      d.bytes = 0;
      return;
    }
}

void best_effort(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return;
  if (std::getenv("H2MG_DEBUG")) std::fprintf(stderr, "[h2mg] %s failed: %s\n", what, cudaGetErrorString(e));
  cudaGetLastError();
}

Matrix::~Matrix() {
  if (stream) best_effort(cudaStreamSynchronize(stream), "cudaStreamSynchronize (release)");
  destroy_graphs(*this);
  destroy_panel_plan(*this);
  for (auto e : prof.ev) best_effort(cudaEventDestroy(e), "cudaEventDestroy (profile)");
  for (auto& d : owned)
    if (d.p) best_effort(cudaFree(d.p), "cudaFree (release)");
}

bool is_device_pointer(const void* p);
static bool is_device_ptr(const void* p) { return is_device_pointer(p); }
bool is_device_pointer(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// A device view of a caller buffer: the buffer itself, or a staged copy.
struct DevView {
  double* d = nullptr;
  bool staged = false;
  DevView(const double* p, int64_t n, bool copy_in, cudaStream_t s) {
    if (p == nullptr) return;
    if (is_device_ptr(p)) {
      d = const_cast<double*>(p);
    } else {
      staged = true;
      H2_CUDA(cudaMalloc(&d, sizeof(double) * std::max<int64_t>(n, 1)));
      if (copy_in) H2_CUDA(cudaMemcpyAsync(d, p, sizeof(double) * n, cudaMemcpyHostToDevice, s));
    }
  }
  void copy_out(double* host, int64_t n, cudaStream_t s) {
    if (staged) {
      H2_CUDA(cudaMemcpyAsync(host, d, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
      H2_CUDA(cudaStreamSynchronize(s));
    }
  }
  ~DevView() {
    if (staged && d) best_effort(cudaFree(d), "cudaFree (staging)");
  }
};

// A group of g columns of length n at stride ld, seen from the device. Device
// columns are used in place unless a packed layout (leading dimension n) is needed
// and ld != n; host columns (and those) are staged through a packed device copy.
struct ColsView {
  double* d = nullptr;
  int64_t ldd = 0;
  bool staged = false;
  const double* src;
  int64_t n, ld;
  int g;
  ColsView(const double* p, int64_t n_, int64_t ld_, int g_, bool copy_in, bool packed, cudaStream_t s)
      : src(p), n(n_), ld(ld_), g(g_) {
    if (is_device_ptr(p) && (!packed || ld == n || g == 1)) {
      d = const_cast<double*>(p);
      ldd = ld;
      return;
    }
    staged = true;
    ldd = n;
    H2_CUDA(cudaMalloc(&d, sizeof(double) * std::max<int64_t>(n * g, 1)));
    if (copy_in)
      H2_CUDA(cudaMemcpy2DAsync(d, sizeof(double) * n, p, sizeof(double) * ld, sizeof(double) * n, g,
                                cudaMemcpyDefault, s));
  }
  void copy_out(double* dst, cudaStream_t s) {
    if (!staged) return;
    H2_CUDA(cudaMemcpy2DAsync(dst, sizeof(double) * ld, d, sizeof(double) * n, sizeof(double) * n, g,
                              cudaMemcpyDefault, s));
    H2_CUDA(cudaStreamSynchronize(s));
  }
  ~ColsView() {
    if (staged && d) best_effort(cudaFree(d), "cudaFree (staging)");
  }
};

__global__ void k_point_weights(const int* __restrict__ perm, int64_t n, int dim, const double* __restrict__ Xt,
                                const double* __restrict__ w, const double* __restrict__ dg, KernelParams kp,
                                double* __restrict__ sw, double* __restrict__ dgo) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  int i = perm[p];
  double wi = w ? w[i] : 1.0;
  sw[p] = sqrt(wi);
  // single layer without an override: self-potential of a flat disk of area w_i
  double d = dg ? dg[i]
                : (kp.kind == H2MG_K_LAPLACE_SL ? 0.5 * sqrt(wi / 3.141592653589793)
                                                : wi * kernel_self(kp, Xt + p * dim, dim));
  dgo[p] = d + kp.nugget;
}

__global__ void k_check_pos(const double* __restrict__ v, int64_t n, int* __restrict__ flag) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && !(v[i] > 0.0 && isfinite(v[i]))) atomicOr(flag, 2);
}

static int pad_dim(int v) { return v <= 16 ? 16 : v <= 32 ? 32 : 64; }

static void build_all(Matrix& M, const double* points, const h2mg_kernel* k, const h2mg_build_opts* o) {
  cudaStream_t s = M.stream;
  M.d_flag = (int*)M.alloc(sizeof(int) * 4);
  DevView P(points, M.n * M.dim, true, s);
  build_tree(M, P.d);
  // weights and diagonal in tree order
  {
    DevView W(k->weights, k->weights ? M.n : 0, true, s);
    DevView G(k->diag, k->diag ? M.n : 0, true, s);
    if (k->weights) {
      H2_CUDA(cudaMemsetAsync(M.d_flag, 0, sizeof(int), s));
      { k_check_pos<<<ceil_div(M.n, 256), 256, 0, s>>>(W.d, M.n, M.d_flag); ::h2mg::count_launch(); }
      int h = 0;
      H2_CUDA(cudaMemcpyAsync(&h, M.d_flag, sizeof(int), cudaMemcpyDeviceToHost, s));
      H2_CUDA(cudaStreamSynchronize(s));
      H2_REQUIRE(h == 0, H2MG_ERR_INVALID_ARG, "weights must be positive and finite");
    }
    M.d_sw = (double*)M.alloc(sizeof(double) * M.n);
    M.d_dg = (double*)M.alloc(sizeof(double) * M.n);
    { k_point_weights<<<ceil_div(M.n, 256), 256, 0, s>>>(M.d_perm, M.n, M.dim, M.d_X, k->weights ? W.d : nullptr,
                                                       k->diag ? G.d : nullptr, M.kp, M.d_sw, M.d_dg); ::h2mg::count_launch(); }
    H2_LAUNCH_CHECK();
    H2_CUDA(cudaStreamSynchronize(s));
  }
  build_partition(M);
  M.KC = pad_dim(M.k);
  M.lev = o->coarse_level < 0 ? M.lev_nat : o->coarse_level;
  H2_REQUIRE(M.lev >= 1 && M.lev <= M.lev_nat, H2MG_ERR_INVALID_ARG,
             "coarse_level must be -1 or in [1, " + std::to_string(M.lev_nat) + "]");
  if (M.apply_only) M.lev = std::min(M.lev, 1);
  build_bases(M);
  build_blocks(M, nullptr);
  if (!M.apply_only) build_coarse_near(M);
  build_f32_copies(M);
  setup_operators(M);
  if (!M.apply_only) {
    build_dense_coarse(M);
    alloc_solve_workspace(M);
  }
  H2_CUDA(cudaStreamSynchronize(s));
}

// A sibling shares the base's tree, partition, bases and transfers (not owned) and
// owns only its block pools, operators and workspaces.
static void build_sibling(Matrix& B, const Matrix& A, const h2mg_kernel* k) {
  cudaStream_t s = B.stream;
  B.n = A.n; B.dim = A.dim; B.leaf = A.leaf; B.q = A.q; B.k = A.k; B.eta = A.eta;
  B.fmt = A.fmt; B.with_f32 = false; B.apply_only = true;
  B.basis = A.basis; B.basis_tol = A.basis_tol;
  B.L = A.L; B.KD = A.KD; B.KC = A.KC; B.tstar = A.tstar; B.lev_nat = A.lev_nat; B.lev = 1;
  B.offsets = A.offsets; B.far = A.far; B.inadm = A.inadm;
  B.d_perm = A.d_perm; B.d_slot_of = A.d_slot_of; B.d_leafoff = A.d_leafoff; B.d_X = A.d_X;
  B.d_box = A.d_box;
  // Chebyshev bases interpolate any smooth kernel and do not depend on the kernel's
  // parameters: the sibling shares them, and dK/dtheta's H2 form is the exact derivative
  // of K's. Skeleton bases are chosen from K's own values, which would not carry the
  // derivative kernel's far field: the sibling skeletonizes its own kernel on the same
  // tree and partition.
  const bool own_bases = A.basis == H2MG_BASIS_SKELETON;
  if (!own_bases) {
    B.d_nsw = A.d_nsw; B.d_skel = A.d_skel; B.h_rank = A.h_rank; B.d_nodes = A.d_nodes; B.d_rank = A.d_rank;
    B.d_U = A.d_U; B.d_E = A.d_E; B.d_R = A.d_R; B.d_UT = A.d_UT; B.d_ET = A.d_ET;
    B.poolE = A.poolE;            // swizzled transfers (shared, not owned)
  }
  B.d_flag = (int*)B.alloc(sizeof(int) * 4);
  B.d_sw = (double*)B.alloc(sizeof(double) * B.n);
  B.d_dg = (double*)B.alloc(sizeof(double) * B.n);
  { k_point_weights<<<ceil_div(B.n, 256), 256, 0, s>>>(B.d_perm, B.n, B.dim, B.d_X, nullptr, nullptr, B.kp,
                                                       B.d_sw, B.d_dg); ::h2mg::count_launch(); }
  H2_LAUNCH_CHECK();
  if (own_bases) build_bases(B);
  build_blocks(B, &A);
  setup_operators(B);
  H2_CUDA(cudaStreamSynchronize(s));
}

}  // namespace h2mg

using namespace h2mg;

template <class F>
static h2mg_status guard(F f) {
  try {
    g_last_error.clear();
    // an error left by an unchecked release (destructors) is not this call's
    const cudaError_t stale = cudaGetLastError();
    if (stale != cudaSuccess && std::getenv("H2MG_DEBUG"))
      std::fprintf(stderr, "[h2mg] CUDA error pending at entry: %s\n", cudaGetErrorString(stale));
    return f();
  } catch (const Error& e) {
    set_error(e.msg);
    return e.status;
  } catch (const std::bad_alloc&) {
    set_error("host allocation failed");
    return H2MG_ERR_OOM;
  } catch (...) {
    set_error("unknown error");
    return H2MG_ERR_CUDA;
  }
}

extern "C" {

const char* h2mg_error_string(h2mg_status s) {
  switch (s) {
    case H2MG_OK: return "success";
    case H2MG_ERR_INVALID_ARG: return "invalid argument";
    case H2MG_ERR_OOM: return "out of device memory";
    case H2MG_ERR_CUDA: return "CUDA error";
    case H2MG_ERR_NOT_SPD: return "coarse operator is not positive definite";
    case H2MG_ERR_NOT_CONVERGED: return "not converged";
    case H2MG_ERR_NAN: return "NaN or Inf encountered";
    case H2MG_ERR_TIMEOUT: return "device wait timed out";
    case H2MG_ERR_UNSUPPORTED: return "unsupported configuration";
  }
  return "unknown status";
}

const char* h2mg_last_error(void) { return g_last_error.c_str(); }

h2mg_status h2mg_build(const double* points, int64_t n, int dim, const h2mg_kernel* k,
                       const h2mg_build_opts* o, void* stream, h2mg_matrix* out) {
  if (out) *out = nullptr;
  return guard([&]() -> h2mg_status {
    H2_REQUIRE(out && points && k && o, H2MG_ERR_INVALID_ARG, "null pointer argument");
    H2_REQUIRE(n >= 1 && n <= (1ll << 30), H2MG_ERR_INVALID_ARG, "n must be in [1, 2^30]");
    H2_REQUIRE(dim >= 1 && dim <= 3, H2MG_ERR_INVALID_ARG, "dim must be 1, 2 or 3");
    H2_REQUIRE(o->leaf_size >= 2 && o->leaf_size <= 64, H2MG_ERR_INVALID_ARG, "leaf_size must be in [2, 64]");
    H2_REQUIRE(o->basis == H2MG_BASIS_CHEBYSHEV || o->basis == H2MG_BASIS_SKELETON, H2MG_ERR_INVALID_ARG,
               "basis must be H2MG_BASIS_CHEBYSHEV or H2MG_BASIS_SKELETON");
    int kk = 1;
    if (o->basis == H2MG_BASIS_CHEBYSHEV) {
      H2_REQUIRE(o->cheb_q >= 1, H2MG_ERR_INVALID_ARG, "cheb_q must be >= 1");
      for (int d = 0; d < dim; ++d) kk *= o->cheb_q;
      H2_REQUIRE(kk <= 64, H2MG_ERR_UNSUPPORTED, "rank q^dim must be <= 64");
    } else {
      H2_REQUIRE(o->rank_max >= 1 && o->rank_max <= 64, H2MG_ERR_INVALID_ARG, "rank_max must be in [1, 64]");
      H2_REQUIRE(o->basis_tol >= 0.0 && std::isfinite(o->basis_tol), H2MG_ERR_INVALID_ARG,
                 "basis_tol must be finite and >= 0");
      kk = o->rank_max;
    }
    H2_REQUIRE(o->eta >= 0.0 && std::isfinite(o->eta), H2MG_ERR_INVALID_ARG, "eta must be finite and >= 0");
    H2_REQUIRE(o->storage == H2MG_STORE_F64 || o->storage == H2MG_STORE_DF64, H2MG_ERR_INVALID_ARG,
               "storage must be H2MG_STORE_F64 or H2MG_STORE_DF64");
    H2_REQUIRE(k->kind >= 0 && k->kind <= H2MG_K_DMATERN32_DL, H2MG_ERR_INVALID_ARG, "unknown kernel kind");
    H2_REQUIRE(k->kind == H2MG_K_POLY || k->kind == H2MG_K_LAPLACE_SL || (k->length > 0 && std::isfinite(k->length)),
               H2MG_ERR_INVALID_ARG, "length must be > 0");
    H2_REQUIRE(k->kind != H2MG_K_POLY || (k->degree >= 0 && k->degree <= 16), H2MG_ERR_INVALID_ARG,
               "degree must be in [0, 16]");
    H2_REQUIRE(k->kind != H2MG_K_LAPLACE_SL || k->diag || k->weights, H2MG_ERR_INVALID_ARG,
               "the single-layer kernel needs panel areas (weights) or a diagonal override");
    H2_REQUIRE(std::isfinite(k->nugget), H2MG_ERR_INVALID_ARG, "nugget must be finite");
    auto* h = new h2mg_matrix_s();
    Matrix& M = h->M;
    M.n = n;
    M.dim = dim;
    M.kp = KernelParams{k->kind, k->length, k->nugget, k->degree};
    M.has_weights = k->weights != nullptr;
    M.has_diag = k->diag != nullptr;
    M.leaf = o->leaf_size;
    M.q = o->cheb_q;
    M.k = kk;
    M.eta = o->eta;
    M.basis = o->basis;
    M.basis_tol = o->basis_tol;
    M.fmt = o->storage == H2MG_STORE_DF64 ? FMT_DF : FMT_F64;
    M.with_f32 = o->with_f32 != 0;
    M.stream = (cudaStream_t)stream;
    try {
      build_all(M, points, k, o);
    } catch (...) {
      delete h;
      throw;
    }
    *out = h;
    return H2MG_OK;
  });
}

h2mg_status h2mg_destroy(h2mg_matrix A) {
  return guard([&]() -> h2mg_status {
    delete A;
    return H2MG_OK;
  });
}

h2mg_status h2mg_apply(h2mg_matrix A, const double* x, double* y, int nrhs, int64_t ld, void* stream) {
  return guard([&]() -> h2mg_status {
    H2_REQUIRE(A && x && y, H2MG_ERR_INVALID_ARG, "null pointer argument");
    Matrix& M = A->M;
    H2_REQUIRE(nrhs >= 1 && ld >= M.n, H2MG_ERR_INVALID_ARG, "need nrhs >= 1 and ld >= n");
    cudaStream_t s = (cudaStream_t)stream;
    for (int c = 0; c < nrhs; c += NRMAX) {
      const int g = std::min(NRMAX, nrhs - c);
      ColsView X(x + (int64_t)c * ld, M.n, ld, g, true, false, s), Y(y + (int64_t)c * ld, M.n, ld, g, false, false, s);
      apply_level_multi(M, 1, false, X.d, X.ldd, Y.d, Y.ldd, g, s);
      Y.copy_out(y + (int64_t)c * ld, s);
    }
    return H2MG_OK;
  });
}

h2mg_status h2mg_apply_ex(h2mg_matrix A, int precision, const double* x, double* y, int nrhs, int64_t ld,
                          void* stream) {
  return guard([&]() -> h2mg_status {
    H2_REQUIRE(A && x && y, H2MG_ERR_INVALID_ARG, "null pointer argument");
    Matrix& M = A->M;
    H2_REQUIRE(nrhs >= 1 && ld >= M.n, H2MG_ERR_INVALID_ARG, "need nrhs >= 1 and ld >= n");
    H2_REQUIRE(precision == H2MG_PREC_F64 || precision == H2MG_PREC_MIXED_F32 || precision == H2MG_PREC_TF32X3,
               H2MG_ERR_INVALID_ARG, "precision must be F64, MIXED_F32 or TF32X3");
    H2_REQUIRE(precision == H2MG_PREC_F64 || M.with_f32, H2MG_ERR_INVALID_ARG,
               "the FP32 and tensor-core products need a matrix built with_f32");
    H2_REQUIRE(precision != H2MG_PREC_TF32X3 || panel_supported(M), H2MG_ERR_UNSUPPORTED,
               "the tensor-core product needs leaf and rank blocks of 64");
    cudaStream_t s = (cudaStream_t)stream;
    if (precision == H2MG_PREC_TF32X3) {
      ColsView X(x, M.n, ld, nrhs, true, false, s), Y(y, M.n, ld, nrhs, false, false, s);
      apply_panel(M, X.d, X.ldd, Y.d, Y.ldd, nrhs, s);
      Y.copy_out(y, s);
      return H2MG_OK;
    }
    for (int c = 0; c < nrhs; c += NRMAX) {
      const int g = std::min(NRMAX, nrhs - c);
      ColsView X(x + (int64_t)c * ld, M.n, ld, g, true, false, s), Y(y + (int64_t)c * ld, M.n, ld, g, false, false, s);
      apply_level_multi(M, 1, precision == H2MG_PREC_MIXED_F32, X.d, X.ldd, Y.d, Y.ldd, g, s);
      Y.copy_out(y + (int64_t)c * ld, s);
    }
    return H2MG_OK;
  });
}

h2mg_status h2mg_solve(h2mg_matrix A, const double* b, double* x, int nrhs, int64_t ld,
                       const h2mg_solve_opts* o, h2mg_solve_info* info, void* stream) {
  return guard([&]() -> h2mg_status {
    H2_REQUIRE(A && b && x && o, H2MG_ERR_INVALID_ARG, "null pointer argument");
    Matrix& M = A->M;
    H2_REQUIRE(nrhs >= 1 && ld >= M.n, H2MG_ERR_INVALID_ARG, "need nrhs >= 1 and ld >= n");
    H2_REQUIRE(o->max_cycles >= 0 && o->n_f >= 0 && o->n_c >= 0 && o->tol >= 0, H2MG_ERR_INVALID_ARG,
               "bad solve options");
    H2_REQUIRE(o->outer >= H2MG_OUTER_VCYCLE && o->outer <= H2MG_OUTER_CG, H2MG_ERR_INVALID_ARG, "unknown outer loop");
    H2_REQUIRE(o->cycle >= H2MG_CYCLE_V && o->cycle <= H2MG_CYCLE_F, H2MG_ERR_INVALID_ARG, "unknown cycle type");
    H2_REQUIRE(o->residual_dd >= 0 && o->residual_dd <= 2, H2MG_ERR_INVALID_ARG, "residual_dd must be 0, 1 or 2");
    H2_REQUIRE(o->precision == H2MG_PREC_F64 || (o->precision == H2MG_PREC_MIXED_F32 && M.with_f32),
               H2MG_ERR_INVALID_ARG, "mixed precision needs a matrix built with_f32");
    H2_REQUIRE(!M.apply_only, H2MG_ERR_INVALID_ARG, "matrix was built for products only");
    if (!M.coarse_ok) throw Error{H2MG_ERR_NOT_SPD, "the coarsest operator is not positive definite"};
    cudaStream_t s = (cudaStream_t)stream;
    h2mg_status worst = H2MG_OK;
    h2mg_solve_info inf[NRMAX];
    for (int c = 0; c < nrhs; c += NRMAX) {
      const int g = std::min(NRMAX, nrhs - c);
      ColsView B(b + (int64_t)c * ld, M.n, ld, g, true, true, s), X(x + (int64_t)c * ld, M.n, ld, g, true, true, s);
      h2mg_status st = solve_multi(M, B.d, X.d, g, *o, inf, s);
      X.copy_out(x + (int64_t)c * ld, s);
      if (info)
        for (int j = 0; j < g; ++j) info[c + j] = inf[j];
      if (st != H2MG_OK && worst == H2MG_OK) worst = st;
    }
    if (worst != H2MG_OK) set_error(h2mg_error_string(worst));
    return worst;
  });
}

h2mg_status h2mg_solve_batched(int nprob, const h2mg_matrix* A, const double* const* b, double* const* x,
                               const h2mg_solve_opts* o, h2mg_solve_info* info, void* stream) {
  return guard([&]() -> h2mg_status {
    H2_REQUIRE(nprob >= 1 && A && b && x && o && info, H2MG_ERR_INVALID_ARG, "null pointer argument");
    H2_REQUIRE(o->max_cycles >= 0 && o->n_f >= 0 && o->n_c >= 0 && o->tol >= 0, H2MG_ERR_INVALID_ARG,
               "bad solve options");
    H2_REQUIRE(o->outer == H2MG_OUTER_VCYCLE || o->outer == H2MG_OUTER_FCG, H2MG_ERR_INVALID_ARG,
               "the batched solve runs repeated cycles or flexible CG");
    H2_REQUIRE(o->cycle >= H2MG_CYCLE_V && o->cycle <= H2MG_CYCLE_F, H2MG_ERR_INVALID_ARG, "unknown cycle type");
    std::vector<Matrix*> Ms(nprob);
    for (int p = 0; p < nprob; ++p) {
      H2_REQUIRE(A[p] && b[p] && x[p], H2MG_ERR_INVALID_ARG, "null pointer argument");
      Matrix& M = A[p]->M;
      H2_REQUIRE(o->precision == H2MG_PREC_F64 || (o->precision == H2MG_PREC_MIXED_F32 && M.with_f32),
                 H2MG_ERR_INVALID_ARG, "mixed precision needs matrices built with_f32");
      H2_REQUIRE(!M.apply_only, H2MG_ERR_INVALID_ARG, "matrix was built for products only");
      for (int q = 0; q < p; ++q)
        H2_REQUIRE(A[q] != A[p], H2MG_ERR_INVALID_ARG, "a matrix appears twice (use nrhs columns instead)");
      if (!M.coarse_ok) throw Error{H2MG_ERR_NOT_SPD, "the coarsest operator of a problem is not positive definite"};
      Ms[p] = &M;
    }
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<std::unique_ptr<DevView>> B, X;
    std::vector<const double*> bd(nprob);
    std::vector<double*> xd(nprob);
    for (int p = 0; p < nprob; ++p) {
      B.emplace_back(new DevView(b[p], Ms[p]->n, true, s));
      X.emplace_back(new DevView(x[p], Ms[p]->n, true, s));
      bd[p] = B.back()->d;
      xd[p] = X.back()->d;
    }
    const h2mg_status st = solve_batched(Ms, bd.data(), xd.data(), *o, info, s);
    for (int p = 0; p < nprob; ++p) X[p]->copy_out(x[p], Ms[p]->n, s);
    if (st != H2MG_OK) set_error(h2mg_error_string(st));
    return st;
  });
}

h2mg_status h2mg_query(h2mg_matrix A, int what, int arg, int64_t* value) {
  return guard([&]() -> h2mg_status {
    H2_REQUIRE(A && value, H2MG_ERR_INVALID_ARG, "null pointer argument");
    Matrix& M = A->M;
    int64_t v = 0;
    switch (what) {
      case H2MG_Q_N: v = M.n; break;
      case H2MG_Q_DIM: v = M.dim; break;
      case H2MG_Q_L: v = M.L; break;
      case H2MG_Q_TSTAR: v = M.tstar; break;
      case H2MG_Q_LEVELS: v = M.lev; break;
      case H2MG_Q_KD: v = M.KD; break;
      case H2MG_Q_KC: v = M.KC; break;
      case H2MG_Q_RANK: v = M.k; break;
      case H2MG_Q_NEAR_PAIRS: v = M.nD; break;
      case H2MG_Q_FAR_PAIRS: {
        H2_REQUIRE(arg >= 0 && arg <= M.L, H2MG_ERR_INVALID_ARG, "level out of range");
        const HostCSR& F = M.far[arg];
        for (int t = 0; t + 1 < (int)F.rowptr.size(); ++t)
          for (int e = F.rowptr[t]; e < F.rowptr[t + 1]; ++e) v += F.col[e] > t;
        break;
      }
      case H2MG_Q_LEVEL_SIZE:
        H2_REQUIRE(arg >= 1 && arg <= M.lev, H2MG_ERR_INVALID_ARG, "level out of range");
        v = level_size(M, arg);
        break;
      case H2MG_Q_BYTES_PRIMARY: {
        v = M.poolD.bytes + M.poolS.bytes;
        for (auto& p : M.poolP) v += p.bytes;
        break;
      }
      case H2MG_Q_BYTES_F32: {
        v = M.poolD32.bytes + M.poolS32.bytes;
        for (auto& p : M.poolP32) v += p.bytes;
        break;
      }
      case H2MG_Q_APPLY_BYTES:
        H2_REQUIRE(arg >= 1 && arg <= M.lev, H2MG_ERR_INVALID_ARG, "level out of range");
        v = apply_bytes(M, arg);
        break;
      case H2MG_Q_DEVICE_BYTES:
        for (auto& d : M.owned) v += d.bytes;
        break;
      case H2MG_Q_PRODUCT_BYTES_F32: {
        H2_REQUIRE(arg >= 0 && arg < (int)M.opC.size(), H2MG_ERR_INVALID_ARG, "operator out of range");
        const SymOp& op = arg == 0 ? M.opD : M.opC[arg];
        v = op.bytes(4, 4);
        break;
      }
      case H2MG_Q_PANEL_ENTRIES:
        v = panel_entries(M);
        break;
      default:
        throw Error{H2MG_ERR_INVALID_ARG, "unknown query"};
    }
    *value = v;
    return H2MG_OK;
  });
}

h2mg_status h2mg_export(h2mg_matrix A, int what, int arg, void* buf, int64_t cap, int64_t* bytes) {
  return guard([&]() -> h2mg_status {
    H2_REQUIRE(A && bytes, H2MG_ERR_INVALID_ARG, "null pointer argument");
    Matrix& M = A->M;
    std::vector<char> out;
    auto put_ints = [&](const std::vector<int>& v) {
      out.resize(v.size() * sizeof(int));
      if (!v.empty()) memcpy(out.data(), v.data(), out.size());
    };
    switch (what) {
      case H2MG_X_PERM: {
        std::vector<int> v(M.n);
        H2_CUDA(cudaMemcpy(v.data(), M.d_perm, sizeof(int) * M.n, cudaMemcpyDeviceToHost));
        put_ints(v);
        break;
      }
      case H2MG_X_LEAF_OFFSETS:
        put_ints(M.offsets[M.L]);
        break;
      case H2MG_X_NEAR:
      case H2MG_X_FAR: {
        int ell = what == H2MG_X_NEAR ? M.L : arg;
        H2_REQUIRE(ell >= 0 && ell <= M.L, H2MG_ERR_INVALID_ARG, "level out of range");
        const HostCSR& C = what == H2MG_X_NEAR ? M.inadm[M.L] : M.far[ell];
        std::vector<int> v;
        for (int t = 0; t + 1 < (int)C.rowptr.size(); ++t)
          for (int e = C.rowptr[t]; e < C.rowptr[t + 1]; ++e)
            if (what == H2MG_X_NEAR ? C.col[e] >= t : C.col[e] > t) {
              v.push_back(t);
              v.push_back(C.col[e]);
            }
        put_ints(v);
        break;
      }
      case H2MG_X_RANKS: {
        H2_REQUIRE(M.tstar >= 0 && arg >= M.tstar && arg <= M.L, H2MG_ERR_INVALID_ARG, "level has no basis");
        std::vector<int> v(M.h_rank.begin() + M.slot0(arg), M.h_rank.begin() + M.slot0(arg) + (1 << arg));
        put_ints(v);
        break;
      }
      case H2MG_X_SKELETON: {
        H2_REQUIRE(M.basis == H2MG_BASIS_SKELETON && M.d_skel, H2MG_ERR_INVALID_ARG, "matrix has no skeletons");
        H2_REQUIRE(M.tstar >= 0 && arg >= M.tstar && arg <= M.L, H2MG_ERR_INVALID_ARG, "level has no basis");
        std::vector<int> v((size_t)64 << arg), perm(M.n);
        H2_CUDA(cudaMemcpy(v.data(), M.d_skel + (size_t)M.slot0(arg) * 64, sizeof(int) * v.size(),
                           cudaMemcpyDeviceToHost));
        H2_CUDA(cudaMemcpy(perm.data(), M.d_perm, sizeof(int) * M.n, cudaMemcpyDeviceToHost));
        for (auto& e : v)
          if (e >= 0) e = perm[e];
        put_ints(v);
        break;
      }
      case H2MG_X_BOXES: {
        H2_REQUIRE(arg >= 0 && arg <= M.L, H2MG_ERR_INVALID_ARG, "level out of range");
        size_t nb = sizeof(double) * 2 * M.dim * (1 << arg);
        out.resize(nb);
        H2_CUDA(cudaMemcpy(out.data(), M.d_box[arg], nb, cudaMemcpyDeviceToHost));
        break;
      }
      default:
        throw Error{H2MG_ERR_INVALID_ARG, "unknown export"};
    }
    *bytes = (int64_t)out.size();
    if (buf && cap >= (int64_t)out.size() && !out.empty()) memcpy(buf, out.data(), out.size());
    else if (buf && cap < (int64_t)out.size()) throw Error{H2MG_ERR_INVALID_ARG, "buffer too small"};
    return H2MG_OK;
  });
}

h2mg_status h2mg_apply_level(h2mg_matrix A, int level, int precision, const double* x, double* y,
                             void* stream) {
  return guard([&]() -> h2mg_status {
    H2_REQUIRE(A && x && y, H2MG_ERR_INVALID_ARG, "null pointer argument");
    Matrix& M = A->M;
    H2_REQUIRE(level >= 1 && level <= M.lev, H2MG_ERR_INVALID_ARG, "level out of range");
    H2_REQUIRE(precision == H2MG_PREC_F64 || (precision == H2MG_PREC_MIXED_F32 && M.with_f32) ||
                   (precision == H2MG_PREC_F64_DD && level == 1 && M.fmt == FMT_F64),
               H2MG_ERR_INVALID_ARG, "no FP32 copy, or double-double sums asked off level 1 / float64 storage");
    cudaStream_t s = (cudaStream_t)stream;
    int64_t n = level_size(M, level);
    DevView X(x, n, true, s), Y(y, n, false, s);
    if (precision == H2MG_PREC_F64_DD)
      apply_level1_dd(M, X.d, Y.d, s);
    else
      apply_level(M, level, precision == H2MG_PREC_MIXED_F32, X.d, Y.d, s);
    Y.copy_out(y, n, s);
    return H2MG_OK;
  });
}

h2mg_status h2mg_coarse_solve(h2mg_matrix A, const double* r, double* e, void* stream) {
  return guard([&]() -> h2mg_status {
    H2_REQUIRE(A && r && e, H2MG_ERR_INVALID_ARG, "null pointer argument");
    Matrix& M = A->M;
    H2_REQUIRE(!M.apply_only, H2MG_ERR_INVALID_ARG, "matrix was built for products only");
    if (!M.coarse_ok) throw Error{H2MG_ERR_NOT_SPD, "the coarsest operator is not positive definite"};
    cudaStream_t s = (cudaStream_t)stream;
    int64_t n = level_size(M, M.lev);
    DevView R(r, n, true, s), E(e, n, false, s);
    coarse_solve(M, R.d, E.d, s);
    E.copy_out(e, n, s);
    return H2MG_OK;
  });
}

h2mg_status h2mg_smooth(h2mg_matrix A, int level, int precision, const double* f, const double* x0, int n,
                        double* x, double* r, void* stream) {
  return guard([&]() -> h2mg_status {
    H2_REQUIRE(A && f && x && n >= 0, H2MG_ERR_INVALID_ARG, "bad argument");
    Matrix& M = A->M;
    H2_REQUIRE(level >= 1 && level <= M.lev, H2MG_ERR_INVALID_ARG, "level out of range");
    H2_REQUIRE(precision == H2MG_PREC_F64 || (precision == H2MG_PREC_MIXED_F32 && M.with_f32),
               H2MG_ERR_INVALID_ARG, "no FP32 copy");
    cudaStream_t s = (cudaStream_t)stream;
    int64_t N = level_size(M, level);
    DevView F(f, N, true, s), X(x, N, false, s);
    DevView X0(x0 ? x0 : f, x0 ? N : 0, x0 != nullptr, s);
    DevView R(r ? r : x, N, false, s);
    smooth(M, level, precision == H2MG_PREC_MIXED_F32, F.d, x0 ? X0.d : nullptr, n, X.d, r ? R.d : nullptr, s);
    X.copy_out(x, N, s);
    if (r) R.copy_out(r, N, s);
    H2_CUDA(cudaStreamSynchronize(s));
    return H2MG_OK;
  });
}

h2mg_status h2mg_vcycle(h2mg_matrix A, const double* x0, const double* r1, double* x_out,
                        const h2mg_solve_opts* o, void* stream) {
  return guard([&]() -> h2mg_status {
    H2_REQUIRE(A && x0 && r1 && x_out && o, H2MG_ERR_INVALID_ARG, "null pointer argument");
    H2_REQUIRE(o->cycle >= H2MG_CYCLE_V && o->cycle <= H2MG_CYCLE_F, H2MG_ERR_INVALID_ARG, "unknown cycle type");
    Matrix& M = A->M;
    H2_REQUIRE(!M.apply_only, H2MG_ERR_INVALID_ARG, "matrix was built for products only");
    if (!M.coarse_ok) throw Error{H2MG_ERR_NOT_SPD, "the coarsest operator is not positive definite"};
    cudaStream_t s = (cudaStream_t)stream;
    DevView X0(x0, M.n, true, s), R(r1, M.n, true, s), X(x_out, M.n, false, s);
    vcycle(M, *o, X0.d, R.d, X.d, s);
    X.copy_out(x_out, M.n, s);
    H2_CUDA(cudaStreamSynchronize(s));
    return H2MG_OK;
  });
}

int64_t h2mg_launch_count(void) { return g_launches.load(); }

h2mg_status h2mg_transfer(h2mg_matrix A, int level, int direction, const double* v, double* out, void* stream) {
  return guard([&]() -> h2mg_status {
    H2_REQUIRE(A && v && out, H2MG_ERR_INVALID_ARG, "null pointer argument");
    Matrix& M = A->M;
    H2_REQUIRE(level >= 1 && level < M.lev, H2MG_ERR_INVALID_ARG, "level must be in [1, l-1]");
    H2_REQUIRE(direction == 0 || direction == 1, H2MG_ERR_INVALID_ARG, "direction must be 0 or 1");
    cudaStream_t s = (cudaStream_t)stream;
    int64_t nf = level_size(M, level), nc = level_size(M, level + 1);
    if (direction == 0) {
      DevView V(v, nf, true, s), O(out, nc, false, s);
      restrict_level(M, level, V.d, O.d, s);
      O.copy_out(out, nc, s);
    } else {
      DevView V(v, nc, true, s), O(out, nf, false, s);
      H2_CUDA(cudaMemsetAsync(O.d, 0, sizeof(double) * nf, s));
      prolong_add(M, level, V.d, O.d, s);
      O.copy_out(out, nf, s);
    }
    return H2MG_OK;
  });
}

h2mg_status h2mg_profile(h2mg_matrix A, int enable, int64_t* launches, double* ms, double* bytes) {
  return guard([&]() -> h2mg_status {
    H2_REQUIRE(A, H2MG_ERR_INVALID_ARG, "null handle");
    Profile& P = A->M.prof;
    if (enable == 1) {
      P.used = 0;
      P.bytes.clear();
      P.g_ms = P.g_bytes = 0.0;
      P.g_launches = 0;
    }
    double t = P.g_ms, by = P.g_bytes;
    for (size_t i = 0; i < P.used; ++i) {
      H2_CUDA(cudaEventSynchronize(P.ev[2 * i + 1]));
      float f = 0.f;
      H2_CUDA(cudaEventElapsedTime(&f, P.ev[2 * i], P.ev[2 * i + 1]));
      t += f;
      by += P.bytes[i];
    }
    P.on = (enable != 0);
    P.f32_only = (enable == 2);
    if (launches) *launches = (int64_t)P.used + P.g_launches;
    if (ms) *ms = t;
    if (bytes) *bytes = by;
    return H2MG_OK;
  });
}

h2mg_status h2mg_autotune(h2mg_matrix A, void* stream, double* report, int cap, int* count) {
  return guard([&]() -> h2mg_status {
    H2_REQUIRE(A && cap >= 0 && (report || cap == 0), H2MG_ERR_INVALID_ARG, "bad argument");
    Matrix& M = A->M;
    const int n = autotune_products(M, (cudaStream_t)stream, report, cap);
    if (count) *count = n;
    return H2MG_OK;
  });
}

h2mg_status h2mg_build_sibling(h2mg_matrix A, const h2mg_kernel* k, void* stream, h2mg_matrix* out) {
  if (out) *out = nullptr;
  return guard([&]() -> h2mg_status {
    H2_REQUIRE(A && k && out, H2MG_ERR_INVALID_ARG, "null pointer argument");
    H2_REQUIRE(k->kind >= 0 && k->kind <= H2MG_K_DMATERN32_DL && k->kind != H2MG_K_LAPLACE_SL,
               H2MG_ERR_INVALID_ARG, "unsupported kernel for a sibling");
    H2_REQUIRE(!k->weights && !k->diag, H2MG_ERR_INVALID_ARG, "siblings take no weights or diagonal");
    H2_REQUIRE(k->kind == H2MG_K_POLY || (k->length > 0 && std::isfinite(k->length)), H2MG_ERR_INVALID_ARG,
               "length must be > 0");
    H2_REQUIRE(!A->M.has_weights && !A->M.has_diag, H2MG_ERR_INVALID_ARG,
               "the base matrix has weights or a diagonal override");
    auto* h = new h2mg_matrix_s();
    h->M.stream = (cudaStream_t)stream;
    h->M.kp = KernelParams{k->kind, k->length, k->nugget, k->degree};
    try {
      build_sibling(h->M, A->M, k);
    } catch (...) {
      delete h;
      throw;
    }
    *out = h;
    return H2MG_OK;
  });
}

__global__ void k_fill(double* __restrict__ v, int64_t n, double a) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) v[i] = a;
}

h2mg_status h2mg_matern_loss_grad(h2mg_matrix K, h2mg_matrix dK, const double* y, const double* b,
                                  const h2mg_solve_opts* o, double* loss, double* dLdy, double* dLdb, double* dLdl,
                                  double* dLds, h2mg_solve_info* info, void* stream) {
  return guard([&]() -> h2mg_status {
    H2_REQUIRE(K && y && b && o && loss, H2MG_ERR_INVALID_ARG, "null pointer argument");
    Matrix& M = K->M;
    H2_REQUIRE(M.kp.kind == H2MG_K_MATERN32 && !M.apply_only, H2MG_ERR_INVALID_ARG,
               "K must be a Matern-3/2 matrix built for solves");
    H2_REQUIRE(!M.has_weights && !M.has_diag, H2MG_ERR_INVALID_ARG, "K must have no weights or diagonal override");
    const bool want_l = dLdl != nullptr;
    H2_REQUIRE(!want_l || dK, H2MG_ERR_INVALID_ARG, "dL/dl needs the derivative matrix dK");
    if (dK) {
      const Matrix& D = dK->M;
      H2_REQUIRE(D.apply_only && D.kp.kind == H2MG_K_DMATERN32_DL && D.d_perm == M.d_perm &&
                     D.kp.length == M.kp.length,
                 H2MG_ERR_INVALID_ARG, "dK must be the d/dlength sibling of K (same length)");
    }
    H2_REQUIRE(o->outer >= H2MG_OUTER_VCYCLE && o->outer <= H2MG_OUTER_CG && o->cycle >= H2MG_CYCLE_V &&
                   o->cycle <= H2MG_CYCLE_F && o->max_cycles >= 0 && o->tol >= 0,
               H2MG_ERR_INVALID_ARG, "bad solve options");
    H2_REQUIRE(o->precision == H2MG_PREC_F64 || (o->precision == H2MG_PREC_MIXED_F32 && M.with_f32),
               H2MG_ERR_INVALID_ARG, "mixed precision needs a matrix built with_f32");
    if (!M.coarse_ok) throw Error{H2MG_ERR_NOT_SPD, "the coarsest operator is not positive definite"};
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = M.n;
    const bool want_w = dLdb || dLdl || dLds;
    const int nr = want_w ? 3 : 2;
    // columns [y, b, 1] and their solutions [a, x, w], packed column-major
    struct Tmp {
      void* p = nullptr;
      ~Tmp() {
        if (p) best_effort(cudaFree(p), "cudaFree (loss)");
      }
    } tb, ts, tq;
    H2_CUDA(cudaMalloc(&tb.p, sizeof(double) * n * nr));
    H2_CUDA(cudaMalloc(&ts.p, sizeof(double) * n * nr));
    H2_CUDA(cudaMalloc(&tq.p, sizeof(double) * n * 2));
    double* B = (double*)tb.p;
    double* X = (double*)ts.p;
    double* Q = (double*)tq.p;
    H2_CUDA(cudaMemcpyAsync(B, y, sizeof(double) * n, cudaMemcpyDefault, s));
    H2_CUDA(cudaMemcpyAsync(B + n, b, sizeof(double) * n, cudaMemcpyDefault, s));
    if (want_w) {
      { k_fill<<<ceil_div(n, 256), 256, 0, s>>>(B + 2 * n, n, 1.0); ::h2mg::count_launch(); }
      H2_LAUNCH_CHECK();
    }
    H2_CUDA(cudaMemsetAsync(X, 0, sizeof(double) * n * nr, s));
    h2mg_solve_info inf[NRMAX];
    const h2mg_status st = solve_multi(M, B, X, nr, *o, inf, s);     // a, x (and w) to tol
    if (info)
      for (int c = 0; c < nr; ++c) info[c] = inf[c];
    if (st != H2MG_OK) {
      set_error(h2mg_error_string(st));
      return st;
    }
    const double* a = X;
    const double* x = X + n;
    const double* w = X + 2 * n;
    double ya, ox;
    dots(M, B, a, n, 1, &ya, s);                                      // y^T a
    dots(M, B + 2 * n, x, n, 1, &ox, s);                              // 1^T x (the ones column)
    if (!want_w) {
      // 1^T x without the ones column: x against a ones vector written into Q
      { k_fill<<<ceil_div(n, 256), 256, 0, s>>>(Q, n, 1.0); ::h2mg::count_launch(); }
      H2_LAUNCH_CHECK();
      dots(M, Q, x, n, 1, &ox, s);
    }
    *loss = 0.5 * ya + ox;                                            // L = 1/2 y^T K^-1 y + 1^T K^-1 b
    if (dLdy) H2_CUDA(cudaMemcpyAsync(dLdy, a, sizeof(double) * n, cudaMemcpyDefault, s));   // dL/dy = a
    if (dLdb) H2_CUDA(cudaMemcpyAsync(dLdb, w, sizeof(double) * n, cudaMemcpyDefault, s));   // dL/db = w
    if (dLds) {                                                       // dK/ds = I
      double aa, wx;
      dots(M, a, a, n, 1, &aa, s);
      dots(M, w, x, n, 1, &wx, s);
      *dLds = -0.5 * aa - wx;
    }
    if (want_l) {                                                     // dK/dl: the sibling's product
      apply_level_multi(dK->M, 1, false, X, n, Q, n, 2, s);           // [dK a, dK x]
      double adka, wdkx;
      dots(M, a, Q, n, 1, &adka, s);
      dots(M, w, Q + n, n, 1, &wdkx, s);
      *dLdl = -0.5 * adka - wdkx;
    }
    H2_CUDA(cudaStreamSynchronize(s));
    return H2MG_OK;
  });
}

h2mg_status h2mg_dot(const double* x, const double* y, int64_t n, double* out, void* stream) {
  return guard([&]() -> h2mg_status {
    H2_REQUIRE(x && y && out && n >= 0, H2MG_ERR_INVALID_ARG, "bad argument");
    cudaStream_t s = (cudaStream_t)stream;
    DevView X(x, n, true, s), Y(y, n, true, s);
    *out = device_dot(X.d, Y.d, n, s);
    return H2MG_OK;
  });
}

}  // extern "C"
