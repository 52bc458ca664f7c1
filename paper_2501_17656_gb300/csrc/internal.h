// internal.h -- handle layout and internal entry points of the H2-MG library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "common.cuh"

namespace h2mg {

// Device allocation owned by a handle; freed by the handle's destructor.
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

// A symmetric block-sparse operator over one index space of "slots" (clusters),
// stored as its upper triangle: row t holds entries (t, s) with s >= t. Each
// entry points at a K x K block in some pool (swizzled layout, see swz). The
// transposed product of entry (t, s), s > t, is added into output row s.
struct SymOp {
  int K = 0;
  int nrows = 0;          // slots
  int nnz = 0;            // stored entries
  int* rowptr = nullptr;  // [nrows + 1]
  int* col = nullptr;     // [nnz]
  const void** blk = nullptr;      // [nnz] block pointers into the primary pool
  const void** blk32 = nullptr;    // [nnz] block pointers into the FP32 pool (or null)
  int64_t noff = 0;       // off-diagonal entries (each adds K transposed partials)
  // CTAs per block row chosen by the autotuner, per element format (F64, DF, F32) and
  // column group size (NR = 1, 2, 4); 0 = the fixed heuristic
  int split[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
  int64_t bytes(int eb, int vb) const {   // algorithmic bytes of one product
    return (int64_t)nnz * K * K * eb + (int64_t)nrows * K * vb * 2 + noff * K * vb;
  }
};
inline int nr_index(int nr) { return nr >= 4 ? 2 : nr - 1; }
// Fixed heuristic of the block product: enough CTAs to fill the GPU when the operator
// has few block rows (at most 16 CTAs per row).
inline int split_heuristic(int nrows) {
  const int v = (2048 + nrows - 1) / (nrows > 0 ? nrows : 1);
  return v < 1 ? 1 : (v > 16 ? 16 : v);
}

// CUDA events around the launches of the block product (h2mg_profile).
struct Profile {
  bool on = false;
  bool f32_only = false;         // record only the products of the FP32 copy
  std::vector<cudaEvent_t> ev;   // pairs (start, stop)
  size_t used = 0;               // pairs in use
  std::vector<double> bytes;
  // while a V-cycle graph is captured with profiling on: the graph's own event pairs,
  // recorded as nodes of the graph, taken in order (cap_next pairs used so far)
  std::vector<cudaEvent_t>* cap_ev = nullptr;
  std::vector<double>* cap_bytes = nullptr;
  size_t cap_next = 0;
  // block products run inside graph replays, added once each replay has finished
  double g_ms = 0.0, g_bytes = 0.0;
  int64_t g_launches = 0;
};

struct GraphSet;   // captured V-cycles of a matrix (solve.cu)
struct PanelPlan;  // block lists and panels of the tensor-core product (panel.cu)

// Host-side copy of a full (both triangles) CSR list of cluster pairs.
struct HostCSR {
  std::vector<int> rowptr, col;
  int nnz() const { return rowptr.empty() ? 0 : rowptr.back(); }
};

struct Matrix {
  // ---- problem
  int64_t n = 0;
  int dim = 0;
  KernelParams kp{};
  bool has_weights = false, has_diag = false;
  int leaf = 0, q = 0, k = 0;   // k: Chebyshev nodes q^dim, or the rank cap of skeleton bases
  double eta = 0;
  int basis = H2MG_BASIS_CHEBYSHEV;
  double basis_tol = 0.0;       // relative tolerance of skeleton bases
  int fmt = FMT_F64;      // primary block format (FMT_F64 or FMT_DF)
  bool with_f32 = false;
  bool apply_only = false;
  cudaStream_t stream = nullptr;

  // ---- tree (tree order = leaf-major, padded to KD slots per leaf)
  int L = 0;              // leaf depth
  int KD = 0, KC = 0;     // padded leaf size and padded rank
  int tstar = -1;         // first level with a far pair (-1: none)
  int lev_nat = 1, lev = 1;  // natural and chosen coarsest multigrid level l
  std::vector<std::vector<int>> offsets;  // per level, cluster offsets in compact tree order
  int* d_perm = nullptr;       // [n] original index of compact tree position
  int* d_slot_of = nullptr;    // [n] padded slot of each original index
  int* d_leafoff = nullptr;    // [2^L + 1] compact offsets of the leaves
  double* d_X = nullptr;       // [n * dim] points in compact tree order
  double* d_sw = nullptr;      // [n] sqrt(w) in compact tree order
  double* d_dg = nullptr;      // [n] diagonal entries A_ii in compact tree order
  std::vector<double*> d_box;  // per level, [2^ell * 2 * dim] (lo, hi)
  double* d_nodes = nullptr;   // coupling points of clusters at levels tstar..L (heap slots):
                               // Chebyshev nodes (k per slot) or skeleton points (KC per slot)
  double* d_nsw = nullptr;     // skeleton bases: sqrt(w) of each slot's skeleton points (KC per slot)
  int* d_skel = nullptr;       // skeleton bases: tree positions of each slot's skeleton (64 per slot)
  DevBuf tid;                  // skeleton bases, during the build: interpolation matrices
  int* d_rank = nullptr;       // ranks per slot (levels tstar..L)
  std::vector<int> h_rank;     // host copy

  // ---- partition (host copies, full lists per level)
  std::vector<HostCSR> far, inadm;

  // ---- bases (float64, natural column-major, padded)
  double* d_U = nullptr;       // [2^L][KD x KC]
  double* d_E = nullptr;       // per slot at levels tstar+1..L: [KC x KC] (child -> parent transfer)
  double* d_R = nullptr;       // per slot at levels tstar..L: [KC x KC] (rows >= rank are zero)
  float* d_U32 = nullptr;
  float* d_E32 = nullptr;
  double* d_UT = nullptr;      // transposes (KC x KD per leaf, KC x KC per slot)
  double* d_ET = nullptr;
  float* d_UT32 = nullptr;
  float* d_ET32 = nullptr;

  // ---- block pools (primary format and optional FP32 copy)
  DevBuf poolD, poolS, poolD32, poolS32;
  DevBuf poolE, poolE32;                      // swizzled transfers, one per slot (levels > t*)
                                              // (a sibling matrix shares its base's poolE)
  std::vector<DevBuf> poolP, poolP32;         // index = multigrid level i (2..lev)
  int64_t nD = 0, nS = 0;                     // stored blocks
  std::vector<int64_t> nP;
  std::vector<int64_t> s_level_base;          // first S block of each level (index ell)

  // ---- operators
  SymOp opD;                    // level 1 close part (KD, point slots = leaves)
  std::vector<SymOp> opC;       // index i: coupling (+ P_i) operator of multigrid level i
  int slot0(int ell) const { return (1 << ell) - (1 << tstar); }   // first coef slot of level ell
  int nslots() const { return tstar < 0 ? 0 : (1 << (L + 1)) - (1 << tstar); }

  // ---- dense coarsest operator and Cholesky factor
  int nl = 0;                   // size of A_l
  double* d_Al = nullptr;       // [nl * nl] column-major; lower triangle holds the factor
  double* d_Ainv = nullptr;     // [nl * nl] A_l^{-1} formed from the factor
  bool coarse_ok = false;

  // ---- workspaces
  DevBuf wx, wyrow, wyc;        // coefficient buffers (nslots * KC elements, 8 B)
  DevBuf wxp, wyp;              // point buffers (2^L * KD elements, 8 B)
  DevBuf wstage;                // host staging
  DevBuf wvec;                  // multigrid vectors (float64)
  DevBuf wred;                  // reduction partials + scalars
  DevBuf wcoarse;               // three vectors of the coarse size (triangular solves)
  DevBuf wfcg;                  // five point vectors of the flexible-CG outer loop
  int* d_flag = nullptr;        // device error flags

  Profile prof;
  GraphSet* graphs = nullptr;   // captured V-cycle graphs, by solve settings
  PanelPlan* panel = nullptr;   // tensor-core product plan, built on first use
  cudaStream_t cap_stream = nullptr;
  std::vector<DevBuf> owned;    // everything else
  ~Matrix();
  void* alloc(size_t bytes);    // owned allocation, zero-initialised
  void free_owned(void* p);     // release an owned allocation before the handle goes
};

// ---- tree.cu
void build_tree(Matrix& M, const double* d_points_user);
void build_partition(Matrix& M);
// ---- skeleton.cu
void build_skeletons(Matrix& M);
// ---- fill.cu
void build_bases(Matrix& M);
void build_blocks(Matrix& M, const Matrix* base);
void build_coarse_near(Matrix& M);
void build_f32_copies(Matrix& M);
// ---- dense.cu
void build_dense_coarse(Matrix& M);
void coarse_solve(Matrix& M, const double* r, double* e, cudaStream_t s);
void coarse_solve_multi(Matrix& M, const double* r, double* e, int nr, cudaStream_t s);
// ---- apply.cu
struct ApplyWork {                // workspace of one product (see apply_impl)
  void *xc, *yr, *yc, *xp, *yp;
};
void setup_operators(Matrix& M);
void apply_level1_ws(Matrix& M, const double* x, double* y, cudaStream_t s, const ApplyWork& ws);
void apply_level1_ws_sizes(const Matrix& M, size_t* coef, size_t* pts);
void apply_level1_dd(Matrix& M, const double* x, double* y, cudaStream_t s);
void apply_level(Matrix& M, int i, bool f32, const double* x, double* y, cudaStream_t s);
// Right-hand sides that one product, smoother, V-cycle or solve handles together.
constexpr int NRMAX = 4;
void apply_level_multi(Matrix& M, int i, bool f32, const double* x, int64_t ldx, double* y, int64_t ldy, int nr,
                       cudaStream_t s);
int64_t apply_bytes(const Matrix& M, int i);
// Autotuner of the block product: per operator, format and column group, the row
// split of the fastest timed trial. out (cap entries of 4 doubles) receives
// (operator index, nr, fixed-heuristic ms, tuned ms) per tuned combination.
int autotune_products(Matrix& M, cudaStream_t s, double* out, int cap);
// ---- panel.cu
// Y = A X at level 1 for nr columns on the tensor cores (split-TF32 products of the FP32
// blocks, 128 columns per pass); synchronises s.
void apply_panel(Matrix& M, const double* x, int64_t ldx, double* y, int64_t ldy, int nr, cudaStream_t s);
bool panel_supported(const Matrix& M);
int64_t panel_entries(const Matrix& M);   // block products of one pass (0: no plan yet)
void destroy_panel_plan(Matrix& M);
// ---- solve.cu
void smooth(Matrix& M, int i, bool f32, const double* f, const double* x0, int n, double* x,
            double* r, cudaStream_t s);
void restrict_level(Matrix& M, int i, const double* v, double* out, cudaStream_t s);
void prolong_add(Matrix& M, int i, const double* e, double* out, cudaStream_t s);
void vcycle(Matrix& M, const h2mg_solve_opts& o, const double* x0, const double* r1, double* xout,
            cudaStream_t s);
h2mg_status solve(Matrix& M, const double* b, double* x, const h2mg_solve_opts& o,
                  h2mg_solve_info* info, cudaStream_t s);
void alloc_solve_workspace(Matrix& M);
void destroy_graphs(Matrix& M);
// nr <= NRMAX columns, column-major with leading dimension N_i (n for the solve)
void smooth_multi(Matrix& M, int i, bool f32, const double* f, const double* x0, int n, double* x, double* r,
                  int nr, cudaStream_t s);
void vcycle_multi(Matrix& M, const h2mg_solve_opts& o, const double* x0, const double* r1, double* xout, int nr,
                  cudaStream_t s);
h2mg_status solve_multi(Matrix& M, const double* b, double* x, int nr, const h2mg_solve_opts& o,
                        h2mg_solve_info* info, cudaStream_t s);
h2mg_status solve_batched(const std::vector<Matrix*>& Ms, const double* const* b, double* const* x,
                          const h2mg_solve_opts& o, h2mg_solve_info* info, cudaStream_t s);
int64_t level_size(const Matrix& M, int i);
// out[c] = a_c^T b_c for nr columns of length n (leading dimension n), reduced on the
// device; the nr results are read back (synchronises s).
void dots(Matrix& M, const double* a, const double* b, int64_t n, int nr, double* out, cudaStream_t s);
double device_dot(const double* a, const double* b, int64_t n, cudaStream_t s);

// ---- sort.cu (device primitives)
void exclusive_scan_i32(const int* in, int* out, int n, cudaStream_t s, Matrix& M);
void radix_sort_u64(uint64_t* keys, int* vals, int n, int bits, Matrix& M, cudaStream_t s);

bool is_device_pointer(const void* p);

}  // namespace h2mg

// The opaque handle behind h2mg_matrix.
struct h2mg_matrix_s {
  h2mg::Matrix M;
};
