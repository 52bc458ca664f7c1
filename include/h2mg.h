/* h2mg.h -- C ABI of the GB300 H2-MG library (libh2mg.so).
 *
 * H2-MG (Sushnikova, Turkiyyah, Chow, Keyes, "H2-MG: A multigrid method for
 * hierarchical rank structured matrices") solves A x = b for a dense symmetric
 * positive definite kernel matrix A held in H2 form,
 *     A = D + U_1 (D_2 + U_2 ( ... (D_l + U_l S_l V_l) ... ) V_2) V_1      (Sec. 3.1, eq. h2)
 * with a multigrid V-cycle whose coarse spaces are the nested cluster bases
 * (Sec. 3.3, Algorithm 1). This header declares the three operations of the
 * paper's problem statement -- build the H2 matrix from points, a kernel, a leaf
 * size, a rank and an admissibility parameter; apply it; solve with H2-MG to a
 * relative-residual tolerance -- plus introspection calls used by tests.
 *
 * Conventions (all calls):
 *  - Pointer arguments for points, vectors, weights and diagonals may be host or
 *    device memory; the library detects which (cudaPointerGetAttributes) and
 *    stages host data through its own device buffers. Device pointers must be on
 *    the current device.
 *  - Vectors are float64, in the user's point order (the library owns the tree
 *    permutation). Several right-hand sides are column-major with leading
 *    dimension ld >= n.
 *  - Work is enqueued on `stream` (a cudaStream_t, NULL = legacy default stream).
 *    h2mg_build and h2mg_solve synchronise the stream to read sizes/residuals;
 *    h2mg_apply returns without synchronising when x and y are device pointers.
 *  - The caller owns every buffer it passes. The handle owns all device memory it
 *    allocates; h2mg_destroy frees it.
 *  - No exception crosses the ABI. Every call returns an h2mg_status; on failure
 *    h2mg_last_error() returns a message for the calling thread.
 */
#ifndef H2MG_H
#define H2MG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct h2mg_matrix_s* h2mg_matrix;   /* opaque, library-owned */

typedef enum {
    H2MG_OK = 0,
    H2MG_ERR_INVALID_ARG = 1,    /* bad pointer, size, option; nothing was launched   */
    H2MG_ERR_OOM = 2,            /* device memory exhausted (or above the set budget)  */
    H2MG_ERR_CUDA = 3,           /* a CUDA runtime call failed                          */
    H2MG_ERR_NOT_SPD = 4,        /* Cholesky of the coarse operator met a pivot <= 0    */
    H2MG_ERR_NOT_CONVERGED = 5,  /* max_cycles reached above tol (info is filled)      */
    H2MG_ERR_NAN = 6,            /* a NaN/Inf appeared in the input or the residual     */
    H2MG_ERR_TIMEOUT = 7,        /* a bounded device-side wait gave up                  */
    H2MG_ERR_UNSUPPORTED = 8     /* valid request outside what the library implements   */
} h2mg_status;

/* Kernel functions k(x, y), r = |x - y| (Sec. 4: eqs. a_gau, a_exp; Sec. 4.3). */
typedef enum {
    H2MG_K_GAUSSIAN = 0,      /* exp(-r^2 / length^2)     (Sec. 4.1 with sigma = length^2) */
    H2MG_K_EXPONENTIAL = 1,   /* exp(-r / length)          (Sec. 4.2 with sigma = length)   */
    H2MG_K_MATERN32 = 2,      /* (1 + sqrt3 r/length) exp(-sqrt3 r/length)                 */
    H2MG_K_LAPLACE_SL = 3,    /* 1 / (4 pi r)  single-layer potential (Sec. 4.3); needs weights
                                 (panel areas a_i) or diag                                  */
    H2MG_K_POLY = 4,          /* (1 + x.y)^degree  (test kernel: exact in H2 if degree < q)  */
    H2MG_K_DMATERN32_DL = 5   /* d/dlength of the Matern-3/2 kernel: (3 r^2/l^3) exp(-sqrt3 r/l) */
} h2mg_kernel_kind;

/* A_ij = sqrt(w_i) k(x_i, x_j) sqrt(w_j) for i != j;
 * A_ii = (diag ? diag[i] : w_i k(x_i, x_i)) + nugget       (eqs. a_gau/a_exp: 1 + c).
 * LAPLACE_SL without diag: A_ii = sqrt(w_i / pi) / 2, the potential at the centre of a
 * flat disk of area w_i carrying unit density (the panel's self-interaction, Sec. 4.3,
 * in the symmetric scaling of the off-diagonal entries). */
typedef struct {
    int kind;                 /* h2mg_kernel_kind */
    double length;            /* length scale, > 0 (ignored by POLY and LAPLACE_SL) */
    double nugget;            /* added to every diagonal entry */
    int degree;               /* POLY only, 0..16 */
    const double* weights;    /* optional, n entries, user order, > 0 (host or device) */
    const double* diag;       /* optional, n entries, user order (host or device) */
} h2mg_kernel;

/* Block storage format of the primary copy of D, the couplings S and the coarse
 * near fields P_i. F64 = IEEE double, products on the FP64 pipe. DF64 = each
 * entry stored as a pair of floats (hi, lo), hi + lo = the double to ~2^-48
 * relative, products in double-float arithmetic on the FP32 pipes (same bytes). */
typedef enum { H2MG_STORE_F64 = 0, H2MG_STORE_DF64 = 1 } h2mg_storage;

/* How the nested cluster bases are made before their QR orthonormalisation (Sec. 3.3).
 * CHEBYSHEV: tensor interpolation with cheb_q first-kind nodes per axis on each
 *   cluster's tight box (rank q^dim).
 * SKELETON: recursive skeletonization to a relative tolerance, the kind of
 *   tolerance-driven algebraic construction the paper builds its matrices with
 *   (Sec. 4.1: relative accuracy 1e-9, adaptive ranks): each cluster keeps the
 *   subset of its points (a leaf) or of its children's skeletons (a parent) whose
 *   rows interpolate its sampled far-field rows, A(X_t, F_t) ~= T_t A(skel_t, F_t),
 *   chosen by a column-pivoted QR stopped at basis_tol relative to the first pivot or
 *   at rank_max. The sample F_t is every far partner's candidates plus every far
 *   partner of the parent (their children's candidates, thinned to 128 points).
 *   Leaf basis = T_leaf, transfers = rows of T_parent, couplings A(skel_t, skel_s). */
typedef enum { H2MG_BASIS_CHEBYSHEV = 0, H2MG_BASIS_SKELETON = 1 } h2mg_basis;

typedef struct {
    int leaf_size;      /* max points per leaf cluster, 2..64 */
    int cheb_q;         /* Chebyshev nodes per dimension; rank k = q^dim <= 64 (CHEBYSHEV) */
    double eta;         /* admissibility: far iff dist > 0 and max(diam) <= eta*dist; >= 0 */
    int storage;        /* h2mg_storage of the primary copy */
    int with_f32;       /* 1: also keep an FP32 copy of every V-cycle operator (mixed solves) */
    int coarse_level;   /* coarsest multigrid level l; -1 = natural l = L - t* + 1 */
    int basis;          /* h2mg_basis */
    double basis_tol;   /* SKELETON: relative tolerance of the pivoted QR, >= 0 */
    int rank_max;       /* SKELETON: rank cap, 1..64 */
} h2mg_build_opts;

/* Arithmetic of the V-cycle products (h2mg_solve_opts.precision) and of
 * h2mg_apply_level. F64_DD (h2mg_apply_level at level 1 on float64 storage only): the
 * float64 blocks with double-double vectors and sums, the product the extended-precision
 * outer residual uses (h2mg_solve_opts.residual_dd). */
typedef enum { H2MG_PREC_F64 = 0, H2MG_PREC_MIXED_F32 = 1, H2MG_PREC_F64_DD = 2, H2MG_PREC_TF32X3 = 3 } h2mg_precision;
typedef enum { H2MG_OUTER_VCYCLE = 0, H2MG_OUTER_FCG = 1, H2MG_OUTER_CG = 2 } h2mg_outer;
/* Multigrid cycle of the outer loops. V: Algorithm 1 (Sec. 3.3). W and F, which the
 * paper names as further options after Algorithm 1: the textbook recursions, where
 * each visit of level i < l pre-smooths from its start (zero on the first visit),
 * restricts the residual, visits level i + 1 twice (W) or once as an F-cycle and once
 * as a V-cycle (F), each visit starting from the previous one's result, prolongs and
 * post-smooths; level l solves directly. */
typedef enum { H2MG_CYCLE_V = 0, H2MG_CYCLE_W = 1, H2MG_CYCLE_F = 2 } h2mg_cycle;

typedef struct {
    double tol;                     /* stop when |b - A x| / |b| <= tol */
    int max_cycles;                 /* cap on V-cycles (outer iterations), >= 0 */
    int n_f;                        /* CG iterations on the finest level (Remark rem:fine_coarse) */
    int n_c;                        /* CG iterations on the coarse levels 2..l-1 */
    int precision;                  /* h2mg_precision of the V-cycle */
    int explicit_restrict_residual; /* 1: r_{i+1} = U_i^T (r_i - A_i e_i) with an explicit apply;
                                       0: use CG's recurrence residual (equal in exact arithmetic) */
    int outer;                      /* h2mg_outer: repeated cycles (Sec. 3.3), flexible CG
                                       preconditioned by one cycle, or unpreconditioned CG
                                       (the paper's comparison solver, Sec. 4; each CG
                                       iteration counts as one "cycle" in the info, the
                                       multigrid settings are unused) */
    int use_graph;                  /* 1: capture the V-cycle (smoothers, transfers, coarse
                                       solve: no host synchronisation inside) as a CUDA graph
                                       on the first solve with these settings and column
                                       count, then replay it with one launch per outer
                                       iteration; the graph is kept with the matrix.
                                       While h2mg_profile is enabled a graph with event
                                       nodes around every block product is captured and
                                       replayed instead, and its timings are read after
                                       each replay */
    int skip_square_levels;         /* 1: no smoothing on a level i >= 2 whose restriction
                                       U_{i-1} is square (every leaf, or every cluster of
                                       level m(i), has as many basis columns as rows), so
                                       that A_i is an orthogonal similarity of A_{i-1} and
                                       not a coarser operator: the V-cycle passes the
                                       residual through it. 0: Algorithm 1 literally */
    int cycle;                      /* h2mg_cycle */
    int residual_dd;                /* outer residual b - A x of repeated cycles and flexible CG.
                                       0: the float64 product. 1: the float64 blocks with
                                       double-double vectors and sums (float64 storage only;
                                       about ten times the FP64 work of that product). When
                                       |x| >> |b| (ill-conditioned systems) the float64 sum
                                       rounds at about eps |A| |x|, which can exceed tol |b|;
                                       the extended product removes that floor. 2 (automatic):
                                       float64 until a column's residual is within 100 tol,
                                       then extended for that column from that cycle on; a
                                       column whose float64 residual makes no new minimum for
                                       5 cycles is probed with one extended residual and
                                       switches if that is below 0.8 of the float64 one (the
                                       float64 value is mostly rounding) */
} h2mg_solve_opts;

typedef struct {
    int cycles;                /* V-cycles executed */
    int converged;             /* 1 if relres <= tol */
    double relres;             /* final |b - A x| / |b| (float64) */
    double relres_hist[256];   /* relres before each cycle (first 256) */
    double ms_solve;           /* wall time of the solve on the stream */
} h2mg_solve_info;

/* Build the H2 matrix of kernel `k` on `n` points of dimension `dim` (1..3),
 * row-major n x dim float64 (Sec. 3.1). Tree, block partition, Chebyshev bases,
 * QR orthonormalisation, couplings, coarse near fields P_i (Sec. 3.3, eq. a2_str)
 * and the Cholesky factor of the coarsest operator are all computed on the GPU.
 * Errors: INVALID_ARG (n < 1, dim not in 1..3, leaf/q/eta out of range, null
 * pointers, NaN coordinates), OOM, NOT_SPD (coarse Cholesky failed), CUDA.
 * On error *out is NULL and nothing is leaked. */
h2mg_status h2mg_build(const double* points, int64_t n, int dim, const h2mg_kernel* k,
                       const h2mg_build_opts* o, void* stream, h2mg_matrix* out);

/* y = A x (Sec. 3.1, the H2 matrix-vector product x_i = V_i x_{i-1},
 * y_{i-1} = D_i x_{i-1} + U_i y_i). nrhs >= 1 columns, leading dimension ld >= n.
 * x and y must not overlap. Uses the primary storage copy. Columns are taken in
 * groups of up to four: each stored block is read once per group (two columns at a
 * time go through one block product in float64 / double-float storage). */
h2mg_status h2mg_apply(h2mg_matrix A, const double* x, double* y, int nrhs, int64_t ld,
                       void* stream);

/* Y = A X (Sec. 3.1) in a chosen arithmetic, nrhs >= 1 columns, leading dimension
 * ld >= n, host or device buffers (not overlapping):
 *   H2MG_PREC_F64        the primary storage, as h2mg_apply;
 *   H2MG_PREC_MIXED_F32  the FP32 copy on the CUDA cores, four columns per block read;
 *   H2MG_PREC_TF32X3     the FP32 copy on the tensor cores (tcgen05), 128 columns per
 *                        block read: every step of the product -- U_l^T x_l and E_c^T x_c
 *                        upward, the near and coupling blocks, E_c y_p and U_l y_l
 *                        downward -- is a 64 x 64 block times a 64 x 128 panel. Each FP32
 *                        operand a is split into a TF32 head h = tf32(a) and tail
 *                        t = tf32(a - h), and a b is formed as h_a h_b + h_a t_b + t_a h_b
 *                        in FP32 (relative error of each product below 2^-20).
 *                        Needs leaf and rank blocks of 64 (KD = KC = 64). Each
 *                        off-diagonal stored block is read twice (once per triangle), so
 *                        that no output needs atomic sums. Synchronises the stream.
 * Errors: INVALID_ARG (unknown precision, no FP32 copy for MIXED_F32 / TF32X3),
 * UNSUPPORTED (TF32X3 with blocks other than 64), CUDA. */
h2mg_status h2mg_apply_ex(h2mg_matrix A, int precision, const double* x, double* y, int nrhs, int64_t ld,
                          void* stream);

/* Solve A x = b with H2-MG (Algorithm 1, repeated V-cycles, Sec. 3.3). On entry
 * x holds the initial guess x_0 (zeros are the paper's choice), on exit the
 * solution. nrhs >= 1 columns, leading dimension ld. Columns are solved in groups
 * of up to four that share every product, smoother step and V-cycle launch; each
 * column has its own CG scalars, outer-loop coefficients and stopping test (a
 * column that has converged keeps its x while the rest of its group runs on).
 * info (optional) points to nrhs structs that receive each column's statistics
 * (relres_hist and ms_solve are those of the column's group). Returns NOT_CONVERGED
 * (with x and info filled) if max_cycles is reached for some column, NAN if b or a
 * residual is not finite. */
h2mg_status h2mg_solve(h2mg_matrix A, const double* b, double* x, int nrhs, int64_t ld,
                       const h2mg_solve_opts* o, h2mg_solve_info* info, void* stream);

/* Solve nprob independent problems A[p] x[p] = b[p] (one column each, each matrix
 * built separately with its own size, kernel and tree; no matrix twice) with H2-MG,
 * together: every outer iteration computes all residuals and reads all their norms
 * with one synchronisation, runs the V-cycles of all unconverged problems and then
 * the outer updates. With o->use_graph the V-cycles are one launch of a CUDA graph
 * with one branch per problem (each problem's captured V-cycle), so the kernels of
 * small problems run concurrently. b[p], x[p]: n_p entries, host or device; x[p]
 * holds the initial guess. info: nprob structs, one per problem. Same statuses as
 * h2mg_solve (NOT_CONVERGED if any problem did not converge). */
h2mg_status h2mg_solve_batched(int nprob, const h2mg_matrix* A, const double* const* b, double* const* x,
                               const h2mg_solve_opts* o, h2mg_solve_info* info, void* stream);

/* Build the H2 matrix of another kernel on the same points with the same cluster
 * tree and block partition as A (Sec. 3.1). With Chebyshev bases it also shares A's
 * nodes and orthonormalisation factors (only D and the couplings S = R k'(xi, xi) R^T
 * change); with H2MG_K_DMATERN32_DL (length = A's length, nugget 0) it is then
 * d A / d length of a Matern-3/2 H2 matrix exactly, since interpolation bases do not
 * depend on the kernel's parameters. Skeleton bases are chosen from A's kernel values
 * and do not span another kernel's far field: a sibling of a skeleton matrix
 * skeletonizes its own kernel (same tolerance and rank cap) on A's tree and
 * partition, and approximates d A / d length of the exact kernel to that tolerance.
 * The result supports products only (h2mg_apply, h2mg_apply_level at level 1);
 * h2mg_solve on it returns INVALID_ARG. It refers to A's device structures:
 * destroy it before A. Weights and diagonal overrides of k are not supported
 * (INVALID_ARG). */
h2mg_status h2mg_build_sibling(h2mg_matrix A, const h2mg_kernel* k, void* stream, h2mg_matrix* out);

/* The differentiation form on a Matern-3/2 matrix K = (1 + sqrt3 r/l) exp(-sqrt3 r/l) + s I
 * in H2 form: the loss L(y, b, l, s) = 1/2 y^T K^{-1} y + 1^T K^{-1} b and its adjoint
 * gradients. With a = K^{-1} y, x = K^{-1} b and w = K^{-1} 1 (K symmetric):
 *     L = 1/2 y^T a + 1^T x,   dL/dy = a,   dL/db = w,
 *     dL/dl = -1/2 a^T (dK/dl) a - w^T (dK/dl) x,   dL/ds = -1/2 a^T a - w^T x  (dK/ds = I).
 * The three solves run as one three-column H2-MG solve with the options o (two
 * columns when none of dLdb, dLdl, dLds is wanted); dK is the d/dlength sibling of K
 * (h2mg_build_sibling with H2MG_K_DMATERN32_DL and K's length), applied to a and x as
 * one two-column product; the inner products are reduced on the GPU and combined
 * here. Only the scalars leave the device; dLdy and dLdb (optional, n entries, host or
 * device) receive a and w. dK may be NULL when dLdl is NULL. info (optional) receives
 * the statistics of the two or three columns. Statuses as h2mg_solve; INVALID_ARG
 * when K is not a Matern-3/2 matrix built for solves or dK is not its sibling. The
 * problem statement is Sec. 3.1's A x = b with A depending on kernel parameters; the
 * loss and gradient formulas are the adjoint method's. Allocates its column buffers
 * (3 n doubles) and synchronises the stream. */
h2mg_status h2mg_matern_loss_grad(h2mg_matrix K, h2mg_matrix dK, const double* y, const double* b,
                                  const h2mg_solve_opts* o, double* loss, double* dLdy, double* dLdb,
                                  double* dLdl, double* dLds, h2mg_solve_info* info, void* stream);

/* *out = x^T y for n float64 values (host or device vectors), reduced on the GPU
 * with the library's deterministic two-pass sum; synchronises the stream. */
h2mg_status h2mg_dot(const double* x, const double* y, int64_t n, double* out, void* stream);

/* Free every device buffer of the handle. NULL is accepted. */
h2mg_status h2mg_destroy(h2mg_matrix A);

/* Static description of a status code. */
const char* h2mg_error_string(h2mg_status s);

/* Message of the last failed call on this thread ("" if none). */
const char* h2mg_last_error(void);

/* ---------------------------------------------------------------- introspection
 * Used by tests to compare the GPU structures with an independent implementation.
 * `what` selects an integer: */
typedef enum {
    H2MG_Q_N = 0, H2MG_Q_DIM = 1, H2MG_Q_L = 2, H2MG_Q_TSTAR = 3, H2MG_Q_LEVELS = 4,
    H2MG_Q_KD = 5, H2MG_Q_KC = 6, H2MG_Q_RANK = 7, H2MG_Q_NEAR_PAIRS = 8,
    H2MG_Q_FAR_PAIRS = 9, H2MG_Q_LEVEL_SIZE = 10, H2MG_Q_BYTES_PRIMARY = 11,
    H2MG_Q_BYTES_F32 = 12, H2MG_Q_APPLY_BYTES = 13, H2MG_Q_DEVICE_BYTES = 14,
    H2MG_Q_PRODUCT_BYTES_F32 = 15, H2MG_Q_PANEL_ENTRIES = 16
} h2mg_query_what;

/* *value = the quantity `what` (arg = tree level for FAR_PAIRS, multigrid level
 * for LEVEL_SIZE / APPLY_BYTES, operator index for PRODUCT_BYTES_F32, 0 otherwise).
 * APPLY_BYTES = algorithmic bytes (stored blocks read once plus vectors) of one A_i
 * apply in the primary format. PRODUCT_BYTES_F32 = algorithmic bytes of one launch of
 * the block-sparse product of operator arg (0: the close part of level 1; i >= 1:
 * the coupling operator of level i) on the FP32 copy, one column. PANEL_ENTRIES =
 * block-times-panel products of one 128-column pass of the tensor-core product
 * (h2mg_apply_ex, TF32X3), 0 before its first call. */
h2mg_status h2mg_query(h2mg_matrix A, int what, int arg, int64_t* value);

typedef enum {
    H2MG_X_PERM = 0,        /* int32[n]: original index of each tree position       */
    H2MG_X_LEAF_OFFSETS = 1,/* int32[2^L + 1]: tree-order offsets of the leaves       */
    H2MG_X_NEAR = 2,        /* int32[2 * pairs]: close leaf pairs (t, s), t <= s      */
    H2MG_X_FAR = 3,         /* int32[2 * pairs]: far pairs (t, s), t < s, of tree level arg */
    H2MG_X_RANKS = 4,       /* int32[2^arg]: ranks r_j of the clusters of tree level arg */
    H2MG_X_BOXES = 5,       /* double[2^arg * 2 * dim]: (lo, hi) boxes of tree level arg */
    H2MG_X_SKELETON = 6     /* int32[2^arg * 64]: SKELETON bases: skeleton of each cluster of
                               tree level arg, as original point indices in pivot order,
                               -1 beyond the cluster's rank */
} h2mg_export_what;

/* Copy the structure `what` to host memory `buf` of `cap` bytes; *bytes = size needed. */
h2mg_status h2mg_export(h2mg_matrix A, int what, int arg, void* buf, int64_t cap,
                        int64_t* bytes);

/* y = A_i x for multigrid level i (1..l) of the hierarchy (Sec. 3.3): at i = 1 the
 * H2 matrix itself in user point order (like h2mg_apply); for i >= 2 the Galerkin
 * operator on the coefficient space of tree level m(i) = L - i + 2, with k_pad =
 * KC slots per cluster in cluster order (slots beyond a cluster's rank are zero).
 * precision selects the primary copy (F64) or the FP32 copy (MIXED_F32). Device
 * or host vectors; one column. For i = l it applies the dense coarse matrix. */
h2mg_status h2mg_apply_level(h2mg_matrix A, int level, int precision, const double* x,
                             double* y, void* stream);

/* e = dir_sol(A_l, r) through A_l^{-1}, formed at build from the Cholesky factor of
 * the coarsest operator (Sec. 3.3, the dir_sol step of Algorithm 1). Vectors as for h2mg_apply_level at i = l. */
h2mg_status h2mg_coarse_solve(h2mg_matrix A, const double* r, double* e, void* stream);

/* One call of the smoother Iter(A_i, f, x0) = n iterations of CG (Sec. 3.3) on
 * multigrid level i; x0 = NULL means zero. x receives the iterate and r (optional)
 * the recurrence residual. Vectors as for h2mg_apply_level. */
h2mg_status h2mg_smooth(h2mg_matrix A, int level, int precision, const double* f,
                        const double* x0, int n, double* x, double* r, void* stream);

/* Inter-level transfer of Algorithm 1 (Sec. 3.3): direction 0 = restriction
 * out = U_i^T v (level i -> level i+1), direction 1 = prolongation out = U_i v
 * (level i+1 -> level i; out is overwritten). Vectors as for h2mg_apply_level. */
h2mg_status h2mg_transfer(h2mg_matrix A, int level, int direction, const double* v, double* out,
                          void* stream);

/* One V-cycle (Algorithm 1) from x0 with r1 = b - A x0 given: x_out = x0 + e_1. */
h2mg_status h2mg_vcycle(h2mg_matrix A, const double* x0, const double* r1, double* x_out,
                        const h2mg_solve_opts* o, void* stream);

/* Number of CUDA kernels this library has launched in this process so far (all
 * handles, all threads). Callers difference two readings to count the launches of a
 * region of work. */
int64_t h2mg_launch_count(void);

/* Timing of the symmetric block-sparse product (the kernel that streams the stored
 * blocks D, S and P_i). enable = 1 clears the record and starts recording a pair of
 * CUDA events around each of its launches on the launching stream; enable = 2 does the
 * same for the launches on the FP32 copy only (the mixed-precision cycle's products,
 * without the float64 and double-double residual products); enable = 0 stops.
 * On every call *launches, *ms (sum of the launch durations) and *bytes (sum of the
 * algorithmic bytes: stored blocks, input and output vectors, transposed partials)
 * are returned for the record so far; reading synchronises the recorded events.
 * Any output pointer may be NULL. */
h2mg_status h2mg_profile(h2mg_matrix A, int enable, int64_t* launches, double* ms, double* bytes);

/* Autotuner of the block-sparse product (the kernel that streams D, S and P_i). The
 * library launches it with a number of CTAs per block row; by default a fixed rule
 * (enough CTAs to fill the GPU when an operator has few block rows). This call times
 * trial launches of every operator of the hierarchy (index 0: the close part of level
 * 1; index i >= 1: the coupling operator of level i), for the primary format with 1
 * and 2 columns and the FP32 copy with 1, 2 and 4 columns, over the splits 1..64, and
 * keeps the fastest in the handle; later products, smoothers and solves use it (a
 * CUDA graph captured before the call keeps the old choice). report (optional, cap
 * entries of 4 doubles) receives (operator index, columns, ms with the fixed rule, ms
 * tuned) per combination; *count (optional) = the number of combinations. Runs on
 * `stream` and synchronises it; h2mg_profile must be off. No counterpart in the paper
 * (a launch-configuration choice of this implementation). */
h2mg_status h2mg_autotune(h2mg_matrix A, void* stream, double* report, int cap, int* count);

/* ---------------------------------------------------------------- allocation-free product
 * The paper has no counterpart to this call; it exists for callers that cannot
 * allocate device memory where they need a product: code inside allocator callbacks
 * (which must not re-enter the allocator), or processes whose device memory another
 * allocator (a framework's caching pool) has reserved in full, so that a cudaMalloc
 * would fail.
 *
 * h2mg_apply_noalloc computes y = A x like h2mg_apply (one column, device x and y
 * only; host pointers are rejected with INVALID_ARG) but calls no cudaMalloc,
 * cudaFree or allocating library routine: its workspace lives in one fixed array of
 * H2MG_NOALLOC_SCRATCH_BYTES bytes of device memory that every GPU loading this
 * library holds until the process exits. Matrices whose product needs more scratch
 * than that are rejected with UNSUPPORTED (the workspace is three coefficient buffers
 * of 8 * clusters * KC bytes and two point buffers of 8 * leaves * KD bytes: about 64
 * bytes per point in 3-D with leaf 64 and 64 nodes, so some 2^18 such points fit).
 * Vectors must be n float64 entries on the current device. The first call on a device
 * looks up the array's address with that device current. All calls
 * share the array and it keeps the last call's contents: calls whose work overlaps
 * on the GPU (different streams, or different host threads) race and give wrong
 * results. */
#define H2MG_NOALLOC_SCRATCH_BYTES (16u << 20)
h2mg_status h2mg_apply_noalloc(h2mg_matrix A, const double* x, double* y, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* H2MG_H */
