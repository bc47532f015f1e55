/*
 * h2sp -- non-extensive sparsification of H^2 matrices on one GB300 GPU.
 *
 * The library builds, for an H^2 matrix A given by its parameters
 * (Definition 4.9, §4.1), the factorization  A = U S V^T  of §2 (Eq.
 * main_fact): U and V are orthogonal products of block-diagonal and
 * permutation matrices (Eq. main_uv), S is a sparse N x N matrix of the same
 * size as A.  It then factors S by a block LU and solves  A x = b  as
 * S y = U^T b,  x = V y  (§1, Eq. sp0), directly or as the preconditioner of
 * iterative refinement / GMRES driven by the H^2 matrix-vector product (§5.5).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Index space.  Vectors are indexed in cluster-tree order: the points are
 *   ordered so that every cluster owns the contiguous range
 *   [begin[t], begin[t] + size[t]).  Vectors are FP64, column-major, with a
 *   leading dimension >= n; nrhs columns.
 * - Memory.  Pointers documented as "host" must be host memory; pointers
 *   documented as "device" must be device memory of the current device.  The
 *   H^2 numeric arrays are BORROWED: the handle keeps pointers to them and
 *   reads them again in h2sp_apply(H2SP_OP_H2) and in iterative solves, so
 *   they must stay valid and unchanged until h2sp_destroy.  Everything else
 *   the library needs (the blocks of U and V, S, the factors, workspaces) is
 *   allocated by the library with cudaMallocAsync on the call's stream and
 *   owned by the handle.
 * - Asynchrony.  Work is enqueued on the stream passed to each call.  Calls
 *   that must look at device results (h2sp_factor's pivot check, h2sp_solve's
 *   residual checks, exports) synchronise that stream before returning.
 * - Errors.  Every entry point returns an h2sp_status; nothing aborts or
 *   throws.  On error the handle is left in a state where h2sp_destroy is
 *   the only guaranteed-safe call.  h2sp_status_string names each code.
 * - Threading.  A handle must not be used by two host threads at once.
 */
#ifndef H2SP_H
#define H2SP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *h2sp_stream; /* a cudaStream_t; NULL = legacy default stream */
typedef struct h2sp_handle h2sp_handle;

typedef enum {
  H2SP_OK = 0,
  H2SP_EINVAL = -1,     /* malformed descriptor or argument; nothing was launched */
  H2SP_ENOMEM = -2,     /* device allocation failed */
  H2SP_ECUDA = -3,      /* a CUDA runtime call failed (see h2sp_last_cuda_error) */
  H2SP_ESINGULAR = -4,  /* a pivot block of S is singular (zero pivot) */
  H2SP_ESTATE = -5,     /* calls in the wrong order (e.g. solve before factor) */
  H2SP_ENOCONV = -6,    /* the iteration did not reach the tolerance in maxit */
  H2SP_ETIMEOUT = -7,   /* a bounded device wait gave up */
  H2SP_EUNSUPPORTED = -8 /* a valid input outside what the library supports (block too large) */
} h2sp_status;

/* Precision and kind of the factorization of S (h2sp_factor).  Bit 0: FP32
 * fronts; bit 1: block Cholesky S = L L^T instead of the block LU; bit 2: BF16
 * block-end updates; bit 3: their two-term split. */
typedef enum {
  H2SP_FP64 = 0,      /* block LU, FP64 fronts, FP64 arithmetic */
  H2SP_FP32 = 1,      /* block LU, FP32 fronts, FP32 arithmetic (a preconditioner for FP64 IR/GMRES) */
  H2SP_FP64_CHOL = 2, /* block Cholesky of a symmetric positive definite S, FP64 */
  H2SP_FP32_CHOL = 3, /* block Cholesky of a symmetric positive definite S, FP32 (tensor-core updates) */
  H2SP_BF16_CHOL = 7, /* H2SP_FP32_CHOL with the block-end updates in BF16: each 128-row tile of L21 scaled by
                         a power of two (its largest entry's exponent) and rounded to BF16, products accumulated
                         in FP32 and rescaled; a preconditioner for FP64 GMRES / refinement */
  H2SP_BF16X3_CHOL = 15 /* as H2SP_BF16_CHOL, with each scaled entry split into two BF16 values, x = hi + lo
                           (lo = the rounding error of hi, rounded), and three BF16 products per update:
                           hi*hi + hi*lo + lo*hi (about 16 significant bits) */
} h2sp_prec;

/* Operators for h2sp_apply. */
typedef enum {
  H2SP_OP_UT = 0,   /* out = U^T in   (point space -> S space)         Eq. sp0 */
  H2SP_OP_V = 1,    /* out = V in     (S space -> point space)         Eq. sp0 */
  H2SP_OP_U = 2,    /* out = U in                                      Eq. main_uv */
  H2SP_OP_VT = 3,   /* out = V^T in                                    Eq. main_uv */
  H2SP_OP_S = 4,    /* out = S in     (S space -> S space)             Eq. main_fact */
  H2SP_OP_H2 = 5,   /* out = A in, the FP64 H^2 product of Definition 4.9 */
  H2SP_OP_SINV = 6  /* out = S^{-1} in with the current factors (needs h2sp_factor) */
} h2sp_op;

/* Solve modes for h2sp_solve. */
typedef enum {
  H2SP_DIRECT = 0, /* x = V S^{-1} U^T b once (Eq. sp0) */
  H2SP_IR = 1,     /* iterative refinement on the FP64 H^2 residual, preconditioned by the factors */
  H2SP_GMRES = 2   /* restarted right-preconditioned GMRES on the FP64 H^2 product (§5.5) */
} h2sp_mode;

/*
 * One H^2 matrix (Definition 4.9, §4.1).
 *
 * The cluster tree is level-uniform (every leaf at depth `depth`); clusters
 * are numbered depth by depth, and inside one depth in the order of their
 * parents, so the children of a cluster have consecutive numbers and a
 * cluster's children come in increasing number.  Row and column cluster
 * trees are the same tree.  Column ranks equal row ranks.
 *
 * Batched form: depth 0 may hold several roots.  Each root's tree is then an
 * independent system (a diagonal block of A; no close or admissible pair may
 * join two trees, else H2SP_EINVAL).  All systems go through the same
 * launches level by level, their supernodes are factored in the same
 * elimination levels, and iterative solves stop when every system's relative
 * residual (per right-hand side) meets the tolerance.
 *
 * Blocks are column-major and packed; *_off arrays give each block's first
 * element in the packed array.
 */
typedef struct {
  int64_t n;                         /* number of points / rows of A */
  int32_t depth;                     /* leaf depth D >= 0 */
  /* ---- structure: HOST arrays ---- */
  const int32_t *level_ptr;          /* [D+2]; clusters of depth d: [level_ptr[d], level_ptr[d+1]) */
  const int32_t *parent;             /* [ncl]; -1 for cluster 0 (the root) */
  const int64_t *begin, *size;       /* [ncl]; contiguous index range of each cluster */
  const int32_t *rank;               /* [ncl]; k_t, the cluster-basis rank (Definition 4.7) */
  const int64_t *far_ptr;            /* [ncl+1]; CSR of the interaction list by row cluster */
  const int32_t *far_col;            /* [nfar];  same-depth column cluster of each admissible pair, ascending per row */
  const int64_t *near_ptr;           /* [nleaf+1]; CSR of the close blocks by leaf (leaf = cluster - level_ptr[D]) */
  const int32_t *near_col;           /* [nnear]; column leaf cluster ids, ascending per row */
  const int64_t *leaf_basis_off;     /* [nleaf]; R_t, |t| x k_t */
  const int64_t *transfer_off;       /* [ncl];   T_c, k_c x k_parent (entry 0 unused) */
  const int64_t *coupling_off;       /* [nfar];  D_ts, k_t x k_s */
  const int64_t *near_off;           /* [nnear]; C_ts, |t| x |s| */
  const int64_t *col_leaf_basis_off; /* [nleaf] or NULL */
  const int64_t *col_transfer_off;   /* [ncl] or NULL */
  /* ---- numbers: DEVICE arrays (borrowed, see above) ---- */
  const double *leaf_basis;          /* row cluster basis of the leaves */
  const double *transfer;            /* row transfer matrices */
  const double *coupling;            /* coupling matrices of the interaction list */
  const double *near_block;          /* close matrix blocks (Definition 4.8) */
  const double *col_leaf_basis;      /* column basis E of the leaves; NULL => E = R (symmetric bases) */
  const double *col_transfer;        /* column transfer matrices; NULL iff col_leaf_basis is NULL */
} h2sp_h2_desc;

/*
 * ---- GPU construction of an H^2 matrix (the parameters of Definition 4.9) ----
 *
 * h2sp_construct builds, for a kernel function a(x, y) and points in a
 * cluster tree, the H^2 matrix the sparsification takes: cluster bases by
 * tensor Chebyshev interpolation on each cluster's box (order p per axis,
 * rank p^dim <= 64; the leaf basis R_t[i, alpha] = L_alpha(x_i), the transfer
 * T_c[alpha, beta] = L^{parent}_beta(y_alpha) at the Chebyshev points y of
 * c), the coupling blocks D_ts = a(y_t, y_s) at the Chebyshev points, and
 * the close blocks a(x_i, x_j) with `diag` on the diagonal.  With tol > 0
 * the bases are then recompressed on the GPU:
 *   orthogonalised bottom-up by Householder QR (R_t = Q_t Z_t, and
 *   [Z_c T_c]_c = Q_t Z_t above the leaves, whose row blocks give the
 *   transfers Tq_c of the orthonormal basis); every cluster weighted by the
 *   far field its basis carries, top-down, M_t = sum_s Do_ts Do_ts^T +
 *   Tq_t M_parent Tq_t^T with Do_ts = Z_t D_ts Z_s^T; the eigenvectors B_t
 *   of M_t (Jacobi) with sqrt(lambda_i) > tol sqrt(lambda_0) kept; and the
 *   parameters rewritten as Q_t B_t, B_c^T Tq_c B_parent and B_t^T Do_ts B_s.
 * The weights are Gram matrices, so tol must be 0 or >= 1e-7 (H2SP_EINVAL).
 * Symmetric kernels only: column bases equal row bases.
 */
typedef enum {
  H2SP_KERNEL_LOG = 0,    /* -log r */
  H2SP_KERNEL_INV = 1,    /* 1 / r */
  H2SP_KERNEL_YUKAWA = 2, /* e^{-r} / r */
  H2SP_KERNEL_GAUSS = 3   /* e^{-r^2} */
} h2sp_kernel;

typedef struct {
  int64_t n;                     /* points */
  int32_t dim;                   /* 2 or 3 */
  int32_t depth;                 /* leaf depth D of the level-uniform tree */
  /* tree and lists: HOST arrays, with the rules of h2sp_h2_desc */
  const int32_t *level_ptr;      /* [D+2] */
  const int32_t *parent;         /* [ncl] */
  const int64_t *begin, *size;   /* [ncl]; every leaf non-empty */
  const double *box_lo, *box_hi; /* [ncl * dim], row-major: the box of each cluster (its Chebyshev grid) */
  const int64_t *far_ptr;        /* [ncl+1] */
  const int32_t *far_col;        /* [nfar] */
  const int64_t *near_ptr;       /* [nleaf+1] */
  const int32_t *near_col;       /* [nnear] */
  const double *points;          /* DEVICE [n * dim], row-major, in tree order */
  int32_t kernel;                /* h2sp_kernel */
  double diag;                   /* a_ii */
  int32_t order;                 /* Chebyshev points per axis p; p^dim <= 64 */
  double tol;                    /* 0: no recompression (rank p^dim); else >= 1e-7 */
} h2sp_construct_desc;

typedef struct h2sp_h2 h2sp_h2;  /* a constructed H^2 matrix: owns its arrays */

/* Builds the matrix on the current device, enqueued on `stream` and
 * synchronised before the call returns.  H2SP_EINVAL for a malformed tree or
 * argument (message in h2sp_last_cuda_error), H2SP_ENOMEM / H2SP_ECUDA on
 * device failures; *out is NULL then. */
int h2sp_construct(const h2sp_construct_desc *c, h2sp_stream stream, h2sp_h2 **out);

/* Fills *desc with m's structure (host arrays owned by m) and numbers
 * (device arrays owned by m; symmetric bases), valid until h2sp_h2_destroy:
 * the descriptor h2sp_analyze / h2sp_sparsify take. */
int h2sp_h2_describe(const h2sp_h2 *m, h2sp_h2_desc *desc);

/* Copies numeric array `which` (0 leaf_basis, 1 transfer, 2 coupling,
 * 3 near_block) of m to dst (host or device memory) and gives its element
 * count in *count; dst may be NULL to query the count.  Synchronous. */
int h2sp_h2_copy(const h2sp_h2 *m, int32_t which, double *dst, int64_t *count, h2sp_stream stream);

/* Frees m (NULL is allowed). */
void h2sp_h2_destroy(h2sp_h2 *m);

/* Bits of h2sp_opts.flags. */
enum {
  /* Sparsify with FP32 products: the sandwich products of the close blocks
   * and cross-level panels (Eq. cl0) run in FP32 and S is stored in FP32,
   * while the Householder completions (U and V orthogonal to FP64 accuracy)
   * and the coupling projections stay FP64.  Meant for the mixed-precision
   * solve, where S only builds the FP32 preconditioner and the FP64 H^2
   * product of Definition 4.9 decides convergence (§5.5); every apply and
   * product of the handle still takes and returns FP64 vectors. */
  H2SP_SPARSIFY_FP32 = 1
};

typedef struct {
  int32_t flags;       /* 0 or H2SP_SPARSIFY_FP32; any other bit is H2SP_EINVAL; opts may be NULL (= 0) */
} h2sp_opts;

typedef struct {
  int32_t mode;        /* h2sp_mode */
  double tol;          /* target max_k ||b_k - A x_k|| / ||b_k|| for IR / GMRES (e.g. 1e-10) */
  int32_t maxit;       /* iteration cap (IR: refinement steps; GMRES: total inner steps); <= 0: default */
  int32_t restart;     /* GMRES restart length (1..60; <= 0: 20); ignored by IR / DIRECT */
} h2sp_solve_opts;

typedef struct {
  int32_t iters;       /* refinement steps / GMRES inner steps taken */
  double rel_residual; /* final max_k ||b_k - A x_k|| / ||b_k|| (FP64 H^2 product); -1 for DIRECT */
  int32_t status;      /* h2sp_status of the solve */
} h2sp_solve_info;

/* Sizes and counters of a handle (filled by h2sp_query). */
typedef struct {
  int64_t n;
  int32_t depth, lstop;           /* leaf depth; first uncompressed level (levels count from the leaves) */
  int32_t nnodes;                 /* S nodes (non-basis blocks + top clusters) */
  int64_t nnzb, nnz;              /* blocks and scalar nonzeros of S */
  int32_t nsupernodes, nfront_levels;
  int64_t max_front;              /* largest front (s + b) */
  int64_t front_elems;            /* sum of (s+b)^2 over the fronts */
  double factor_flops;            /* sum over supernodes of (2/3)s^3 + 2 s^2 b + 2 s b^2 */
  double sparsify_flops;          /* algorithmic flops of the sparsification */
  int32_t factor_prec;            /* h2sp_prec of the current factors, -1 if none */
  double plan_seconds;            /* host time spent planning in the last h2sp_sparsify */
  int32_t sparsify_prec;          /* h2sp_prec of S (U and V are always FP64); -1 for an analysis-only handle */
  int32_t nsys;                   /* independent systems (roots at depth 0) */
  int32_t factor_chol;            /* 1 if the current factors come from the block Cholesky */
  double chol_flops;              /* sum over supernodes of s^3/3 + s^2 b + s b^2 (the block Cholesky's work) */
  int32_t compensated_pivots;     /* pivots of the last BF16-mode block Cholesky that were not positive and were
                                     replaced by their diagonal entry before the panel (0 otherwise) */
} h2sp_stats;

/*
 * h2sp_sparsify -- build A = U S V^T from the H^2 parameters (§2.1-2.3 with
 * the factors of §4.2-4.3).  Validates the descriptor on the host (returns
 * H2SP_EINVAL without launching anything if it is malformed: unsorted lists,
 * inconsistent tree, ranks that do not fit, a missing column array), plans
 * the level recursion and the symbolic factorization of S on the host, and
 * enqueues the kernels on `stream` (FP64; the products into S in FP32 with
 * H2SP_SPARSIFY_FP32): the Householder completions of the
 * cluster bases per level, the coupling projections, the transforms of the
 * close blocks and of the cross-level panels, and the scatter into S.
 * On success *out owns a new handle.
 */
int h2sp_sparsify(const h2sp_h2_desc *desc, const h2sp_opts *opts, h2sp_stream stream, h2sp_handle **out);

/*
 * h2sp_sparsify_analyzed -- h2sp_sparsify reusing the host analysis held by
 * `an` (a handle from h2sp_analyze or h2sp_sparsify) for a descriptor with the
 * same structure (every HOST array equal: sizes, tree, ranks, both lists and
 * all offsets) and new numbers.  This is the split of a sparse direct solver
 * into symbolic analysis and numeric phases; the paper builds its plan once
 * per structure as well (§4).  The structure is checked (its sizes, then a
 * 64-bit fingerprint of every structure array) before anything is launched:
 * a mismatch returns H2SP_EINVAL.  `an` stays valid and may be destroyed
 * before or after *out (the analysis is shared, reference counted).  The
 * device arrays of `desc` are borrowed as in h2sp_sparsify.
 */
int h2sp_sparsify_analyzed(const h2sp_handle *an, const h2sp_h2_desc *desc, const h2sp_opts *opts,
                           h2sp_stream stream, h2sp_handle **out);

/*
 * h2sp_analyze -- the host-only part of h2sp_sparsify: validate the
 * descriptor and plan the level recursion, the block pattern of S (§3) and
 * the symbolic factorization of S.  Makes no CUDA call and does not read the
 * numeric arrays of the descriptor (they may be NULL).  The resulting handle
 * supports h2sp_query, h2sp_export_structure, h2sp_export_S with vals == NULL
 * and h2sp_destroy; every other call returns H2SP_ESTATE.
 */
int h2sp_analyze(const h2sp_h2_desc *desc, h2sp_handle **out);

/*
 * h2sp_factor -- block LU of S (the paper factors S with a sparse direct
 * method, §5.3-5.4): nested-dissection order along the cluster tree,
 * multifrontal elimination level by level, partial pivoting inside each
 * supernode's diagonal block.  `prec` selects FP64 or FP32 fronts.  FP64
 * fronts take one trailing update per 32-column panel.  FP32 fronts are
 * factored in 256-column outer blocks of four panels: interchanges and
 * updates stay inside the block until its end, then the other columns take
 * the interchanges, the triangular solve for U12 and one rank-256 update on
 * the tensor cores with operands split into two TF32 terms (FP32-level
 * products); the same factorization up to rounding order.  The panels and
 * the next block's columns run on an internal high-priority stream, the rest
 * of each block end on an internal low-priority one; both are joined back to
 * `stream` before the call returns.
 *
 * H2SP_FP64_CHOL / H2SP_FP32_CHOL select the block Cholesky S = L L^T
 * instead: the sparse package of §5.3-5.4 is a Cholesky code, and
 * Proposition 2.1 makes S symmetric positive definite when A is.  Same
 * supernodes and fronts, no pivoting, half the work (h2sp_stats.chol_flops):
 * per panel the diagonal tile's Cholesky and L21 = F21 L11^-T, then the lower
 * triangle of the trailing matrix only, C -= L21 L21^T (FP32: 256-column outer
 * blocks with rank-256 tensor-core updates of the lower 128 x 128 tiles).
 * The factors are stored in the LU form (unit L = L_chol D^-1, U = D L_chol^T,
 * D = diag(L_chol)), so h2sp_solve, H2SP_OP_SINV and h2sp_logdet work as for
 * the LU.  Needs symmetric bases (no column bases; H2SP_EINVAL otherwise) and
 * a symmetric S; a pivot that is not positive (S not positive definite in the
 * factor's precision) returns H2SP_ESINGULAR with a message in
 * h2sp_last_cuda_error.  H2SP_BF16_CHOL / H2SP_BF16X3_CHOL are H2SP_FP32_CHOL
 * with the rank-256 block-end updates on BF16 tensor cores (one power-of-two
 * scale per 128-row tile of L21); they need the tensor-core path
 * (H2SP_EUNSUPPORTED otherwise).  One BF16 term keeps 8 significant bits; the
 * two-term split about 16, at half the tensor work of the TF32 split.  Their
 * factors are a preconditioner only: a pivot that comes out not positive is
 * replaced by the diagonal entry as the panel found it (the pivot before the
 * panel's own sums: diagonal compensation) and counted in
 * h2sp_stats.compensated_pivots, instead of failing the call.
 *
 * Synchronises the stream; returns H2SP_ESINGULAR on a zero or non-finite
 * pivot and H2SP_ETIMEOUT if a bounded device wait gave up.
 */
int h2sp_factor(h2sp_handle *h, int32_t prec, h2sp_stream stream);

/*
 * h2sp_factor_ilut -- threshold incomplete LU of S, the preconditioner of
 * §5.5 (ILUt with a drop tolerance tau; the paper takes 1e-2 and 2e-2):
 * the rows of S in the elimination order of the block LU (supernodes in
 * order, each node's rows together), no pivoting; for each row i, with
 * tau_i = tau ||S_i||_2, the multipliers w_k (k < i in increasing order)
 * below tau_i are dropped before their update, and at the end every entry
 * below tau_i except the diagonal.  tau = 0 gives the exact LU without
 * pivoting of that matrix.  Computed in FP64 on the GPU from S (either
 * sparsification precision); the supernodes of each elimination level in
 * parallel, the rows of a supernode in order.  Afterwards h2sp_solve,
 * H2SP_OP_SINV and the preconditioner of IR / GMRES use (L U)^{-1}
 * (h2sp_stats.factor_prec = H2SP_FP64); h2sp_logdet, h2sp_refactor,
 * h2sp_solve_captured and h2sp_export_front return H2SP_ESTATE until the next
 * h2sp_factor.  H2SP_EINVAL for tau < 0 or not finite; H2SP_ESINGULAR on a
 * zero pivot; H2SP_ENOMEM if the factors outgrow the memory.  Synchronous.
 * Work space: a dense row and a bitmap of n entries for each CTA of the
 * widest elimination level (at most two per SM), about 8.1 n bytes each,
 * and a pool for the factors that starts at max(4 nnz(S), 64 n) entries and
 * grows fourfold (recomputing the factorization) while it overflows.
 */
int h2sp_factor_ilut(h2sp_handle *h, double tau, h2sp_stream stream);

/*
 * h2sp_export_ilut -- the incomplete factors, host arrays in elimination
 * order (row e is row perm[e] of S): L strictly lower (unit diagonal not
 * stored) as CSR l_ptr[n+1], l_col, l_val; U upper, diagonal first in each
 * row, as u_ptr[n+1], u_col, u_val; columns ascending, in elimination order.
 * Any pointer may be NULL (query *nnz_l and *nnz_u first).  H2SP_ESTATE
 * unless the current factors come from h2sp_factor_ilut.
 */
int h2sp_export_ilut(h2sp_handle *h, int32_t *perm, int64_t *l_ptr, int32_t *l_col, double *l_val, int64_t *u_ptr,
                     int32_t *u_col, double *u_val, int64_t *nnz_l, int64_t *nnz_u);

/*
 * h2sp_refactor -- repeat the numeric sparsification and the factorization of
 * `h`, in the precision of its last h2sp_factor, for new numbers written into
 * the borrowed H^2 arrays the handle was built from (same device pointers,
 * same structure): the persistent form of the batched path.  The first call
 * captures every launch of both phases, on every internal stream, into a CUDA
 * graph that the handle owns; later calls replay it with one graph launch.
 * No counterpart in the paper, which refactors by running its pipeline again.
 * Needs a previous h2sp_factor (H2SP_ESTATE otherwise).  Synchronises the
 * stream; returns H2SP_ESINGULAR / H2SP_ETIMEOUT as h2sp_factor.
 */
int h2sp_refactor(h2sp_handle *h, h2sp_stream stream);

/*
 * h2sp_solve -- x = A^{-1} b through S y = U^T b, x = V y (Eq. sp0), either
 * once (DIRECT, needs h2sp_factor) or iterated on the FP64 H^2 residual
 * (IR, or GMRES right-preconditioned by the factored S, §5.5).  b (ldb >= n)
 * and x (ldx >= n) are device arrays of nrhs columns (1 <= nrhs <= 64, else
 * H2SP_EINVAL); x may not alias b.
 * `info` (host, may be NULL) receives iterations and the final relative
 * residual.  The triangular sweeps are one cooperative launch per level and
 * direction whose row blocks wait (bounded) for the blocks they depend on;
 * a wait that gives up makes the call return H2SP_ETIMEOUT.  Synchronises
 * the stream.
 */
int h2sp_solve(h2sp_handle *h, const h2sp_solve_opts *opts, int32_t nrhs, const double *b, int64_t ldb,
               double *x, int64_t ldx, h2sp_solve_info *info, h2sp_stream stream);

/*
 * h2sp_solve_captured -- iterative refinement with a fixed number of steps,
 * captured in a CUDA graph: x_0 = M^-1 b, then `steps` times
 * x += M^-1 (b - A x) with M^-1 = V S^-1 U^T from the current factors and A
 * the FP64 H^2 product (§5.5), then the final residual; no host decision
 * between the launches.  The first call for given (b, ldb, x, ldx, nrhs,
 * steps) and factor precision captures every launch into a graph the handle
 * owns; later calls with the same arguments replay it with one graph launch
 * (new values in b, or new factors from h2sp_refactor, are picked up).  The
 * sweeps' flags are zeroed at the start of every replay, so the epochs fixed
 * at capture are new each time.  Needs h2sp_factor; device arrays as for
 * h2sp_solve, 1 <= nrhs <= 64, 0 <= steps <= 100.  info (may be NULL) gets
 * steps and the final max relative residual over systems and columns;
 * returns H2SP_ENOCONV if that is above tol (x is still the last iterate),
 * H2SP_ETIMEOUT if a sweep's wait gave up.  Synchronises the stream.
 */
int h2sp_solve_captured(h2sp_handle *h, int32_t steps, double tol, int32_t nrhs, const double *b, int64_t ldb,
                        double *x, int64_t ldx, h2sp_solve_info *info, h2sp_stream stream);

/*
 * h2sp_solve_host -- the whole path in one call, from and to HOST memory:
 * x = A^{-1} b with A = U S V^T built (§2.1-2.3, §4.2-4.3), S factored and
 * the system solved as h2sp_sparsify_analyzed + h2sp_factor + h2sp_solve do.
 * Here the numeric arrays of `desc` (leaf_basis, transfer, coupling,
 * near_block and, if present, the column arrays) and b (ldb >= n, nrhs
 * columns, 1 <= nrhs <= 64) are HOST arrays (page-locked memory copies
 * fastest); the call copies them to the device on `stream`, runs the
 * sparsification (opts), the factorization (prec, an h2sp_prec) and the solve
 * (sopts), copies the solution to the host array x (ldx >= n) and frees every
 * device buffer it made before returning.  `an` is an analysis of the same
 * structure (h2sp_analyze / h2sp_sparsify; checked as h2sp_sparsify_analyzed
 * checks it) or NULL to plan one inside the call.  info (may be NULL) as for
 * h2sp_solve.  Returns the first failing status of the three steps; with
 * H2SP_ENOCONV x still holds the last iterate.  Synchronises the stream.
 */
int h2sp_solve_host(const h2sp_handle *an, const h2sp_h2_desc *desc, const h2sp_opts *opts, int32_t prec,
                    const h2sp_solve_opts *sopts, int32_t nrhs, const double *b, int64_t ldb, double *x, int64_t ldx,
                    h2sp_solve_info *info, h2sp_stream stream);

/*
 * h2sp_logdet -- log|det A| of every independent system from the current
 * factors of S.  §5.3 proposes the factorization of the sparse S as a way to
 * the determinant of the dense matrix: U and V are orthogonal (Eq. main_uv),
 * so |det A| = |det S|, and block elimination makes det S the product over
 * the supernodes of det F11 = (-1)^(row interchanges) * prod_j u_jj of their
 * pivot blocks.  logabsdet (host, nsys doubles, nsys from h2sp_query) gets
 * the sums of log|u_jj|, accumulated in FP64 in a fixed order; sign (host,
 * nsys int32, may be NULL) gets the sign of det S, +1 or -1, which is also
 * the sign of det A when the column bases are NULL (V = U, so det A =
 * det(U)^2 det S); with separate column bases det A = det U det V det S and
 * det U, det V (each +1 or -1) are not computed.  The value is that of the
 * factored S in the factors' precision: with H2SP_FP32 factors it carries
 * the FP32 rounding of the pivots.  Needs h2sp_factor (H2SP_ESTATE
 * otherwise).  Synchronises the stream.
 */
int h2sp_logdet(h2sp_handle *h, double *logabsdet, int32_t *sign, h2sp_stream stream);

/*
 * h2sp_apply -- out = op(in) for one of the operators above; device arrays,
 * nrhs columns, leading dimensions >= n.  `in` and `out` must not alias.
 */
int h2sp_apply(h2sp_handle *h, int32_t op, int32_t nrhs, const double *in, int64_t ldin, double *out,
               int64_t ldout, h2sp_stream stream);

/*
 * h2sp_export_S -- copy S to host arrays in its variable-block (VBR) layout:
 * node_size[nnodes], brow_ptr[nnodes+1] (int64), bcol_idx[nnzb] (int32,
 * ascending per block row), val_off[nnzb] (int64), vals[nnz] (each block
 * column-major).  Pass NULL for any array to skip it; call h2sp_query first
 * for the sizes.  Synchronises the stream.
 */
int h2sp_export_S(h2sp_handle *h, int64_t *node_size, int64_t *brow_ptr, int32_t *bcol_idx, int64_t *val_off,
                  double *vals, h2sp_stream stream);

/*
 * h2sp_export_Q -- copy the square orthogonal block Q_t of cluster t (the
 * diagonal block of U_l at t's level, §4.2; columns [0, k') span the basis,
 * columns [k', m) the non-basis part) to host memory `q` (m x m, column
 * major), and its local size to *m.  col != 0 selects the column side (V).
 * q may be NULL to query m.  Clusters at or above the top level have m = 0.
 */
int h2sp_export_Q(h2sp_handle *h, int32_t cluster, int32_t col, int64_t *m, double *q, h2sp_stream stream);

/*
 * h2sp_export_structure -- integer structure for verification, host arrays:
 * node_level[nnodes], node_cluster[nnodes], closure[nnodes] (closure cluster
 * of each node), order[nnodes] (elimination order), sn_ptr[nsupernodes+1]
 * (supernodes as ranges of `order`), bnd_ptr[nsupernodes+1] and
 * bnd[bnd_ptr[nsupernodes]] (boundary nodes of each supernode, in
 * elimination order).  Any pointer may be NULL.  *nbnd receives the total
 * boundary length when not NULL.
 */
int h2sp_export_structure(h2sp_handle *h, int32_t *node_level, int32_t *node_cluster, int32_t *closure,
                          int32_t *order, int32_t *sn_ptr, int32_t *bnd_ptr, int32_t *bnd, int64_t *nbnd);

/*
 * h2sp_export_schedule -- the level schedule of §2.2-2.3 as the device
 * kernels build it: runs them now, on the current device, for the structure
 * of h (an analysis or a numeric handle), and copies the result to host
 * arrays (any pointer may be NULL).  Per cluster (ncl = level_ptr[depth + 1]
 * entries): m (local block size m_t: |t| at the leaves, the sum of the
 * children's k' above), kp (basis part k'_t = min(k_t, m_t) below l_stop, 0 at
 * l_stop; d_t = m_t - k'_t rows of t enter S), off (row of t's basis part in
 * its parent's block), xoff (offset of X_l(t) in the level-l vector; 0 above
 * l_stop).  Per S node (nnodes + 1 entries, h2sp_query): node_off (first row
 * of the node in S, node_off[nnodes] = n); node_cluster (nnodes entries).
 * *lstop: l_stop, the level whose clusters are kept whole (one above the
 * highest level with an admissible pair).  Synchronous.  The same kernels
 * build the plan of h2sp_sparsify and the level maps of every numeric
 * handle; this entry exposes them for verification.
 */
int h2sp_export_schedule(h2sp_handle *h, int32_t *lstop, int64_t *m, int64_t *kp, int64_t *off, int64_t *xoff,
                         int64_t *node_off, int32_t *node_cluster);

/*
 * h2sp_export_near -- the close list Near_level (1 <= level <= l_stop) of the
 * device level schedule: Near_{l+1} = {(par a, par b) : (a, b) in Near_l or
 * Far_l}, each pair once (§2.3: the admissible pairs of level l join their
 * parents' close blocks).  CSR over the clusters of the level in tree order:
 * ptr (clusters of the level + 1 entries), col (*nnz cluster indices,
 * ascending within a row).  Query *nnz first with col == NULL.  H2SP_EINVAL
 * for a level outside [1, l_stop].  Synchronous.
 */
int h2sp_export_near(h2sp_handle *h, int32_t level, int64_t *ptr, int32_t *col, int64_t *nnz);

/*
 * h2sp_export_front -- copy the front of supernode k (0 <= k < nsupernodes, in
 * elimination order; rows and columns = the supernode's S rows, then its
 * boundary rows, as h2sp_export_structure lists them) to host memory vals
 * (f x f, column-major, FP64; FP32 factors are widened).  After h2sp_factor its
 * first s columns hold the factors of the supernode (§5.3): unit lower L
 * strictly below the diagonal and U on and above it, rows interchanged by the
 * supernode's pivoting (none for the block Cholesky, whose L_chol is
 * L D^1/2 with D = diag(U)).  The last f - s columns hold U12 above row s;
 * the rest is work space.  *f and *s (may be NULL) receive the sizes; vals
 * may be NULL to query them.  H2SP_ESTATE before h2sp_factor.  Synchronises
 * the stream.
 */
int h2sp_export_front(h2sp_handle *h, int32_t k, int64_t *f, int64_t *s, double *vals, h2sp_stream stream);

/* Per-kernel-class counters of a handle (h2sp_profile).  Classes:
 *  0 trailing GEMM update of the fronts     6 basis completions (Householder)
 *  1 panel factorization with pivoting      7 coupling projections, W stacking
 *  2 row swaps + U12 triangular solve       8 triangular solves with the fronts
 *  3 extend-add into parent fronts          9 FP64 H^2 product
 *  4 S blocks into fronts                  10 U^T / V applies
 *  5 close-block / panel transforms        11 vector kernels, casts, permutations
 * 12 FP32 blocked factorizations: in-block rank-64 tensor-core updates and
 *    operand packing
 * work[] is the algorithmic flop count (classes 0, 1, 2, 5, 9), bytes (4, 8,
 * 11, 12) or elements (3) of the timed launches; 0 where not defined (6, 7,
 * 10). */
typedef struct {
  int64_t launches[16];   /* kernel launches since the last reset (always counted) */
  int64_t timed[16];      /* launches or launch groups bracketed by CUDA events */
  double ms[16];          /* summed event time of the timed launches */
  double work[16];        /* algorithmic work of the timed launches */
} h2sp_kernel_times;

/*
 * h2sp_profile -- per-kernel-class timing.  timing = 1 brackets every later
 * launch (or launch group of a solve sweep) of this handle with CUDA events
 * recorded on the launching stream, timing = 0 stops, timing = -1 leaves it
 * as is.  Synchronises on the last recorded event, then copies the counters
 * to *out (may be NULL) and zeroes them when reset != 0.
 */
int h2sp_profile(h2sp_handle *h, int32_t timing, int32_t reset, h2sp_kernel_times *out);

/*
 * h2sp_h2_matvec_static -- y = A x, the same FP64 H^2 product as
 * h2sp_apply(H2SP_OP_H2), for callers that cannot allocate device memory at
 * the point of the call: code running while a memory pool is locked or
 * budgeted by someone else, inside a tight real-time loop that must not hit
 * the allocator, or in a plug-in whose host forbids cudaMalloc.  The paper
 * has no counterpart of this entry point; it is an interface convenience.
 *
 * It allocates nothing: the two coefficient workspaces of the upward and
 * downward passes live in a file-scope __device__ array of the library of
 * 2^21 doubles (16 MiB), which every GPU that loads the library keeps until
 * the process exits.  It needs 2 * 16 * (sum of the cluster ranks) doubles;
 * a larger matrix is rejected with H2SP_EUNSUPPORTED and a message in
 * h2sp_last_cuda_error.  The first call on each device looks up the array's
 * device address (cudaGetSymbolAddress) with that device current; make that
 * first call before any stream capture.  Every call shares the one array and
 * leaves its last contents there (each element is written before it is read,
 * so nothing needs clearing), so calls that overlap on the GPU -- on
 * different streams, or from different host threads -- race; serialise them.
 * h is a handle from h2sp_sparsify (its device structure is read, not
 * changed), and the current device must be the one it was built on
 * (H2SP_EINVAL otherwise, with a message in h2sp_last_cuda_error); x
 * (ldx >= n) and y (ldy >= n) are device arrays of nrhs columns.
 * Enqueued on `stream`; does not synchronise.
 */
int h2sp_h2_matvec_static(const h2sp_handle *h, int32_t nrhs, const double *x, int64_t ldx, double *y, int64_t ldy,
                          h2sp_stream stream);

/* Options of h2sp_set_option. */
enum {
  /* Polls of one flag wait of the triangular sweeps before it gives up (the
   * solve then returns H2SP_ETIMEOUT); 1 .. 2^31, default 2^22 (on the order
   * of a second: each poll is an acquire load and a 32 ns back-off). */
  H2SP_OPTION_WAIT_POLLS = 1,
  /* Test of the bounded waits: value != 0 makes the forward sweeps of the
   * next solve of this handle await an epoch that no solved block publishes,
   * so every wait of a block on another runs out; that solve returns
   * H2SP_ETIMEOUT and the option clears itself.  The handle, its factors and
   * the device stay usable (a wait that runs out raises an error word and
   * leaves; nothing faults or traps). */
  H2SP_OPTION_TEST_STALE_EPOCH = 2,
  /* Schedule of the FP32 block Cholesky (H2SP_FP32_CHOL), the knobs the
   * package's autotuner sets; none changes the result beyond rounding order.
   * TILES_PER_CTA: most 128-column tiles one CTA of the low-priority
   * block-end update takes (0, the default: a whole-wave split); short CTAs
   * let the panel stream reach the SMs sooner.  PANEL_SMS: SMs that update
   * leaves to the panel stream (-1, the default: one per front of the
   * level).  LOOKAHEAD: 1 (default) factors the next block's panels on a
   * high-priority stream while the rest of the update runs, 0 serialises.
   * WIDE: the TF32 block-end update's tiles: 2 (default) 128 x 256 output
   * tiles (one N = 256 MMA over two packed column tiles: a quarter fewer
   * operand bytes per product) with the product subtracted from C by a TMA
   * reduce-add, which frees a shared-memory buffer for a fourth operand
   * stage; 1 the same tiles with C loaded and stored; 0 128 x 128 tiles. */
  H2SP_OPTION_CHOL_TILES_PER_CTA = 3,
  H2SP_OPTION_CHOL_PANEL_SMS = 4,
  H2SP_OPTION_CHOL_LOOKAHEAD = 5,
  H2SP_OPTION_CHOL_WIDE = 6
};

/*
 * h2sp_set_option -- set a runtime option of handle h (the enum above).
 * H2SP_EINVAL for an unknown option or a value out of range.
 */
int h2sp_set_option(h2sp_handle *h, int32_t option, int64_t value);

/*
 * h2sp_measure_peak -- the fused multiply-add rate of the current device in
 * TFLOP/s into *tflops: kind 0 for FP64, 1 for FP32 on the CUDA cores.  One
 * warm-up and one timed launch (CUDA events on `stream`, about 50 ms) of
 * independent FMA chains on every multiprocessor.  A measurement aid for the
 * roofline fractions of the FP64 / FP32 CUDA-core kernels; the paper has no
 * counterpart.  Synchronises the stream.
 */
int h2sp_measure_peak(int32_t kind, double *tflops, h2sp_stream stream);

/* h2sp_query -- fill *st with the handle's sizes and counters. */
int h2sp_query(const h2sp_handle *h, h2sp_stats *st);

/* h2sp_destroy -- free everything the handle owns (synchronises its last stream). NULL is a no-op. */
void h2sp_destroy(h2sp_handle *h);

/* Human-readable name of a status code. */
const char *h2sp_status_string(int32_t status);

/* Text of the last CUDA error seen by the library on this thread ("" if none). */
const char *h2sp_last_cuda_error(void);

#ifdef __cplusplus
}
#endif

#endif /* H2SP_H */
