/*
 * hodlr.h -- C ABI of libhodlr: HODLR-preconditioned GMRES for dense frontal
 * matrices on one GB300 GPU (sm_103a).
 *
 * The library follows Aminfar, Ambikasaran and Darve, "A Fast Block Low-Rank
 * Dense Solver with Applications to Finite-Element Matrices" (arXiv:1403.5337):
 *
 *   problem     K x = F, K in R^{n x n} dense, x, F in R^{n x s}       (Sec. 4.2)
 *   structure   HODLR: K = [[K1, U1 V12^T], [U2 V21^T, K2]] recursively (Sec. 4.1)
 *   compression ACA with partial pivoting (Sec. 5.1) or BDLR, the boundary-
 *               distance pseudo-skeleton with a full-pivoting LU (Sec. 5.3)
 *   factor      the recursive Sherman-Morrison-Woodbury scheme: leaf LU, one
 *               Woodbury core S_i^(p) per node (Sec. 4.3, Factorize)
 *   solve       applying the factored inverse (Sec. 4.3, Solve)
 *   iterative   GMRES with the low-accuracy HODLR solve as preconditioner (Sec. 3)
 *
 * Conventions common to every call
 * --------------------------------
 * - Pointers named "device" are CUDA device pointers on the context's device;
 *   "host" pointers are ordinary host memory.  No call takes ownership of a
 *   caller buffer.  The caller keeps A (and the graph) alive and unchanged for
 *   as long as any hodlr_t built from it, or any gmres_solve using it, is in use.
 * - Dense matrices are FP64 and ROW-major with a leading dimension (ld >= n).
 *   Right-hand sides and solutions are n x s, COLUMN-major (each right-hand side
 *   contiguous), with ld >= n.
 * - The index order of A is the HODLR tree order: every tree node is a
 *   contiguous index range.  By default the tree halves each range (lower half
 *   floor(size/2)) until all leaves hold at most `leaf` rows; explicit leaf
 *   boundaries may be passed instead (hodlr_opts.leaf_bounds).
 * - Calls are ordered on the CUDA stream they are given (NULL = legacy default
 *   stream).  hodlr_build and gmres_solve synchronise that stream before they
 *   return (they read a few device scalars); hodlr_factor and hodlr_solve do not.
 * - Every call returns a hodlr_status.  On failure hodlr_last_error() gives a
 *   thread-local message.  Device-side failures (a zero pivot, a non-finite
 *   value, a wait that ran out of its budget) are reported through a device
 *   status word that the next synchronising call reads; they never trap.
 * - Library-owned device memory comes from the allocator given to
 *   hodlr_ctx_create (or cudaMallocAsync / cudaFreeAsync when none is given).
 */
#ifndef HODLR_H
#define HODLR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HODLR_ABI_VERSION 1

/* Same type as cudaStream_t. */
typedef struct CUstream_st *hodlr_stream;

typedef enum {
    HODLR_OK = 0,
    HODLR_INVALID_ARG = 1,      /* a size, pointer or option is out of range        */
    HODLR_OUT_OF_MEMORY = 2,    /* the allocator returned NULL                       */
    HODLR_CUDA_ERROR = 3,       /* a CUDA runtime call failed                        */
    HODLR_SINGULAR = 4,         /* zero pivot in a leaf block or a Woodbury core     */
    HODLR_NOT_FACTORED = 5,     /* hodlr_solve / gmres_solve before hodlr_factor     */
    HODLR_NOT_CONVERGED = 6,    /* GMRES hit max_iter; X holds the last iterate      */
    HODLR_TIMEOUT = 7,          /* a device-side wait exceeded its budget            */
    HODLR_NONFINITE_INPUT = 8,  /* NaN/Inf (or an FP64 entry outside the range the
                                   double-float matvec represents) in A or B         */
    HODLR_RANGE = 9             /* a size exceeds a fixed limit of the call          */
} hodlr_status;

typedef enum { HODLR_ACA = 0, HODLR_BDLR = 1 } hodlr_method;

/* Arithmetic of the HODLR part (compression is FP64 or FP32, see hodlr_opts).
 * GMRES itself is always FP64-accurate. */
typedef enum {
    HODLR_FP64 = 0,   /* plain FP64 factor and apply                              */
    HODLR_FP32 = 1,   /* FP32 factor and apply                                     */
    HODLR_BF16 = 2,   /* BF16 storage of U, V, d with FP32 accumulation            */
    HODLR_FP16 = 3    /* FP16 storage with a power-of-two scale per column         */
} hodlr_precision;

/* Device allocator callbacks (e.g. a framework's caching allocator).  alloc must
 * return memory usable on `stream` or NULL; free receives the same stream. */
typedef void *(*hodlr_alloc_fn)(size_t bytes, void *user, hodlr_stream stream);
typedef void (*hodlr_free_fn)(void *ptr, size_t bytes, void *user, hodlr_stream stream);

typedef struct hodlr_ctx hodlr_ctx;
typedef struct hodlr_s hodlr_t;

/* A dense FP64 matrix in device memory, row-major, leading dimension ld. */
typedef struct {
    const double *data;   /* device                                                 */
    int64_t n;            /* rows = columns                                         */
    int64_t ld;           /* >= n                                                   */
    int symmetric;        /* 1 if A == A^T exactly: columns are then read as rows
                             (a faster access pattern; values are identical)        */
} hodlr_matrix;

/* The sparse graph whose vertices are the rows/columns of A (Sec. 5.3): CSR in
 * host memory, tree order, no self loops.  Required for BDLR, else NULL. */
typedef struct {
    const int32_t *rowptr;   /* host, n + 1 */
    const int32_t *colind;   /* host, rowptr[n] */
    int64_t n;
} hodlr_graph;

typedef struct {
    int precision;              /* hodlr_precision of factor + apply (default FP32)  */
    int compress_precision;     /* HODLR_FP64 or HODLR_FP32 arithmetic for ACA/BDLR;
                                   -1 = FP64 if precision == FP64, else FP32         */
    int rank_cap;               /* maximum rank of an off-diagonal block (<= 1024);
                                   0 = 1024                                          */
    int bdlr_depth;             /* BDLR distance depth d; -1 = round(-log10 tol) (the
                                   paper's Table 3 pairs); -2 = adaptive (Sec. 5.3):
                                   every block from d = 1, grown while the relative
                                   Frobenius error on the held-out rows and columns
                                   (those at distance d + 1, relative to every row
                                   and column examined) exceeds tol                 */
    double core_cond_threshold; /* Woodbury core condition guard (Sec. 4.3 Factorize,
                                   the cores S_i^(p)): kappa_1(S) = ||S||_1 ||S^-1||_1
                                   of every core is computed exactly from the formed S
                                   and S^-1; with FP32 factor arithmetic (precision
                                   FP32, BF16, FP16) every core above the threshold is
                                   formed again with FP64 products of the stored FP32
                                   factors and inverted in FP64.  0 = tol / 2^-24
                                   (the kappa at which the FP32 inversion error bound
                                   kappa u_32 reaches tol); > 0: that threshold;
                                   < 0: no estimate, no fallback                      */
    const int64_t *leaf_bounds; /* host, optional: 2^L + 1 leaf boundary offsets     */
    int n_leaf_bounds;          /* length of leaf_bounds, or 0                       */
    uint64_t seed;              /* probe seed of hodlr_precond_error                 */
    int defer_factor;           /* 0 (default): hodlr_build also factors, level by level
                                   as the compression of each level completes; 1: only
                                   hodlr_factor factors                               */
} hodlr_opts;

/* Per-call statistics of a built (and possibly factored) HODLR matrix. */
#define HODLR_MAX_LEVELS 16
typedef struct {
    int64_t n;
    int levels;                          /* L: leaves are at level L               */
    int leaf_max;                        /* largest leaf                           */
    int rank_max[HODLR_MAX_LEVELS];      /* max off-diagonal rank at level 1..L (index l-1) */
    int rank_pad[HODLR_MAX_LEVELS];      /* padded rank used for storage           */
    double rank_mean[HODLR_MAX_LEVELS];
    int cap[HODLR_MAX_LEVELS];           /* pivot-list stride of level 1..L       */
    int cap_hit;                        /* 1 if a block stopped at rank_cap       */
    int64_t bytes_factors;               /* device bytes of U, V, d, E, leaf and core factors */
    int factored;
    double ms_compress, ms_factor;       /* device time of the last build / factor */
    /* condition guard, per core level 0..L-1 (the 2^l cores of the parents of
     * level l + 1), zero unless factored with the guard on */
    double core_cond_max[HODLR_MAX_LEVELS];  /* largest kappa_1(S) of the level        */
    int cores_promoted[HODLR_MAX_LEVELS];    /* cores re-inverted in FP64               */
    double core_cond_threshold;              /* the threshold in effect (inf: FP64
                                                arithmetic, never promoted; -1: off)   */
    int bdlr_depth_max;                      /* BDLR: largest depth a block used (0: ACA) */
} hodlr_stats;

/* Per-right-hand-side GMRES results (arrays of length s supplied by the caller,
 * host memory; any pointer may be NULL). */
typedef struct {
    int *iters;                /* Arnoldi steps used                                 */
    double *est_relres;        /* |g_{j+1}| / ||b|| at exit                           */
    double *true_relres;       /* ||b - A x|| / ||b|| recomputed at exit              */
    int restarts;              /* restarts taken (true residual missed tol)          */
    double ms_total;           /* device time of the whole solve                      */
} hodlr_gmres_info;

/* ---------------------------------------------------------------- context */
/* Create a context on CUDA device `device`.  alloc/free may be NULL (then
 * cudaMallocAsync / cudaFreeAsync are used).  *out receives the context. */
hodlr_status hodlr_ctx_create(int device, hodlr_alloc_fn alloc, hodlr_free_fn free_fn,
                              void *alloc_user, hodlr_ctx **out);
hodlr_status hodlr_ctx_destroy(hodlr_ctx *ctx);

/* Default options (precision FP32, compress -1, rank_cap 0, depth -1). */
void hodlr_opts_default(hodlr_opts *o);

/* ---------------------------------------------------------------- HODLR */
/* Compress A into HODLR form (Sec. 4.3 Factorize step 1; Sec. 5.1 / 5.3): every
 * off-diagonal block of every level, A(alpha,beta) ~ U_alpha V_alpha,beta^T, by
 * ACA to relative tolerance `tol` or by BDLR with pivot threshold `tol` and the
 * graph `g`.  `leaf` is the maximum leaf size (>= 1; ignored when leaf_bounds is
 * given).  The result keeps a pointer to A.  Unless opts->defer_factor is set, the
 * factorisation of hodlr_factor is carried out too: each level's share of it is
 * issued as soon as that level (and every deeper one) is compressed, while the
 * compression of the upper levels still runs.  Returns once every level is
 * compressed (the host waits for the ranks); the factorisation completes
 * stream-ordered on `stream`. */
hodlr_status hodlr_build(hodlr_ctx *ctx, const hodlr_matrix *A, int leaf, double tol,
                         int method, const hodlr_graph *g, const hodlr_opts *o,
                         hodlr_stream stream, hodlr_t **out);

/* Recursive Woodbury factorisation (Sec. 4.3 Factorize steps 2-5), level by
 * level from the leaves: leaf inverses, d = K^-1 U for every node, and the core
 * S_i^(p) of every internal node, inverted.  Nothing to do when hodlr_build has
 * factored already (the default).  Stream-ordered, no host sync; a singular leaf
 * or core is reported by the next synchronising call. */
hodlr_status hodlr_factor(hodlr_t *h, hodlr_stream stream);

/* X <- K~^-1 X in place (Sec. 4.3 Solve) for s right-hand sides: X device,
 * n x s column-major, ld >= n.  Arithmetic in the factor's precision, FP64 in
 * and out.  Stream-ordered, no host sync. */
hodlr_status hodlr_solve(hodlr_t *h, int s, double *X, int64_t ldx, hodlr_stream stream);

/* GMRES (Sec. 3) for A X = B with right preconditioner P^-1 = K~^-1 (P may be
 * NULL: no preconditioner).  B, X device, n x s column-major.  Each column is an
 * independent system; x0 = 0.  Flexible right-preconditioned Arnoldi (classical
 * Gram-Schmidt applied twice, Givens rotations, all on the device), stopping
 * when the estimated residual <= tol ||b||; the true residual is then
 * recomputed and the solve restarts from x while it misses tol.  restart = 0
 * means one cycle of up to max_iter steps.  Returns HODLR_NOT_CONVERGED with X
 * = the last iterate if some column misses tol within max_iter steps.  The
 * products with A are those of hodlr_matvec; with s >= 16 (n >= 256) A's digit
 * slices are made once per call.  Synchronises `stream`. */
hodlr_status gmres_solve(hodlr_ctx *ctx, const hodlr_matrix *A, int s, const double *B,
                         int64_t ldb, double *X, int64_t ldx, const hodlr_t *P, double tol,
                         int max_iter, int restart, hodlr_gmres_info *info,
                         hodlr_stream stream);

/* The diagonal (Jacobi) preconditioner P = diag(A), the "Diag" comparison of
 * the paper's Fig. 8 (Sec. 7): a handle without levels, factored on return,
 * that gmres_solve, hodlr_solve (X <- diag(A)^-1 X) and hodlr_precond_error
 * accept in place of a HODLR matrix.  A zero diagonal entry returns
 * HODLR_SINGULAR, a non-finite one HODLR_NONFINITE_INPUT.  The handle keeps a
 * pointer to A.  Synchronises `stream`; release with hodlr_destroy. */
hodlr_status hodlr_build_diag(hodlr_ctx *ctx, const hodlr_matrix *A, hodlr_stream stream, hodlr_t **out);

/* The conventional dense solve of the front, the "LU" comparison of the
 * paper's Table 3 (Sec. 7): LU with row partial pivoting of a copy of A (pivot
 * = the largest |entry| of the column on and below the diagonal, lowest row on
 * ties), right-looking in panels of 64 columns, FP64; then X = U^-1 L^-1 P B
 * for s right-hand sides.  A: device, row-major; B, X: device, n x s
 * column-major (ld >= n; B is not modified).  Allocates 8 n^2 bytes through
 * the context's allocator for the call.  A zero pivot returns HODLR_SINGULAR.
 * Synchronises `stream`. */
hodlr_status hodlr_dense_lu_solve(hodlr_ctx *ctx, const hodlr_matrix *A, int s, const double *B, int64_t ldb,
                                  double *X, int64_t ldx, hodlr_stream stream);

/* ---------------------------------------------------------------- batches */
/* The fronts of one nested-dissection tree solved together (independent
 * problems of uneven sizes; no counterpart call in the paper, which treats one
 * front at a time).  Arrays have nf entries; A[f] is front f (device, FP64),
 * leaf[f] its leaf size, out[f] receives its HODLR matrix.  Every front is
 * compressed with the same tol, method (ACA only: BDLR would need a graph per
 * front) and options.  Synchronises `stream`.  On failure the fronts built so
 * far are destroyed and every out[f] is NULL. */
hodlr_status hodlr_build_batched(hodlr_ctx *ctx, int nf, const hodlr_matrix *A, const int *leaf, double tol,
                                 int method, const hodlr_opts *o, hodlr_stream stream, hodlr_t **out);

/* hodlr_factor of every h[f] (nf entries), stream-ordered. */
hodlr_status hodlr_factor_batched(int nf, hodlr_t *const *h, hodlr_stream stream);

/* gmres_solve for every front f: A[f] X_f = B_f with s[f] right-hand sides,
 * B[f], X[f] device, n_f x s[f] column-major with leading dimensions ldb[f],
 * ldx[f]; P[f] its preconditioner (or NULL, or P itself NULL for none).  info
 * may be NULL or hold nf entries (each with arrays of s[f] entries).  Returns
 * HODLR_NOT_CONVERGED if any front misses tol (all fronts are still solved).
 * Fronts are set up and their first cycles enqueued in windows with one host
 * wait per window, so a front that restarts has an info.ms_total that also spans
 * later fronts' first cycles.  The fronts run on the context's internal streams,
 * after the work already queued on `stream`; all of it is complete when the call
 * returns.  Synchronises `stream`. */
hodlr_status gmres_solve_batched(hodlr_ctx *ctx, int nf, const hodlr_matrix *A, const int *s,
                                 const double *const *B, const int64_t *ldb, double *const *X,
                                 const int64_t *ldx, const hodlr_t *const *P, double tol, int max_iter,
                                 int restart, hodlr_gmres_info *info, hodlr_stream stream);

/* W <- A Z (device, n x s column-major), FP64-accurate, with the products used
 * inside gmres_solve: for s < 16 or n < 256 the double-float product on the FP32
 * pipes (each entry split into FP32 pairs); otherwise every row of A and column
 * of Z is split exactly into seven base-256 digit slices relative to a power of
 * two of its own, the slice products run on the FP16 tensor cores, and the
 * error per term is a few units of 2^-56 max|A(i,:)| max|Z(:,j)| (that path
 * allocates about 7 n^2 bytes for A's digits (one byte each) per call, and falls back to the
 * double-float product when they cannot be allocated).  Synchronises `stream`:
 * a NaN, an infinity or an entry outside the representable range in A or Z
 * returns HODLR_NONFINITE_INPUT (W is then not meaningful). */
hodlr_status hodlr_matvec(hodlr_ctx *ctx, const hodlr_matrix *A, int s, const double *Z,
                          int64_t ldz, double *W, int64_t ldw, hodlr_stream stream);

/* W <- A Z like hodlr_matvec, but without allocating any device memory.
 *
 * There is no counterpart of this call in the paper.  It exists for callers
 * that may not allocate: an application whose memory manager has already
 * claimed all device memory and forbids other allocations, a loop under a
 * fixed memory budget that must not touch the allocator while it runs, or code
 * that cannot pass a context (hodlr_ctx_create allocates).  Such callers pass
 * the inputs and outputs only; the scratch this product needs (the FP32 split
 * of Z) lives in a fixed array inside the library, n * s <= 524288 entries
 * (4 MiB), which every GPU that loads the library holds until the process
 * exits.  Larger sizes return HODLR_RANGE without launching anything.
 *
 * A: device, row-major FP64; Z, W: device, n x s column-major (ld >= n).
 * The first call on a device looks up the array's device address with that
 * device current; make that first call before any stream capture.  All calls
 * share the one array: calls that overlap on the GPU (different streams or
 * host threads at the same time) race and give wrong results.  The call
 * synchronises `stream` (it reads back the non-finite-input flag) and never
 * calls cudaMalloc, cudaFree or an allocating library routine. */
hodlr_status hodlr_matvec_noalloc(const hodlr_matrix *A, int s, const double *Z, int64_t ldz,
                                  double *W, int64_t ldw, hodlr_stream stream);

/* Preconditioner quality ||(I - P^-1 A) Omega||_F / ||Omega||_F for a caller
 * probe block Omega (device, n x k column-major, ld >= n); *out is host.  A is
 * the matrix the HODLR form was built from.  Synchronises `stream`. */
hodlr_status hodlr_precond_error(hodlr_t *h, int k, const double *Omega, int64_t ldo,
                                 double *out, hodlr_stream stream);

hodlr_status hodlr_stats_get(const hodlr_t *h, hodlr_stats *out);

/* Copy one level's factors to host memory, for inspection and testing.
 * level = 1..L.  U, d, V: n x rank_pad[level-1] column-major FP64: the
 * compressed columns U (Sec. 4.3 step 1), d = K_node^-1 U_node (Sec. 4.3
 * step 3; HODLR_NOT_FACTORED before the factorisation) and V; rows of a node
 * beyond its rank are zero.  ranks: 2^level ints.  piv_rows / piv_cols:
 * 2^level x cap[level-1] ints, the block-local pivot rows/columns of each
 * node's block A(node, sibling) in pivot order (ACA: i_k, j_k; BDLR: the kept
 * skeleton rows/columns), -1 past the rank.  Any output may be NULL.
 * Synchronises `stream`. */
hodlr_status hodlr_export_level(const hodlr_t *h, int level, double *U, double *d, double *V,
                                int32_t *ranks, int32_t *piv_rows, int32_t *piv_cols,
                                hodlr_stream stream);

/* Copy the inverted Woodbury cores of level `level` (0..L-1: the parents of
 * level level+1) to host memory: 2^level blocks of (2 rp)^2 FP64, column-major,
 * rp = rank_pad[level].  Block i is S_i^-1 with S_i = [[I, V_ba^T d_a],
 * [V_ab^T d_b, I]] of the node's children a = 2i, b = 2i+1 (Sec. 4.3 step 4).
 * Synchronises `stream`. */
hodlr_status hodlr_export_core(const hodlr_t *h, int level, double *Sinv, hodlr_stream stream);

/* The condition guard's record of the cores of level `level` (0..L-1): kappa_1
 * of each of the 2^level cores (host, may be NULL) and whether it was
 * re-inverted in FP64 (host, may be NULL; 1 = yes).  hodlr_export_core returns
 * the FP64 inverse of such a core.  HODLR_INVALID_ARG when the guard is off.
 * Synchronises `stream`. */
hodlr_status hodlr_export_core_cond(const hodlr_t *h, int level, double *cond, int32_t *promoted,
                                    hodlr_stream stream);

/* Checkpoint of a factored HODLR matrix (or diagonal preconditioner) in host
 * memory: the paper defines no format; the image holds the object's
 * metadata and the contents of its device buffers.  hodlr_save writes the
 * image into buf (host, `bytes` long) and *needed (host) receives its size;
 * with buf NULL only the size is returned.  HODLR_NOT_FACTORED before the
 * factorisation, HODLR_RANGE when bytes < *needed.  Synchronises the device.
 * hodlr_load rebuilds the object on ctx's device from an image of this
 * library version (HODLR_INVALID_ARG for anything else): it holds the same
 * factors bit for bit (saving it again gives the same image), so it applies
 * the same preconditioner up to the apply's own run-to-run rounding (its node
 * sums are atomic); it is factored and keeps a pointer to A (which may be
 * NULL; hodlr_precond_error then refuses).  A restored object is not factored again (hodlr_factor
 * returns at once).  Synchronises `stream`. */
hodlr_status hodlr_save(const hodlr_t *h, void *buf, size_t bytes, size_t *needed, hodlr_stream stream);
hodlr_status hodlr_load(hodlr_ctx *ctx, const hodlr_matrix *A, const void *buf, size_t bytes, hodlr_stream stream,
                        hodlr_t **out);

hodlr_status hodlr_destroy(hodlr_t *h);

const char *hodlr_status_string(hodlr_status s);
const char *hodlr_last_error(void);

/* Diagnostics (no counterpart in the paper): the number of GPU kernels this
 * library has launched in the calling process so far, kernels replayed by a
 * device-side loop of a recorded GMRES iteration included (counted once the
 * solve returns).  `out` is host memory; never fails unless `out` is NULL. */
hodlr_status hodlr_launch_count(long long *out);

/* Per-kernel device time (diagnostics, no counterpart in the paper).  While
 * profiling is on, the library records a CUDA event pair on the launching
 * stream around each launch of its main kernels ("aca_cluster_kernel",
 * "gj_cluster_kernel", "apply_fused_kernel", "df_matvec_kernel",
 * "oz_split_rows_kernel", "oz_split_cols_kernel", "oz_tc_gemm_kernel"),
 * except launches recorded into a graph (the GMRES iterations).
 * hodlr_profile_enable(on) clears the records and switches recording on or
 * off; hodlr_profile_read waits for the recorded launches of `kernel` and
 * returns their total time (ms) and count (host pointers). */
hodlr_status hodlr_profile_enable(int on);
hodlr_status hodlr_profile_read(const char *kernel, double *ms_total, long long *launches);

/* Test hook of the bounded device waits (no counterpart in the paper).  The
 * apply of hodlr_solve and of gmres_solve waits, per tree node, for the arrival
 * of the node's row tiles; every such wait gives up after `spin_limit` polls
 * (0 = the library default, about 2^26 polls of ~32 ns) and then sets the
 * context's status word, which the next synchronising call returns as
 * HODLR_TIMEOUT; the kernel carries on and returns (the results of that call
 * are not meaningful).  With `unreachable` non-zero each wait also expects one
 * tile more than exists, so that every wait runs out: a test of the timeout
 * path that never leaves a kernel waiting without bound.  Reset with (0, 0).
 * Affects later calls on the context (a solve's recorded iteration keeps the
 * values it was recorded with). */
hodlr_status hodlr_ctx_set_wait_test(hodlr_ctx *ctx, unsigned long long spin_limit, int unreachable);

/* How the apply (Sec. 4.3 Solve, in hodlr_solve and every GMRES iteration) is
 * launched; both compute the same result up to the rounding order of the node
 * sums.  1: one cooperative launch for all levels, each CTA walking its row
 * tiles and waiting per node for the tiles of the level below (the waits of
 * hodlr_ctx_set_wait_test); 2: one launch per phase (the leaves, then each
 * level) with one CTA per row tile, the launches ordering the levels; 0
 * (default): 2 when the tiles outnumber twice the CTAs the single launch can
 * hold, else 1.  Affects later calls on the context (a solve's recorded
 * iteration keeps the path it was recorded with).  HODLR_INVALID_ARG for other
 * values. */
hodlr_status hodlr_ctx_set_apply_path(hodlr_ctx *ctx, int path);

#ifdef __cplusplus
}
#endif
#endif /* HODLR_H */
