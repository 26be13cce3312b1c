// Internal declarations of libhodlr (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <deque>
#include <functional>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "hodlr.h"

namespace hodlr {

// ------------------------------------------------------------------ errors
void set_error(const char *fmt, ...);

#define HODLR_TRY_CUDA(call)                                                         \
    do {                                                                             \
        cudaError_t e_ = (call);                                                     \
        if (e_ != cudaSuccess) {                                                     \
            ::hodlr::set_error("%s:%d %s: %s", __FILE__, __LINE__, #call,             \
                               cudaGetErrorString(e_));                              \
            return HODLR_CUDA_ERROR;                                                 \
        }                                                                            \
    } while (0)

#define HODLR_TRY(call)                                                              \
    do {                                                                             \
        hodlr_status s_ = (call);                                                    \
        if (s_ != HODLR_OK) return s_;                                               \
    } while (0)

// Device status word bits (set with atomicOr by kernels, read by synchronising calls).
enum : int {
    ST_SINGULAR = 1,
    ST_NONFINITE = 2,
    ST_TIMEOUT = 4,
    ST_RANGE = 8,
};

hodlr_status status_from_word(int w);

// Process-wide count of the kernels the library launches (hodlr_launch_count).
// While a LaunchCapture lives on the calling thread, launches are being recorded
// into a graph: they are tallied in it instead, and the caller adds them once
// per replay.
void note_launch(long long k = 1);
long long launch_total();
// Per-kernel device time (hodlr_profile_enable): a ProfScope around a launch
// records CUDA events on the launching stream before and after it, unless
// profiling is off or the stream is being captured into a graph.
struct ProfScope {
    const char *name = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr;
    ProfScope(const char *kernel, cudaStream_t stream);
    ~ProfScope();
    ProfScope(const ProfScope &) = delete;
    ProfScope &operator=(const ProfScope &) = delete;
};
struct LaunchCapture {
    long long captured = 0;
    LaunchCapture *prev = nullptr;
    LaunchCapture();
    ~LaunchCapture();
    LaunchCapture(const LaunchCapture &) = delete;
    LaunchCapture &operator=(const LaunchCapture &) = delete;
};

// ------------------------------------------------------------------ context
}  // namespace hodlr

#define HODLR_SIDE_STREAMS 8

// A device block kept by the context after the library released it: reused by
// the next request of the same rounded size (after an event wait when the new
// stream differs from the one it was released on).
struct hodlr_cached_block {
    void *p;
    size_t bytes;
    cudaStream_t stream;
    cudaEvent_t ev;
};

struct hodlr_ctx {
    int device = 0;
    int num_sms = 0;
    cudaStream_t side[HODLR_SIDE_STREAMS] = {};   // forked from the caller's stream per level
    hodlr_alloc_fn alloc = nullptr;
    hodlr_free_fn free_fn = nullptr;
    void *user = nullptr;
    int *d_status = nullptr;      // device status word (one int)
    int *h_status = nullptr;      // pinned mirror
    int *h_scratch = nullptr;     // pinned, 64 ints: small device-to-host reads of the solver
    void *h_report = nullptr;     // pinned, HODLR_REPORT_BYTES: the solver's per-cycle report
    // cache of released device blocks by rounded size (bounded; flushed by
    // hodlr_ctx_destroy); fifo: release order for eviction (entries of blocks
    // handed out again are skipped)
    std::unordered_map<size_t, std::vector<hodlr_cached_block>> cache;
    std::deque<std::pair<void *, size_t>> fifo;
    size_t cache_bytes = 0, cache_count = 0;
    std::vector<cudaEvent_t> spare_events;
    std::mutex cache_mu;
    // executable graphs of finished solves, destroyed by the next solve once
    // it has work queued (their teardown is host time) or by hodlr_ctx_destroy
    std::vector<std::pair<cudaGraphExec_t, cudaGraph_t>> graph_trash;
    // the apply's wait budget (polls; 0 = the library default) and an addition
    // to its arrival targets, set by hodlr_ctx_set_wait_test only
    unsigned long long wait_limit = 0;
    unsigned wait_extra = 0;
    int apply_path = 0;   // 0: automatic, 1: one cooperative launch, 2: one launch per phase
};
#define HODLR_REPORT_BYTES 65536
#define HODLR_CACHE_LIMIT (size_t(16) << 30)

namespace hodlr {

void *dalloc(hodlr_ctx *c, size_t bytes, cudaStream_t s);
void dfree(hodlr_ctx *c, void *p, size_t bytes, cudaStream_t s);

// RAII-less device buffer bookkeeping: every hodlr_t remembers what it owns.
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

// Read and clear the context's device status word (synchronises the stream).
hodlr_status take_status(hodlr_ctx *c, cudaStream_t s);
// The status (and error message) of a device status word already read.
hodlr_status status_word(int w);

// ------------------------------------------------------------------ tree
// Level l (1..L) of the tree holds 2^l nodes; node i covers leaves
// [i << (L-l), (i+1) << (L-l)).  Off-diagonal factors of level l belong to the
// nodes of level l: U rows = the node's rows, paired with V rows = the
// sibling's rows (A(node, sibling) ~ U_node V_sibling^T).
struct Level {
    int nnodes = 0;
    int rp = 0;               // padded rank (columns of this level's U, d and V)
    int64_t coff = 0;         // sum of rp over the levels above (storage accounting)
    int cap = 0;              // staging columns for compression
    std::vector<int> ranks;   // per node
    int rank_max = 0;
    double rank_mean = 0.0;
};

struct FactorPlan;   // factor.cu

}  // namespace hodlr

struct hodlr_s {
    hodlr_ctx *ctx = nullptr;
    const double *A = nullptr;
    int64_t n = 0, lda = 0;
    int sym = 0;
    int L = 0;
    int bmax = 0;                     // largest leaf
    std::vector<int64_t> bounds;      // 2^L + 1 leaf boundaries
    int64_t *d_bounds = nullptr;
    int prec = HODLR_FP32;            // factorisation arithmetic (FP64 or FP32)
    int store = HODLR_FP32;           // storage of the streamed factors V, d in the apply
    std::vector<float *> vscale, escale; // FP16: per level 0..L, [nnodes * rp] (V) and [nnodes * 2 rp] (E) dequantisation factors
    int cprec = HODLR_FP32;           // compression precision
    int method = HODLR_ACA;
    double tol = 0.0;
    int rank_cap = 1024;
    int cap_hit = 0;
    int bdlr_depth_max = 0;           // BDLR: the largest distance depth a block used
    std::vector<hodlr::Level> lv;     // index 1..L used
    int64_t ldn = 0;                  // leading dimension of U, D, V (n rounded up to 32)
    int64_t Wtot = 0;                 // sum of rp over the levels
    // Per level c = 1..L (index 0 unused), each ldn x rp(c) column-major:
    std::vector<void *> Ul;           // the compressed U columns (kept: re-factorable)
    std::vector<void *> Dl;           // d = K_node^-1 U_node after factorisation
    std::vector<void *> El;           // ldn x 2 rp(c): E = d S^-1(half of the parent's core), the apply's update
    std::vector<void *> Vl;           // rows of node nu: V of the sibling's block
    std::vector<void *> Vql, Eql;     // 16-bit copies of V and E (BF16 / FP16 storage)
    void *leafinv = nullptr;          // elem[2^L * bmax * bmax], column-major per leaf
    std::vector<void *> Sinv;         // level l = 0..L-1: elem[2^l * (2 rp(l+1))^2]
    std::vector<int32_t *> piv_rows;  // per level 1..L: [nnodes][cap] pivot rows (ACA) / kept rows (BDLR)
    std::vector<int32_t *> piv_cols;
    std::vector<int32_t *> d_ranks;   // per level 1..L: [nnodes]
    bool factored = false;
    double ms_compress = 0, ms_factor = 0;
    std::vector<hodlr::DevBuf> owned;
    // scratch of the apply
    void *work = nullptr;
    size_t work_bytes = 0;
    // fused apply: 32-row tiles of the leaves (leaf, first row, rows, 0) and the
    // first tile of every leaf (2^L + 1 entries)
    const int4 *d_tiles = nullptr;
    int ntiles = 0;
    int *d_tile_first = nullptr;
    // the recorded factorisation (workspace, descriptors, launches)
    hodlr::FactorPlan *plan = nullptr;
    // events around the last factorisation, read lazily by hodlr_stats_get
    cudaEvent_t fev[2] = {nullptr, nullptr};
    // Woodbury core condition guard (level l = 0..L-1: the 2^l cores of the
    // parents of level l + 1): kappa_1(S) of every core, the flag of the cores
    // re-inverted in FP64, and their FP64 inverses (FP32 arithmetic only)
    // the diagonal (Jacobi) preconditioner of the paper's comparison: no levels,
    // the apply is X <- diag(A)^-1 X (baselines.cu)
    bool diag = false;
    double *dinv = nullptr;
    bool guard = false;                // kappa_1 is computed
    bool promote = false;              // cores above cond_thr are re-inverted in FP64
    double cond_thr = 0.0;
    std::vector<double *> core_cond;
    std::vector<int *> core_flag;
    std::vector<unsigned *> core_count;   // per level: the condition kernel's completion counter (self-resetting)
    std::vector<double *> Sinv64;
};

namespace hodlr {

inline size_t elem_size(int prec) { return prec == HODLR_FP64 ? 8 : 4; }

void *own(hodlr_t *h, size_t bytes, cudaStream_t s);   // allocate and remember

// Offsets of the pieces of one allocation (256-byte aligned): every allocation
// goes through the caller's allocator, so related buffers share one.
struct Arena {
    size_t bytes = 0;
    size_t take(size_t b);
};
hodlr_status ensure_work(hodlr_t *h, size_t bytes, cudaStream_t s);

// ------------------------------------------------------------------ kernels (launchers)
// Compression
struct AcaBlockDesc {
    int64_t r0, m;      // block rows  [r0, r0+m)
    int64_t c0, nc;     // block cols  [c0, c0+nc)
    int64_t ld;         // leading dimension of the U/V staging (column-major)
    void *U;            // staging of the row side  (element type = compression precision)
    void *V;            // staging of the column side
    int cap;            // columns available
    int32_t *rank;      // out
    int32_t *prow;      // out: pivot rows (block-local), cap entries
    int32_t *pcol;      // out: pivot cols (block-local)
    int32_t *cap_hit;   // out
};
// Partial-pivoting ACA, one thread-block cluster per block, one launch per level on the context's side
// streams (forked from s; level l + 1 on side[l mod HODLR_SIDE_STREAMS]).  level_first: first block of
// each level in d_blocks (size nlev + 1); level_maxdim: largest block side per level.
// done[l] (created here, destroyed by the caller) completes with level l + 1's
// compression; s itself does not wait for the levels.  after_first, if set, is
// called once the first level is launched (work issued there is dispatched
// before the other levels' CTAs); its error ends the launch.
hodlr_status launch_aca_levels(hodlr_ctx *c, const double *A, int64_t lda, int sym, int cprec,
                               const AcaBlockDesc *d_blocks, const std::vector<int> &level_first,
                               const std::vector<int64_t> &level_maxdim, double tol, cudaStream_t s,
                               std::vector<cudaEvent_t> &done,
                               const std::function<hodlr_status()> &after_first = {});

struct BdlrHost;   // defined in bdlr.cu
hodlr_status run_bdlr(hodlr_t *h, const hodlr_graph *g, int depth, cudaStream_t s,
                      std::vector<void *> &Ust, std::vector<void *> &Vst);

// Generic batched GEMM:  C_b += alpha * op(A_b) * B_b  (column-major), op = N or T.
// The operands may be stored in a narrower type TI than the accumulation type
// T (FP32 factors multiplied in FP64).  gate (device, optional): the product is
// skipped when *gate == 0, so that work whose need is only known on the device
// can be enqueued without a host round trip.
template <typename T, typename TI = T>
struct GemmDesc {
    const TI *A;
    const TI *B;
    T *C;
    int64_t lda, ldb, ldc;
    int M, N, K;
    const int *gate;
};
template <typename T, typename TI = T>
hodlr_status gemm_batched(hodlr_ctx *c, const GemmDesc<T, TI> *d_desc, int nbatch, int maxM,
                          int maxN, int maxK, int transA, T alpha, cudaStream_t s);

hodlr_status factor_impl(hodlr_t *h, cudaStream_t s);
// Record level c's share of the factorisation (its d columns through every
// deeper level's update, then the cores of level c - 1) and upload its
// descriptors; levels are recorded from c = L down to 1.  run_level issues the
// recorded launches of level c on s; factor_impl replays every level.  With
// share_done (indexed by level), s waits for share_done[l] where level c's
// share starts reading level l's factors, so that the shares of different
// levels can run on different streams.
hodlr_status plan_level(hodlr_t *h, int c, cudaStream_t s);
hodlr_status run_level(hodlr_t *h, int c, cudaStream_t s, const cudaEvent_t *share_done);
// Explicit inverses of the leaf blocks of A (stream-ordered; h->leafinv allocated).
hodlr_status leaf_inverses(hodlr_t *h, cudaStream_t s);
void free_plan(hodlr_t *h, cudaStream_t s);
// Xs (optional): also store the result as FP32 (hi, lo) pairs (ld ldx), the
// split the product reads.
hodlr_status solve_impl(const hodlr_t *h, int s_rhs, double *X, int64_t ldx, cudaStream_t s, float2 *Xs = nullptr);
hodlr_status solve_prepare(const hodlr_t *h, int s_rhs, cudaStream_t s);
hodlr_status diag_solve(const hodlr_t *h, int s_rhs, double *X, int64_t ldx, cudaStream_t s, float2 *Xs);
// Asp / split_state: optional n x n buffer of A's FP32 (hi, lo) pairs, written by
// the first product while *split_state is 0 and read by later ones.
// z_split: work already holds the FP32 split of Z (ld n), written by the apply;
// z_fp32: every entry of Z is exactly an FP32 value (zero low parts).
hodlr_status matvec_impl(hodlr_ctx *c, const double *A, int64_t n, int64_t lda, int s_rhs,
                         const double *Z, int64_t ldz, double *W, int64_t ldw, cudaStream_t s,
                         void *work = nullptr, bool w_zeroed = false, float2 *Asp = nullptr,
                         const int *split_state = nullptr, bool z_split = false, bool z_fp32 = false);

// FP64-accurate product on the FP16 tensor cores for many right-hand sides
// (ozaki.cu): A's rows and Z's columns split exactly into OZ_SLICES base-256
// digit slices.  oz_split_a writes A's slices into abuf (oz_a_bytes(n) bytes,
// once per A); oz_matvec splits Z into zbuf (oz_z_bytes(n, s) bytes) and
// writes W = A Z (every entry; W need not be zeroed).  Used where
// oz_eligible(n, s).
constexpr int OZ_SLICES = 7;
constexpr int OZ_MIN_RHS = 16;
constexpr int64_t OZ_MIN_N = 256;
bool oz_eligible(int64_t n, int s_rhs);
size_t oz_a_bytes(int64_t n);
size_t oz_z_bytes(int64_t n, int s_rhs);
hodlr_status oz_split_a(hodlr_ctx *c, const double *A, int64_t n, int64_t lda, void *abuf, cudaStream_t s);
hodlr_status oz_matvec(hodlr_ctx *c, const void *abuf, int64_t n, int s_rhs, const double *Z, int64_t ldz,
                       double *W, int64_t ldw, void *zbuf, cudaStream_t s);

// Convert / pad kernels
hodlr_status copy_columns(int prec_src, int prec_dst, const void *src, int64_t ld_src,
                          void *dst, int64_t ld_dst, int64_t rows, int64_t cols,
                          cudaStream_t s);

}  // namespace hodlr

// ------------------------------------------------------------------ device helpers
namespace hodlr {
namespace dev {

// Exact-rounding multiply and subtract with no contraction into an FMA, so that a
// residual formed term by term rounds exactly like the reference formulation.
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double div_rn(double a, double b) { return __ddiv_rn(a, b); }
__device__ __forceinline__ float div_rn(float a, float b) { return __fdiv_rn(a, b); }

template <typename T>
__device__ __forceinline__ T from_double(double x);
template <>
__device__ __forceinline__ double from_double<double>(double x) { return x; }
template <>
__device__ __forceinline__ float from_double<float>(double x) { return __double2float_rn(x); }

}  // namespace dev
}  // namespace hodlr
