// Recursive Woodbury factorisation of a HODLR matrix, level by level from the
// leaves (Sec. 4.3, Factorize steps 2-5; Sec. 4.2 eqs. Schur and y).
//
// Layout: per level c, U_c, d_c and V_c are ldn x rp(c) column-major.  Row
// block "node" of U_c holds U_node (the Z stack of the paper, one level at a
// time); after factorisation d_c(node rows) = K_node^-1 U_node.
//
// The share of level c, issued as soon as level c is compressed (on that
// level's stream; step 2 for level l waits for the share of level l + 1):
//  1. d_c <- K_leaf^-1 U_c on every leaf                            (explicit inverses)
//  2. for l = L-1 .. c (parents of level l + 1, deepest first):
//       Y = [V_ba^T d_c(alpha); V_ab^T d_c(beta)],  [y1; y2] = S_l^-1 Y,
//       d_c(alpha) -= d_alpha y2,  d_c(beta) -= d_beta y1      (d_alpha: final d of level l+1)
//  3. the cores of level c - 1: P = V_ba^T d_alpha, Q = V_ab^T d_beta (now final),
//       S = [[I, P], [Q, I]],  M = I - P Q,
//       S^-1 = [[M^-1, -M^-1 P], [-Q M^-1, I + Q M^-1 P]]
//  4. the apply's update E_alpha = d_alpha S^-1(rows rp..2rp-1, :),
//       E_beta = d_beta S^-1(rows 0..rp-1, :)   (x_alpha -= d_alpha y2 = E_alpha w)
// Summed over c this is the level-synchronous sweep of the paper's recursion:
// each d column receives the updates of the deeper levels in the same order.
// The 2x2 block inverse through M = I - P Q is the same algebra as solving with
// S; it halves the size of the dense inversion.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <climits>
#include <cstring>
#include <functional>

#include "internal.cuh"

namespace hodlr {
namespace {

// ------------------------------------------------------------------ batched GEMM
// C_b += alpha op(A_b) B_b on BM x BM output tiles (BM = 64 or 32) with 16-deep
// K slices; 256 threads as 16 x 16, each owning (BM/16)^2 outputs.  The next K
// slice is loaded into registers while the current one is multiplied from
// shared memory.  splitK > 1 splits K into that many chunks (multiples of 16)
// whose partial products are combined with atomics.  Operands of type TI are
// widened to T as they are loaded; a descriptor whose gate reads 0 is skipped.
constexpr int GB_K = 16, GB_THREADS = 256;

template <typename T, typename TI, int BM>
__global__ void __launch_bounds__(GB_THREADS)
    gemm_batched_kernel(const GemmDesc<T, TI> *__restrict__ descs, int transA, T alpha, int splitK) {
    constexpr int TPT = BM / 16;                 // outputs per thread per dimension
    constexpr int LPT = BM * GB_K / GB_THREADS;  // tile elements loaded per thread
    const GemmDesc<T, TI> d = descs[blockIdx.z / splitK];
    const int kz = blockIdx.z % splitK;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BM;
    if (m0 >= d.M || n0 >= d.N || d.K <= 0) return;
    if (d.gate && *d.gate == 0) return;
    const int kper = ((d.K + splitK - 1) / splitK + GB_K - 1) / GB_K * GB_K;
    const int kbeg = kz * kper;
    const int kend = min(d.K, kbeg + kper);
    if (kbeg >= kend) return;
    __shared__ T As[GB_K][BM + 1];
    __shared__ T Bs[GB_K][BM + 1];
    const int tid = threadIdx.x;
    const int ty = tid & 15, tx = tid >> 4;
    T ra[LPT], rb[LPT];
    auto load = [&](int k0) {
#pragma unroll
        for (int u = 0; u < LPT; ++u) {
            const int e = tid + u * GB_THREADS;
            int i, kk;
            if (!transA) {
                i = e % BM;
                kk = e / BM;
            } else {
                kk = e % GB_K;
                i = e / GB_K;
            }
            T v = T(0);
            if (m0 + i < d.M && k0 + kk < kend)
                v = (T)(transA ? d.A[(int64_t)(k0 + kk) + (int64_t)(m0 + i) * d.lda]
                               : d.A[(int64_t)(m0 + i) + (int64_t)(k0 + kk) * d.lda]);
            ra[u] = v;
            const int kb = e % GB_K, j = e / GB_K;
            T w = T(0);
            if (n0 + j < d.N && k0 + kb < kend) w = (T)d.B[(int64_t)(k0 + kb) + (int64_t)(n0 + j) * d.ldb];
            rb[u] = w;
        }
    };
    auto store = [&]() {
#pragma unroll
        for (int u = 0; u < LPT; ++u) {
            const int e = tid + u * GB_THREADS;
            if (!transA)
                As[e / BM][e % BM] = ra[u];
            else
                As[e % GB_K][e / GB_K] = ra[u];
            Bs[e % GB_K][e / GB_K] = rb[u];
        }
    };
    T acc[TPT][TPT];
#pragma unroll
    for (int a = 0; a < TPT; ++a)
#pragma unroll
        for (int b = 0; b < TPT; ++b) acc[a][b] = T(0);
    load(kbeg);
    for (int k0 = kbeg; k0 < kend; k0 += GB_K) {
        store();
        __syncthreads();
        if (k0 + GB_K < kend) load(k0 + GB_K);
#pragma unroll
        for (int kk = 0; kk < GB_K; ++kk) {
            T a[TPT], b[TPT];
#pragma unroll
            for (int q = 0; q < TPT; ++q) {
                a[q] = As[kk][ty + 16 * q];
                b[q] = Bs[kk][tx + 16 * q];
            }
#pragma unroll
            for (int p = 0; p < TPT; ++p)
#pragma unroll
                for (int q = 0; q < TPT; ++q) acc[p][q] = fma(a[p], b[q], acc[p][q]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < TPT; ++q) {
        const int j = n0 + tx + 16 * q;
        if (j >= d.N) continue;
#pragma unroll
        for (int p = 0; p < TPT; ++p) {
            const int i = m0 + ty + 16 * p;
            if (i >= d.M) continue;
            T *cp = d.C + (int64_t)i + (int64_t)j * d.ldc;
            if (splitK == 1)
                *cp += alpha * acc[p][q];
            else
                atomicAdd(cp, alpha * acc[p][q]);
        }
    }
}

// ------------------------------------------------------------------ Gauss-Jordan inverse
// In-place Gauss-Jordan with row partial pivoting on an augmented b x 2b
// column-major work matrix [M | I] (ld = b): pivot = argmax_{i>=k} |W(i,k)|
// (lowest row on ties), swap, scale the pivot row, eliminate every other row.
// The right half ends as M^-1 and is copied to `out` (ld_out).  One CTA per matrix.
template <typename T>
struct GJDesc {
    const double *srcA;   // if non-null: M = A(r0:r0+b, r0:r0+b) (row-major FP64, lda)
    int64_t lda;
    const T *srcM;        // else: M (column-major, ldm)
    int64_t ldm;
    T *work;              // b * 2b
    T *out;               // b x b column-major
    int64_t ldo;
    int b;
    const int *gate;      // device, optional: the matrix is skipped when *gate == 0
};

constexpr int GJ_THREADS = 512;

template <typename T>
__global__ void __launch_bounds__(GJ_THREADS) gj_inverse_kernel(const GJDesc<T> *__restrict__ descs,
                                                                int *status) {
    const GJDesc<T> g = descs[blockIdx.x];
    const int b = g.b, tid = threadIdx.x;
    if (b <= 0 || (g.gate && *g.gate == 0)) return;
    if (g.work == nullptr) {   // host-side sizing error: report, never touch memory
        if (tid == 0) atomicOr(status, ST_RANGE);
        return;
    }
    T *W = g.work;
    extern __shared__ __align__(16) unsigned char smem[];
    T *s_col = reinterpret_cast<T *>(smem);   // b
    T *s_row = s_col + b;                     // 2b
    __shared__ T red_v[GJ_THREADS / 32];
    __shared__ int red_i[GJ_THREADS / 32];
    __shared__ int s_fail;
    const int64_t bb = (int64_t)b * b;
    for (int64_t e = tid; e < 2 * bb; e += GJ_THREADS) {
        const int64_t j = e / b, i = e % b;
        T v;
        if (j < b)
            v = g.srcA ? dev::from_double<T>(g.srcA[i * g.lda + j]) : g.srcM[i + j * g.ldm];
        else
            v = (j - b == i) ? T(1) : T(0);
        W[e] = v;
    }
    if (tid == 0) s_fail = 0;
    __syncthreads();
    const int lane = tid & 31, warp = tid >> 5;
    for (int k = 0; k < b; ++k) {
        T bv = T(-1);
        int bi = INT_MAX;
        for (int i = k + tid; i < b; i += GJ_THREADS) {
            T a = fabs(W[i + (int64_t)k * b]);
            if (a > bv) {
                bv = a;
                bi = i;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            T ov = __shfl_down_sync(0xffffffffu, bv, o);
            int oi = __shfl_down_sync(0xffffffffu, bi, o);
            if (ov > bv || (ov == bv && oi < bi)) {
                bv = ov;
                bi = oi;
            }
        }
        if (lane == 0) {
            red_v[warp] = bv;
            red_i[warp] = bi;
        }
        __syncthreads();
        if (tid == 0) {
            for (int w = 1; w < GJ_THREADS / 32; ++w)
                if (red_v[w] > red_v[0] || (red_v[w] == red_v[0] && red_i[w] < red_i[0])) {
                    red_v[0] = red_v[w];
                    red_i[0] = red_i[w];
                }
            if (!(red_v[0] > T(0))) s_fail = 1;
        }
        __syncthreads();
        if (s_fail) break;
        const int p = red_i[0];
        if (p != k)
            for (int j = tid; j < 2 * b; j += GJ_THREADS) {
                T t = W[k + (int64_t)j * b];
                W[k + (int64_t)j * b] = W[p + (int64_t)j * b];
                W[p + (int64_t)j * b] = t;
            }
        __syncthreads();
        const T piv = W[k + (int64_t)k * b];
        for (int j = tid; j < 2 * b; j += GJ_THREADS) {
            T v = W[k + (int64_t)j * b] / piv;
            W[k + (int64_t)j * b] = v;
            s_row[j] = v;
        }
        for (int i = tid; i < b; i += GJ_THREADS) s_col[i] = (i == k) ? T(0) : W[i + (int64_t)k * b];
        __syncthreads();
        for (int64_t e = tid; e < 2 * bb; e += GJ_THREADS) {
            const int j = (int)(e / b), i = (int)(e % b);
            if (i != k) W[e] = W[e] - s_col[i] * s_row[j];
        }
        __syncthreads();
    }
    if (s_fail) {
        if (tid == 0) atomicOr(status, ST_SINGULAR);
        return;
    }
    for (int64_t e = tid; e < bb; e += GJ_THREADS) {
        const int64_t j = e / b, i = e % b;
        g.out[i + j * g.ldo] = W[bb + e];
    }
}

// Fill of the factorisation's workspace before a sweep: block m of a task is the
// rows x cols column-major array at p + m stride (ld), set to 1 on the diagonal
// from row d0 on and to 0 elsewhere.  One launch serves every task (blockIdx.y).
template <typename T>
struct FillDesc {
    T *p;
    int64_t ld;
    int64_t rows, cols;
    int d0;
    int count;
    int64_t stride;
};

template <typename T>
__global__ void fill_kernel(const FillDesc<T> *__restrict__ tasks) {
    const FillDesc<T> f = tasks[blockIdx.y];
    const int64_t per = f.rows * f.cols, total = per * f.count;
    const int64_t ld = f.ld > 0 ? f.ld : f.rows;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t m = e / per, r = e % per;
        const int64_t j = r / f.rows, i = r % f.rows;
        f.p[m * f.stride + i + j * ld] = (i == j && i >= f.d0) ? T(1) : T(0);
    }
}

// Gauss-Jordan inversion in place in shared memory (ld = b + 1, conflict-free
// row and column access), same pivot rule as above (argmax_{i>=k} |a(i,k)|,
// lowest row on ties).  Step k: swap rows k and p, d = 1/a(k,k), scale row k,
// eliminate column k from every other row, storing -a(i,k) d in column k.  The
// result is (PA)^-1; A^-1 = (PA)^-1 P, i.e. column j of A^-1 is column pos(j) of
// the work matrix, pos(j) = final position of the original row j.
constexpr int GJS_THREADS = 512;

template <typename T>
__global__ void __launch_bounds__(GJS_THREADS) gj_inverse_smem_kernel(const GJDesc<T> *__restrict__ descs,
                                                                      int *status) {
    const GJDesc<T> g = descs[blockIdx.x];
    const int b = g.b, tid = threadIdx.x;
    if (b <= 0 || (g.gate && *g.gate == 0)) return;
    const int ldb = b + 1;
    extern __shared__ __align__(16) unsigned char smem[];
    T *a = reinterpret_cast<T *>(smem);            // ldb * b
    T *rowk = a + (size_t)ldb * b;                 // b
    T *colk = rowk + b;                            // b
    int *orig = reinterpret_cast<int *>(colk + b); // b: original row at each position
    __shared__ int s_p, s_fail;
    for (int e = tid; e < b * b; e += GJS_THREADS) {
        const int j = e / b, i = e % b;
        a[i + j * ldb] = g.srcA ? dev::from_double<T>(g.srcA[(int64_t)i * g.lda + j]) : g.srcM[i + (int64_t)j * g.ldm];
    }
    for (int i = tid; i < b; i += GJS_THREADS) orig[i] = i;
    if (tid == 0) s_fail = 0;
    __syncthreads();
    const int lane = tid & 31, warp = tid >> 5;
    for (int k = 0; k < b; ++k) {
        if (warp == 0) {
            T bv = T(-1);
            int bi = INT_MAX;
            for (int i = k + lane; i < b; i += 32) {
                const T v = fabs(a[i + k * ldb]);
                if (v > bv) {
                    bv = v;
                    bi = i;
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const T ov = __shfl_down_sync(0xffffffffu, bv, o);
                const int oi = __shfl_down_sync(0xffffffffu, bi, o);
                if (ov > bv || (ov == bv && oi < bi)) {
                    bv = ov;
                    bi = oi;
                }
            }
            if (lane == 0) {
                s_p = bi;
                if (!(bv > T(0))) s_fail = 1;
                else if (bi != k) {
                    const int t = orig[k];
                    orig[k] = orig[bi];
                    orig[bi] = t;
                }
            }
        }
        __syncthreads();
        if (s_fail) break;
        const int p = s_p;
        if (p != k)
            for (int j = tid; j < b; j += GJS_THREADS) {
                const T t = a[k + j * ldb];
                a[k + j * ldb] = a[p + j * ldb];
                a[p + j * ldb] = t;
            }
        __syncthreads();
        const T d = T(1) / a[k + k * ldb];
        for (int j = tid; j < b; j += GJS_THREADS) rowk[j] = (j == k) ? d : a[k + j * ldb] * d;
        for (int i = tid; i < b; i += GJS_THREADS) colk[i] = (i == k) ? T(0) : a[i + k * ldb];
        __syncthreads();
        for (int e = tid; e < b * b; e += GJS_THREADS) {
            const int j = e / b, i = e % b;
            T v;
            if (i == k)
                v = rowk[j];
            else if (j == k)
                v = -colk[i] * d;
            else
                v = a[i + j * ldb] - colk[i] * rowk[j];
            a[i + j * ldb] = v;
        }
        __syncthreads();
    }
    if (s_fail) {
        if (tid == 0) atomicOr(status, ST_SINGULAR);
        return;
    }
    // pos(orig[q]) = q
    for (int q = tid; q < b; q += GJS_THREADS) colk[orig[q]] = (T)q;
    __syncthreads();
    for (int e = tid; e < b * b; e += GJS_THREADS) {
        const int j = e / b, i = e % b;
        const int pj = (int)colk[j];
        g.out[i + (int64_t)j * g.ldo] = a[i + pj * ldb];
    }
}

constexpr size_t GJS_SMEM_MAX = 200 * 1024;

// Gauss-Jordan inversion with the matrix held in registers: 256 threads as an
// 8 x 32 grid, thread (ty, tx) owns rows ty + 8 p (p < MR) and columns
// tx + 32 q (q < MC).  Pivoting is implicit (no row exchanges): step k sweeps
// the pivot (p_k, k), p_k = argmax |a(i, k)| over the rows not yet used as
// pivots (lowest row on ties):
//   a(i, j) -= a(i, k) a(p_k, j) / a(p_k, k)   (i != p_k, j != k)
//   a(i, k)  = -a(i, k) / a(p_k, k),  a(p_k, j) = a(p_k, j) / a(p_k, k),
//   a(p_k, k) = 1 / a(p_k, k).
// After the b sweeps the table maps outputs to inputs, M^-1(k, p_j) =
// a(p_k, j).  The steps run as MC unrolled blocks of 32, so the register slot of
// column k is a compile-time index.  A step costs two CTA barriers: one after
// the column owners post their candidate pivots (merged by a shuffle argmax in
// every warp), one after the pivot row's owner posts that row, with the pivot
// entries of the posted row and column adjusted so that a single FMA per
// element performs all four cases of the sweep.  The pivot column and row
// buffers are double-buffered by step parity.
constexpr int GJR_TY = 8, GJR_TX = 32, GJR_THREADS = GJR_TY * GJR_TX;

template <typename T, int MR, int MC>
__global__ void __launch_bounds__(GJR_THREADS, 1) gj_inverse_reg_kernel(const GJDesc<T> *__restrict__ descs,
                                                                       int *status) {
    const GJDesc<T> g = descs[blockIdx.x];
    const int b = g.b;
    if (b <= 0) return;
    if constexpr (sizeof(T) == 8) {   // only the FP64 re-inversion of the guarded cores is gated
        if (g.gate && *g.gate == 0) return;
    }
    const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
    __shared__ T colk[2][MR * GJR_TY];
    __shared__ T rowk[2][MC * GJR_TX];
    __shared__ T cand_v[2][GJR_TY];
    __shared__ int cand_i[2][GJR_TY];
    __shared__ int prow[MR * GJR_TY];   // pivot row of step k
    __shared__ int krow[MR * GJR_TY];   // step at which row i was the pivot
    T a[MR][MC];
    unsigned long long used = 0;        // bit p: row ty + 8 p is a pivot already (or beyond b)
#pragma unroll
    for (int p = 0; p < MR; ++p) {
        const int i = ty + GJR_TY * p;
        if (i >= b) used |= 1ull << p;
#pragma unroll
        for (int q = 0; q < MC; ++q) {
            const int j = tx + GJR_TX * q;
            T v = T(0);
            if (i < b && j < b)
                v = g.srcA ? dev::from_double<T>(g.srcA[(int64_t)i * g.lda + j]) : g.srcM[i + (int64_t)j * g.ldm];
            a[p][q] = v;
        }
    }
    bool fail = false;
#pragma unroll
    for (int kq = 0; kq < MC; ++kq) {
        const int kxe = min(GJR_TX, b - kq * GJR_TX);
        for (int kx = 0; kx < kxe && !fail; ++kx) {
            const int k = kq * GJR_TX + kx;
            const int par = k & 1;
            // A. the owners of column k post it and their best unused row
            if (tx == kx) {
                T bv = T(-1), sv = T(0);
                int bi = INT_MAX;
#pragma unroll
                for (int p = 0; p < MR; ++p) {
                    const T v = a[p][kq];
                    colk[par][ty + GJR_TY * p] = v;
                    const T av = fabs(v);
                    if (!((used >> p) & 1ull) && av > bv) {
                        bv = av;
                        sv = v;
                        bi = ty + GJR_TY * p;
                    }
                }
                cand_v[par][ty] = sv;
                cand_i[par][ty] = bi;
            }
            __syncthreads();
            // B. every warp merges the candidates with a shuffle argmax (same result everywhere)
            T pa = T(-1), piv = T(0);
            int pr = INT_MAX;
            if (tx < GJR_TY) {
                pr = cand_i[par][tx];
                piv = cand_v[par][tx];
                pa = pr == INT_MAX ? T(-1) : fabs(piv);
            }
#pragma unroll
            for (int o = GJR_TY / 2; o > 0; o >>= 1) {
                const T oa = __shfl_xor_sync(0xffffffffu, pa, o);
                const T ov = __shfl_xor_sync(0xffffffffu, piv, o);
                const int oi = __shfl_xor_sync(0xffffffffu, pr, o);
                if (oa > pa || (oa == pa && oi < pr)) {
                    pa = oa;
                    piv = ov;
                    pr = oi;
                }
            }
            pa = __shfl_sync(0xffffffffu, pa, 0);
            piv = __shfl_sync(0xffffffffu, piv, 0);
            pr = __shfl_sync(0xffffffffu, pr, 0);
            if (!(pa > T(0))) {   // uniform: no usable pivot in column k
                fail = true;
                break;
            }
            const int py = pr % GJR_TY, pp = pr / GJR_TY;
            // the pivot row as it is before the sweep (p = a(pr, k))
            if (ty == py) {
#pragma unroll
                for (int p = 0; p < MR; ++p)
                    if (p == pp) {
                        used |= 1ull << p;
#pragma unroll
                        for (int q = 0; q < MC; ++q) rowk[par][tx + GJR_TX * q] = a[p][q];
                    }
            }
            if (tid == 0) {
                prow[k] = pr;
                krow[pr] = k;
            }
            __syncthreads();
            // C. sweep the pivot (pr, k): a(i, j) -= a(i, k) a(pr, j) / p on
            // every element, then the pivot row becomes a(pr, j) / p, the pivot
            // column -a(i, k) / p and the pivot 1 / p (scale-invariant: no step
            // loses digits to the size of p)
            const T d = T(1) / piv;
            T rk[MC];
#pragma unroll
            for (int q = 0; q < MC; ++q) rk[q] = rowk[par][tx + GJR_TX * q];
#pragma unroll
            for (int p = 0; p < MR; ++p) {
                const T f = colk[par][ty + GJR_TY * p] * d;
#pragma unroll
                for (int q = 0; q < MC; ++q) a[p][q] = fma(-f, rk[q], a[p][q]);
                if (tx == kx) a[p][kq] = -f;   // the pivot column
            }
            if (ty == py) {
#pragma unroll
                for (int p = 0; p < MR; ++p)
                    if (p == pp) {
#pragma unroll
                        for (int q = 0; q < MC; ++q) a[p][q] = rk[q] * d;
                        if (tx == kx) a[p][kq] = d;
                    }
            }
        }
    }
    if (fail) {
        if (tid == 0) atomicOr(status, ST_SINGULAR);
        return;
    }
    __syncthreads();
    // M^-1(krow[i], prow[j]) = a(i, j)
#pragma unroll
    for (int p = 0; p < MR; ++p)
#pragma unroll
        for (int q = 0; q < MC; ++q) {
            const int i = ty + GJR_TY * p, j = tx + GJR_TX * q;
            if (i < b && j < b) g.out[krow[i] + (int64_t)prow[j] * g.ldo] = a[p][q];
        }
}

template <typename T, int MR, int MC>
hodlr_status launch_gj_reg(hodlr_ctx *c, const GJDesc<T> *dd, int count, cudaStream_t s) {
    gj_inverse_reg_kernel<T, MR, MC><<<count, GJR_THREADS, 0, s>>>(dd, c->d_status);
    note_launch();
    HODLR_TRY_CUDA(cudaGetLastError());
    return HODLR_OK;
}

// Blocked form of the register Gauss-Jordan above (FP32, b = 65 .. 160):
// the pivots are taken in panels of NB columns.  Warp 0 sweeps a panel's
// columns on all rows by itself (the same implicit pivoting and tie rule: the
// largest |a(i, k)| over unused rows, lowest row first, found with two warp
// reductions on the bit patterns of |a|), then all warps apply the panel to
// the other columns at once.  With R the panel's pivot rows, C its columns and
// P the swept panel (P(R, :) = B^-1, P(i, :) = -a(i, C) B^-1 otherwise, B =
// a(R, C)), sweeping the panel's pivots one after another is, on a column j
// outside C,
//   a(i, j) <- [i not in R] a(i, j) + sum_t P(i, t) a_old(r_t, j),
// r_t the pivot row of the panel's column t.  Three CTA barriers per panel
// instead of two per column.
template <typename T, int MR, int MC, int NB>
__global__ void __launch_bounds__(GJR_THREADS, 1) gj_blocked_kernel(const GJDesc<T> *__restrict__ descs,
                                                                   int *status) {
    static_assert(sizeof(T) == 4, "FP32 only (pivot keys are 32-bit patterns)");
    static_assert(32 % NB == 0 && NB % 4 == 0, "panels of 4k columns within a 32-column slot");
    constexpr int BR = MR * GJR_TY;           // row capacity
    constexpr int MW = (BR + 31) / 32;        // panel rows per lane of warp 0
    const GJDesc<T> g = descs[blockIdx.x];
    const int b = g.b;
    if (b <= 0) return;
    const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
    __shared__ __align__(16) T P[2][BR][NB];  // the panel, by panel parity
    __shared__ T Rold[NB][MC * GJR_TX];       // the panel's pivot rows before its sweeps
    __shared__ int piv[NB];
    __shared__ int prow[BR];                  // pivot row of step k
    __shared__ int krow[BR];                  // step at which row i was the pivot
    __shared__ unsigned char rused[BR];
    __shared__ int s_fail;
    __shared__ T *s_out;                      // the output's address and stride, parked here
    __shared__ int64_t s_ldo;                 // for the final store (registers are the limit)
    T a[MR][MC];
#pragma unroll
    for (int p = 0; p < MR; ++p) {
        const int i = ty + GJR_TY * p;
#pragma unroll
        for (int q = 0; q < MC; ++q) {
            const int j = tx + GJR_TX * q;
            T v = T(0);
            if (i < b && j < b)
                v = g.srcA ? dev::from_double<T>(g.srcA[(int64_t)i * g.lda + j]) : g.srcM[i + (int64_t)j * g.ldm];
            a[p][q] = v;
        }
    }
    for (int i = tid; i < BR; i += GJR_THREADS) rused[i] = i >= b ? 1 : 0;
    for (int e = tid; e < 2 * BR * NB; e += GJR_THREADS) (&P[0][0][0])[e] = T(0);
    if (tid == 0) {
        s_fail = 0;
        s_out = g.out;
        s_ldo = g.ldo;
    }
    __syncthreads();
    bool fail = false;
    // one copy of the panel's code (the slot kq of the panel's columns is a
    // runtime value; unrolling over it multiplied the code beyond the
    // instruction cache)
    for (int k0 = 0, panel = 0; k0 < b && !fail; k0 += NB, ++panel) {
        const int kq = k0 / GJR_TX, kx0 = k0 % GJR_TX;
        const int nbp = min(NB, b - k0);
        const int par = panel & 1;
        const bool inpanel = tx >= kx0 && tx < kx0 + nbp;
        // 1. the owners of the panel's columns post them
        if (inpanel) {
#pragma unroll
            for (int p = 0; p < MR; ++p) {
                T v = a[p][0];
#pragma unroll
                for (int q = 1; q < MC; ++q)
                    if (q == kq) v = a[p][q];
                P[par][ty + GJR_TY * p][tx - kx0] = v;
            }
        }
        __syncthreads();
        // 2. warp 0 sweeps the panel's pivots on the panel
        if (ty == 0) {
            T v[MW][NB];
            unsigned ub = 0;   // bit m: row tx + 32 m is not a candidate
#pragma unroll
            for (int m = 0; m < MW; ++m) {
                const int i = tx + 32 * m;
                if (i < BR) {
                    if (rused[i]) ub |= 1u << m;
#pragma unroll
                    for (int t = 0; t < NB; ++t) v[m][t] = P[par][i][t];
                } else {
                    ub |= 1u << m;
#pragma unroll
                    for (int t = 0; t < NB; ++t) v[m][t] = T(0);
                }
            }
#pragma unroll
            for (int t = 0; t < NB; ++t) {
                if (t >= nbp) break;
                unsigned best = 0u;
                int bi = INT_MAX;
#pragma unroll
                for (int m = 0; m < MW; ++m) {
                    const T av = fabsf(v[m][t]);
                    const unsigned key = (av > T(0)) ? __float_as_uint(av) : 0u;   // NaN: no candidate
                    if (!((ub >> m) & 1u) && key > best) {
                        best = key;
                        bi = tx + 32 * m;
                    }
                }
                const unsigned wmax = __reduce_max_sync(0xffffffffu, best);
                if (wmax == 0u) {   // uniform: no usable pivot in this column
                    if (tx == 0) s_fail = 1;
                    break;
                }
                const int pr = (int)__reduce_min_sync(0xffffffffu, best == wmax ? (unsigned)bi : 0xffffffffu);
                const int o = pr & 31, mo = pr >> 5;
                T rr[NB];
#pragma unroll
                for (int m = 0; m < MW; ++m)
                    if (m == mo) {
#pragma unroll
                        for (int t2 = 0; t2 < NB; ++t2) rr[t2] = __shfl_sync(0xffffffffu, v[m][t2], o);
                    }
                const T pv = rr[t];
                const T d = T(1) / pv;
                // elimination on every entry, then the pivot column -v(i, t) / p,
                // the pivot row v(pr, :) / p and the pivot 1 / p (scale-invariant)
#pragma unroll
                for (int m = 0; m < MW; ++m) {
                    const bool isp = (tx + 32 * m) == pr;
                    const T f = v[m][t] * d;
#pragma unroll
                    for (int t2 = 0; t2 < NB; ++t2) v[m][t2] = fmaf(-f, rr[t2], v[m][t2]);
                    v[m][t] = -f;
                    if (isp) {
#pragma unroll
                        for (int t2 = 0; t2 < NB; ++t2) v[m][t2] = rr[t2] * d;
                        v[m][t] = d;
                        ub |= 1u << m;
                    }
                }
                if (tx == 0) {
                    piv[t] = pr;
                    prow[k0 + t] = pr;
                    krow[pr] = k0 + t;
                    rused[pr] = 1;
                }
            }
#pragma unroll
            for (int m = 0; m < MW; ++m) {
                const int i = tx + 32 * m;
                if (i < BR) {
#pragma unroll
                    for (int t = 0; t < NB; ++t) P[par][i][t] = (t < nbp) ? v[m][t] : T(0);
                }
            }
        }
        __syncthreads();
        if (s_fail) {
            fail = true;
            break;
        }
        // 3. the owners of the panel's pivot rows post them as they were before the panel
        unsigned cur = 0;   // bit p: row ty + 8 p is one of this panel's pivot rows
        for (int t = 0; t < nbp; ++t) {
            const int r = piv[t];
            if ((r & (GJR_TY - 1)) == ty) {
                const int pp = r / GJR_TY;
#pragma unroll
                for (int p = 0; p < MR; ++p)
                    if (p == pp) {
                        cur |= 1u << p;
#pragma unroll
                        for (int q = 0; q < MC; ++q) Rold[t][tx + GJR_TX * q] = a[p][q];
                    }
            }
        }
        __syncthreads();
        // 4. the panel's update of every other column; the panel's columns take
        // P.  Column slots outermost with their NB pivot-row entries in
        // registers and the panel rows read as 16-byte vectors (holding all
        // slots' entries at once measured 2.5x slower at this register budget).
#pragma unroll
        for (int q = 0; q < MC; ++q) {
            T rk[NB];
#pragma unroll
            for (int t = 0; t < NB; ++t) rk[t] = (t < nbp) ? Rold[t][tx + GJR_TX * q] : T(0);
            const bool pcol = (q == kq) && inpanel;
#pragma unroll
            for (int p = 0; p < MR; ++p) {
                const int i = ty + GJR_TY * p;
                T pn[NB];
#pragma unroll
                for (int t = 0; t < NB; t += 4) {
                    const float4 w = *reinterpret_cast<const float4 *>(&P[par][i][t]);
                    pn[t] = w.x;
                    pn[t + 1] = w.y;
                    pn[t + 2] = w.z;
                    pn[t + 3] = w.w;
                }
                T acc = ((cur >> p) & 1u) ? T(0) : a[p][q];
#pragma unroll
                for (int t = 0; t < NB; ++t) acc = fmaf(pn[t], rk[t], acc);
                a[p][q] = pcol ? P[par][i][tx - kx0] : acc;
            }
        }
    }
    if (fail) {
        if (tid == 0) atomicOr(status, ST_SINGULAR);
        return;
    }
    __syncthreads();
    // M^-1(krow[i], prow[j]) = a(i, j)
    T *out = s_out;
    const int64_t ldo = s_ldo;
#pragma unroll
    for (int p = 0; p < MR; ++p)
#pragma unroll
        for (int q = 0; q < MC; ++q) {
            const int i = ty + GJR_TY * p, j = tx + GJR_TX * q;
            if (i < b && j < b) out[krow[i] + (int64_t)prow[j] * ldo] = a[p][q];
        }
}

template <typename T, int MR, int MC, int NB = 4>
hodlr_status launch_gj_blocked(hodlr_ctx *c, const GJDesc<T> *dd, int count, cudaStream_t s) {
    gj_blocked_kernel<T, MR, MC, NB><<<count, GJR_THREADS, 0, s>>>(dd, c->d_status);
    note_launch();
    HODLR_TRY_CUDA(cudaGetLastError());
    return HODLR_OK;
}

// Gauss-Jordan inversion of matrices up to 256 x 256 held in the registers of
// a cluster of CL CTAs: CTA r of the cluster owns the columns r MC 32 ..
// (r + 1) MC 32 - 1 of every row (256 threads as 8 x 32, thread (ty, tx) the
// rows ty + 8 p, p < MR, and the columns tx + 32 q of its slice, q < MC).  The
// sweep is the implicit-pivoting one of gj_inverse_reg_kernel (pivot p_k =
// argmax |a(i, k)| over the rows not yet pivots, lowest row on ties; one FMA
// per element and step).  Per step only the pivot column crosses the cluster:
// the CTA owning column k picks the pivot, writes the column (with its pivot
// entry adjusted) and the pivot's row and value into every CTA's shared memory
// (DSMEM stores), and one cluster barrier publishes them; each CTA then posts
// its part of the pivot row locally and updates its own columns.  Buffers are
// double-buffered by step parity: a CTA writes step k's buffers only after the
// cluster barrier of step k - 1, which its peers pass only once they finished
// reading step k - 2's.  One cluster per matrix (blockIdx.x / CL).
template <typename T, int CL, int MR, int MC>
__global__ void __launch_bounds__(GJR_THREADS, 1) gj_cluster_kernel(const GJDesc<T> *__restrict__ descs,
                                                                   int *status) {
    constexpr int BR = MR * GJR_TY;          // rows held (256)
    constexpr int CW = MC * GJR_TX;          // columns per CTA
    const GJDesc<T> g = descs[blockIdx.x / CL];
    const int b = g.b;
    // every CTA of the cluster reads the same descriptor: all leave here together
    if (b <= 0 || (g.gate && *g.gate == 0)) return;
    unsigned rank;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(rank));
    const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
    const int c0 = (int)rank * CW;           // first column of this CTA
    __shared__ T colk[2][BR];
    __shared__ T rowk[2][CW];
    __shared__ T cand_v[2][GJR_TY];
    __shared__ int cand_i[2][GJR_TY];
    __shared__ int s_pr[2];
    __shared__ T s_piv[2];
    __shared__ int s_fail[2];
    __shared__ int prow[BR];   // pivot row of step k
    __shared__ int krow[BR];   // step at which row i was the pivot
    T a[MR][MC];
    unsigned long long used = 0;
#pragma unroll
    for (int p = 0; p < MR; ++p) {
        const int i = ty + GJR_TY * p;
        if (i >= b) used |= 1ull << p;
#pragma unroll
        for (int q = 0; q < MC; ++q) {
            const int j = c0 + tx + GJR_TX * q;
            T v = T(0);
            if (b > 0 && i < b && j < b)
                v = g.srcA ? dev::from_double<T>(g.srcA[(int64_t)i * g.lda + j]) : g.srcM[i + (int64_t)j * g.ldm];
            a[p][q] = v;
        }
    }
    if (tid < 2) s_fail[tid] = 0;
    // the DSMEM addresses of the shared buffers in every CTA of the cluster
    auto remote = [](const void *p, unsigned r) {
        unsigned out;
        asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(out) : "r"((unsigned)__cvta_generic_to_shared(p)), "r"(r));
        return out;
    };
    auto st_remote = [](unsigned addr, T v) {
        if constexpr (sizeof(T) == 4)
            asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(addr), "f"(v) : "memory");
        else
            asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(addr), "d"(v) : "memory");
    };
    auto st_remote_i = [](unsigned addr, int v) {
        asm volatile("st.shared::cluster.s32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
    };
    auto cluster_sync = []() {
        asm volatile("barrier.cluster.arrive.release.aligned;\nbarrier.cluster.wait.acquire.aligned;" ::: "memory");
    };
    cluster_sync();   // every CTA of the cluster is running and initialised
    bool fail = false;
    for (int owner = 0; owner < CL && !fail; ++owner) {
#pragma unroll
        for (int kq = 0; kq < MC; ++kq) {
            const int kbase = owner * CW + kq * GJR_TX;
            const int kxe = min(GJR_TX, b - kbase);
            for (int kx = 0; kx < kxe && !fail; ++kx) {
                const int k = kbase + kx;
                const int par = k & 1;
                const bool mine = (int)rank == owner;
                // A. the owner's column-k threads post it and their best unused row
                if (mine && tx == kx) {
                    T bv = T(-1), sv = T(0);
                    int bi = INT_MAX;
#pragma unroll
                    for (int p = 0; p < MR; ++p) {
                        const T v = a[p][kq];
                        colk[par][ty + GJR_TY * p] = v;
                        const T av = fabs(v);
                        if (!((used >> p) & 1ull) && av > bv) {
                            bv = av;
                            sv = v;
                            bi = ty + GJR_TY * p;
                        }
                    }
                    cand_v[par][ty] = sv;
                    cand_i[par][ty] = bi;
                }
                __syncthreads();
                // B. the owner merges the candidates and publishes the column
                if (mine) {
                    T pa = T(-1), piv = T(0);
                    int pr = INT_MAX;
                    if (tx < GJR_TY) {
                        pr = cand_i[par][tx];
                        piv = cand_v[par][tx];
                        pa = pr == INT_MAX ? T(-1) : fabs(piv);
                    }
#pragma unroll
                    for (int o = GJR_TY / 2; o > 0; o >>= 1) {
                        const T oa = __shfl_xor_sync(0xffffffffu, pa, o);
                        const T ov = __shfl_xor_sync(0xffffffffu, piv, o);
                        const int oi = __shfl_xor_sync(0xffffffffu, pr, o);
                        if (oa > pa || (oa == pa && oi < pr)) {
                            pa = oa;
                            piv = ov;
                            pr = oi;
                        }
                    }
                    pa = __shfl_sync(0xffffffffu, pa, 0);
                    piv = __shfl_sync(0xffffffffu, piv, 0);
                    pr = __shfl_sync(0xffffffffu, pr, 0);
                    const bool bad = !(pa > T(0));
                    // every other CTA receives the column; every CTA the pivot row and value
                    for (int r = 0; r < CL; ++r) {
                        if (r != (int)rank)
                            for (int i = tid; i < BR; i += GJR_THREADS)
                                st_remote(remote(&colk[par][i], r), colk[par][i]);
                        if (tid == 0) {
                            st_remote_i(remote(&s_pr[par], r), bad ? 0 : pr);
                            st_remote(remote(&s_piv[par], r), piv);
                            st_remote_i(remote(&s_fail[par], r), bad ? 1 : 0);
                        }
                    }
                }
                cluster_sync();
                if (s_fail[par]) {   // uniform across the cluster
                    fail = true;
                    break;
                }
                const int pr = s_pr[par];
                const T piv = s_piv[par];
                const int py = pr % GJR_TY, pp = pr / GJR_TY;
                // C. the pivot row's owners post this CTA's part of it (before the sweep)
                if (ty == py) {
#pragma unroll
                    for (int p = 0; p < MR; ++p)
                        if (p == pp) {
                            used |= 1ull << p;
#pragma unroll
                            for (int q = 0; q < MC; ++q) rowk[par][tx + GJR_TX * q] = a[p][q];
                        }
                }
                if (tid == 0) {
                    prow[k] = pr;
                    krow[pr] = k;
                }
                __syncthreads();
                // D. sweep the pivot (pr, k) on this CTA's columns: the elimination
                // on every element, then the pivot column -a(i, k) / p, the pivot
                // row a(pr, j) / p and the pivot 1 / p (scale-invariant)
                const T d = T(1) / piv;
                T rk[MC];
#pragma unroll
                for (int q = 0; q < MC; ++q) rk[q] = rowk[par][tx + GJR_TX * q];
                const bool kcol = mine && tx == kx;
#pragma unroll
                for (int p = 0; p < MR; ++p) {
                    const T f = colk[par][ty + GJR_TY * p] * d;
#pragma unroll
                    for (int q = 0; q < MC; ++q) a[p][q] = fma(-f, rk[q], a[p][q]);
                    if (kcol) a[p][kq] = -f;
                }
                if (ty == py) {
#pragma unroll
                    for (int p = 0; p < MR; ++p)
                        if (p == pp) {
#pragma unroll
                            for (int q = 0; q < MC; ++q) a[p][q] = rk[q] * d;
                            if (kcol) a[p][kq] = d;
                        }
                }
            }
        }
    }
    if (fail) {
        if (tid == 0 && rank == 0) atomicOr(status, ST_SINGULAR);
        cluster_sync();
        return;
    }
    __syncthreads();
    // M^-1(krow[i], prow[j]) = a(i, j) on this CTA's columns
#pragma unroll
    for (int p = 0; p < MR; ++p)
#pragma unroll
        for (int q = 0; q < MC; ++q) {
            const int i = ty + GJR_TY * p, j = c0 + tx + GJR_TX * q;
            if (i < b && j < b) g.out[krow[i] + (int64_t)prow[j] * g.ldo] = a[p][q];
        }
    cluster_sync();   // no CTA leaves while a peer may still address its shared memory
}

template <typename T, int CL, int MR, int MC>
hodlr_status launch_gj_cluster(hodlr_ctx *c, const GJDesc<T> *dd, int count, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(count * CL));
    cfg.blockDim = dim3(GJR_THREADS);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    {
        ProfScope ps("gj_cluster_kernel", s);
        HODLR_TRY_CUDA(cudaLaunchKernelEx(&cfg, gj_cluster_kernel<T, CL, MR, MC>, dd, c->d_status));
    }
    note_launch();
    return HODLR_OK;
}

template <typename T>
size_t gjs_smem(int b) {
    return ((size_t)(b + 1) * b + 2 * (size_t)b) * sizeof(T) + (size_t)b * sizeof(int) + 16;
}

// 16-bit copy of the columns coff .. coff+rp of a level (node rows): BF16
// directly; FP16 scaled per (node, column) by 2^e so that the column's largest
// magnitude lands just below 2^14, with 2^-e stored as the dequantisation factor.
template <typename S>
__device__ __forceinline__ S to_store(float x);
template <>
__device__ __forceinline__ __nv_bfloat16 to_store<__nv_bfloat16>(float x) { return __float2bfloat16_rn(x); }
template <>
__device__ __forceinline__ __half to_store<__half>(float x) { return __float2half_rn(x); }

template <typename S>
__global__ void quantize_kernel(const float *__restrict__ src, S *__restrict__ dst, int64_t ldn, int64_t coff, int rp,
                                const int64_t *__restrict__ bounds, int L, int l, float *__restrict__ scale) {
    const int node = blockIdx.x, col = blockIdx.y;
    const int64_t r0 = bounds[(size_t)node << (L - l)], r1 = bounds[(size_t)(node + 1) << (L - l)];
    const float *x = src + (coff + col) * ldn;
    S *y = dst + (coff + col) * ldn;
    float f = 1.f;
    if (scale) {
        __shared__ float red[32];
        float mx = 0.f;
        for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) mx = fmaxf(mx, fabsf(x[i]));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
        __syncthreads();
        if (threadIdx.x == 0) {
            float m = 0.f;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, red[w]);
            int e = 0;
            if (m > 0.f) {
                int E;
                frexpf(m, &E);          // m = f 2^E, f in [0.5, 1)
                e = 14 - E;
            }
            red[0] = ldexpf(1.f, e);
            scale[(size_t)node * rp + col] = ldexpf(1.f, -e);
        }
        __syncthreads();
        f = red[0];
    }
    for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) y[i] = to_store<S>(x[i] * f);
}

// Condition of the Woodbury cores of one level in the 1-norm, exactly from the
// matrices the factorisation forms: S = [[I, P], [Q, I]] (P, Q the two halves of
// the children's V^T d, 2r x r column-major, ld 2r) and S^-1 (2r x 2r), so
//   ||S||_1 = 1 + max_j max(sum_i |P(i,j)|, sum_i |Q(i,j)|),
//   ||S^-1||_1 = max_j sum_i |S^-1(i,j)|,  kappa_1 = ||S||_1 ||S^-1||_1.
// One CTA per core, a warp per column.  flag = kappa_1 > thr (or not finite).
// The last CTA to finish (counter, reset by it) sets the graph's conditional
// to whether any core of the level is flagged, when the kernel runs inside the
// guard's graph (has_handle).
constexpr int CC_THREADS = 256;

template <typename T>
__global__ void __launch_bounds__(CC_THREADS)
    core_cond_kernel(const T *__restrict__ Y, const T *__restrict__ Sinv, int r, double thr, double *cond, int *flag,
                     unsigned *counter, int has_handle, cudaGraphConditionalHandle handle) {
    const int i = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int NW = CC_THREADS / 32;
    const int64_t s2 = 2 * (int64_t)r;
    const T *Yi = Y + (size_t)i * s2 * r;
    const T *Si = Sinv + (size_t)i * s2 * s2;
    __shared__ double red_s[NW], red_i[NW];
    double ms = 0.0, mi = 0.0;
    for (int j = warp; j < r; j += NW) {   // columns of P and Q
        double p = 0.0, q = 0.0;
        for (int k = lane; k < r; k += 32) {
            p += fabs((double)Yi[k + j * s2]);
            q += fabs((double)Yi[r + k + j * s2]);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            p += __shfl_xor_sync(0xffffffffu, p, o);
            q += __shfl_xor_sync(0xffffffffu, q, o);
        }
        ms = fmax(ms, fmax(p, q));
    }
    for (int j = warp; j < s2; j += NW) {  // columns of S^-1
        double a = 0.0;
        for (int k = lane; k < s2; k += 32) a += fabs((double)Si[k + j * s2]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        mi = (a > mi || a != a) ? a : mi;   // a NaN column makes the core unusable
    }
    if (lane == 0) {
        red_s[warp] = ms;
        red_i[warp] = mi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < NW; ++w) {
            a = fmax(a, red_s[w]);
            b = (red_i[w] > b || red_i[w] != red_i[w]) ? red_i[w] : b;
        }
        double k = (1.0 + a) * b;
        if (!(k <= 1.7976931348623157e308)) k = __longlong_as_double(0x7ff0000000000000LL);   // NaN, inf -> inf
        cond[i] = k;
        flag[i] = (k > thr) ? 1 : 0;
        __threadfence();
        if (atomicAdd(counter, 1u) == gridDim.x - 1) {   // the last core of the level
            __threadfence();
            int any = 0;
            for (unsigned c = 0; c < gridDim.x; ++c) any |= reinterpret_cast<volatile int *>(flag)[c];
            *counter = 0u;
            if (has_handle) cudaGraphSetConditional(handle, any ? 1u : 0u);
        }
    }
}

// S^-1 of the cores re-inverted in FP64, rounded into the FP32 core array
// (blockIdx.y = core; cores whose flag is 0 keep their FP32 inverse).
__global__ void core_store_kernel(const double *__restrict__ S64, float *__restrict__ S32, int64_t per,
                                  const int *__restrict__ flag) {
    const int i = blockIdx.y;
    if (!flag[i]) return;
    const double *a = S64 + (size_t)i * per;
    float *b = S32 + (size_t)i * per;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < per; e += (int64_t)gridDim.x * blockDim.x)
        b[e] = __double2float_rn(a[e]);
}

// Which Gauss-Jordan variant launch_gj picks for matrices up to bmax: registers,
// shared memory, or the global-memory kernel (the only one that needs GJDesc::work).
template <typename T>
bool gj_needs_work(int bmax) {
    if (bmax <= 256) return false;   // registers (of one CTA, or of a cluster from 161 (FP32) / 129 (FP64))
    return gjs_smem<T>(bmax) > GJS_SMEM_MAX;
}

template <typename T>
hodlr_status launch_gj(hodlr_ctx *c, const GJDesc<T> *dd, int count, int bmax, cudaStream_t s) {
    if (bmax <= 32) return launch_gj_reg<T, 4, 1>(c, dd, count, s);
    if (bmax <= 64) return launch_gj_reg<T, 8, 2>(c, dd, count, s);
    if constexpr (sizeof(T) == 4) {   // blocked from 65 to 160; FP64 tiles beyond 128 would spill registers
        if (bmax <= 96) return launch_gj_blocked<T, 12, 3>(c, dd, count, s);
        if (bmax <= 128) return launch_gj_blocked<T, 16, 4>(c, dd, count, s);
        if (bmax <= 144) return launch_gj_blocked<T, 18, 5>(c, dd, count, s);
        if (bmax <= 160) return launch_gj_blocked<T, 20, 5>(c, dd, count, s);
        if (bmax <= 256) return launch_gj_cluster<T, 2, 32, 4>(c, dd, count, s);   // 161 .. 256: two CTAs
    } else {
        if (bmax <= 96) return launch_gj_reg<T, 12, 3>(c, dd, count, s);
        if (bmax <= 128) return launch_gj_reg<T, 16, 4>(c, dd, count, s);
        if (bmax <= 256) return launch_gj_cluster<T, 8, 32, 1>(c, dd, count, s);   // 129 .. 256: eight CTAs
    }
    if (gjs_smem<T>(bmax) <= GJS_SMEM_MAX) {
        const size_t sm = gjs_smem<T>(bmax);
        HODLR_TRY_CUDA(cudaFuncSetAttribute(gj_inverse_smem_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)sm));
        gj_inverse_smem_kernel<T><<<count, GJS_THREADS, sm, s>>>(dd, c->d_status);
        note_launch();
        HODLR_TRY_CUDA(cudaGetLastError());
        return HODLR_OK;
    }
    size_t sm = 3 * (size_t)bmax * sizeof(T);
    HODLR_TRY_CUDA(cudaFuncSetAttribute(gj_inverse_kernel<T>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    gj_inverse_kernel<T><<<count, GJ_THREADS, sm, s>>>(dd, c->d_status);
    note_launch();
    HODLR_TRY_CUDA(cudaGetLastError());
    return HODLR_OK;
}

}  // namespace

// The factorisation is recorded level by level when the HODLR matrix is built:
// the launches of each level's share (see plan_level) with their arguments, and
// that share's batched-GEMM and inversion descriptors laid out in one blob
// uploaded in a single copy.  Replaying needs no host-device transfer.
struct LevelPlan {
    std::vector<std::function<hodlr_status(cudaStream_t)>> ops;
    // (op index, level l): ops from that index on read level l's share (its d,
    // V and the cores of level l - 1); a replay on its own stream waits there
    std::vector<std::pair<size_t, int>> waits;
    std::vector<char> blob;
    char *dblob = nullptr;
    size_t dbytes = 0;
    void *work = nullptr;
    size_t work_bytes = 0;
    // the condition guard's FP64 re-inversion of the cores of this share's
    // parents: recorded apart, then built into one graph (the condition kernel,
    // then a conditional node whose body runs when some core is flagged)
    std::vector<std::function<hodlr_status(cudaStream_t)>> redo;
    cudaGraph_t ggraph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    struct {
        const void *Y = nullptr, *Sinv = nullptr;
        int r = 0;
        double thr = 0.0;
        double *cond = nullptr;
        int *flag = nullptr;
        unsigned *counter = nullptr;
        int count = 0;
        size_t esize = 0;
    } cond_args;

    size_t put(const void *p, size_t bytes) {
        const size_t off = (blob.size() + 255) & ~size_t(255);
        blob.resize(off + bytes);
        std::memcpy(blob.data() + off, p, bytes);
        return off;
    }
};

struct FactorPlan {
    std::vector<LevelPlan> lv;   // index 1..L
};

namespace {

template <typename T>
struct Rec {
    hodlr_ctx *c;
    LevelPlan *P;
    std::vector<std::function<hodlr_status(cudaStream_t)>> *to = nullptr;   // default: P->ops
    std::vector<std::function<hodlr_status(cudaStream_t)>> &dst() { return to ? *to : P->ops; }
    template <typename TG>
    void gj(const std::vector<GJDesc<TG>> &hd) {
        if (hd.empty()) return;
        int bmax = 0;
        for (auto &g : hd) bmax = std::max(bmax, g.b);
        const size_t off = P->put(hd.data(), hd.size() * sizeof(GJDesc<TG>));
        const int cnt = (int)hd.size();
        hodlr_ctx *cc = c;
        LevelPlan *PP = P;
        dst().push_back([=](cudaStream_t s) {
            return launch_gj<TG>(cc, reinterpret_cast<const GJDesc<TG> *>(PP->dblob + off), cnt, bmax, s);
        });
    }
    template <typename TC, typename TI>
    void gemm(const std::vector<GemmDesc<TC, TI>> &hd, int transA, TC alpha) {
        if (hd.empty()) return;
        int maxM = 0, maxN = 0, maxK = 0;
        for (auto &g : hd) {
            maxM = std::max(maxM, g.M);
            maxN = std::max(maxN, g.N);
            maxK = std::max(maxK, g.K);
        }
        if (maxM == 0 || maxN == 0 || maxK == 0) return;
        const size_t off = P->put(hd.data(), hd.size() * sizeof(GemmDesc<TC, TI>));
        const int cnt = (int)hd.size();
        hodlr_ctx *cc = c;
        LevelPlan *PP = P;
        dst().push_back([=](cudaStream_t s) {
            return gemm_batched<TC, TI>(cc, reinterpret_cast<const GemmDesc<TC, TI> *>(PP->dblob + off), cnt, maxM,
                                        maxN, maxK, transA, alpha, s);
        });
    }
    // generic: one recorded launch
    void op(std::function<hodlr_status(cudaStream_t)> f) { dst().push_back(std::move(f)); }
    template <typename TF>
    void fill(const std::vector<FillDesc<TF>> &hd) {
        if (hd.empty()) return;
        int64_t most = 0;
        for (auto &f : hd) most = std::max(most, f.rows * f.cols * f.count);
        const unsigned gx = (unsigned)std::max<int64_t>(1, std::min<int64_t>(512, (most + 2047) / 2048));
        const size_t off = P->put(hd.data(), hd.size() * sizeof(FillDesc<TF>));
        const int cnt = (int)hd.size();
        LevelPlan *PP = P;
        dst().push_back([=](cudaStream_t s) {
            fill_kernel<TF><<<dim3(gx, cnt), 256, 0, s>>>(reinterpret_cast<const FillDesc<TF> *>(PP->dblob + off));
            note_launch();
            HODLR_TRY_CUDA(cudaGetLastError());
            return HODLR_OK;
        });
    }
};

// The guard's graph of one share: the condition kernel (which sets the
// conditional to whether any core was flagged), then a conditional node whose
// body is the recorded FP64 re-inversion, captured on a side stream.  Kernels
// of the body are not counted by hodlr_launch_count (they run only when a core
// is flagged).
hodlr_status build_guard_graph(hodlr_ctx *cx, LevelPlan *Pl) {
    auto &ca = Pl->cond_args;
    HODLR_TRY_CUDA(cudaGraphCreate(&Pl->ggraph, 0));
    cudaGraphConditionalHandle handle;
    HODLR_TRY_CUDA(cudaGraphConditionalHandleCreate(&handle, Pl->ggraph, 0, cudaGraphCondAssignDefault));
    const float *Y = reinterpret_cast<const float *>(ca.Y);
    const float *Sv = reinterpret_cast<const float *>(ca.Sinv);
    int has = 1;
    void *kargs[] = {(void *)&Y, (void *)&Sv, (void *)&ca.r, (void *)&ca.thr, (void *)&ca.cond, (void *)&ca.flag,
                     (void *)&ca.counter, (void *)&has, (void *)&handle};
    cudaKernelNodeParams kp = {};
    kp.func = (void *)core_cond_kernel<float>;
    kp.gridDim = dim3((unsigned)ca.count);
    kp.blockDim = dim3(CC_THREADS);
    kp.kernelParams = kargs;
    cudaGraphNode_t knode, cnode;
    HODLR_TRY_CUDA(cudaGraphAddKernelNode(&knode, Pl->ggraph, nullptr, 0, &kp));
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = handle;
    cp.conditional.type = cudaGraphCondTypeIf;
    cp.conditional.size = 1;
    HODLR_TRY_CUDA(cudaGraphAddNode(&cnode, Pl->ggraph, &knode, nullptr, 1, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    cudaStream_t cs = cx->side[HODLR_SIDE_STREAMS - 1];
    HODLR_TRY_CUDA(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    hodlr_status rs = HODLR_OK;
    {
        LaunchCapture cap;   // not executed now
        for (auto &f : Pl->redo) {
            rs = f(cs);
            if (rs != HODLR_OK) break;
        }
    }
    cudaGraph_t captured = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(cs, &captured);
    HODLR_TRY(rs);
    if (ce != cudaSuccess) {
        set_error("factor: capture of the condition guard failed: %s", cudaGetErrorString(ce));
        return HODLR_CUDA_ERROR;
    }
    HODLR_TRY_CUDA(cudaGraphInstantiate(&Pl->gexec, Pl->ggraph, 0));
    return HODLR_OK;
}

template <typename T>
hodlr_status plan_level_typed(hodlr_t *h, LevelPlan *Pl, int c, cudaStream_t s) {
    hodlr_ctx *cx = h->ctx;
    const int L = h->L;
    const int64_t ldn = h->ldn;
    const int nleaf = 1 << L;
    const int64_t bmax = h->bmax;
    auto node_range = [&](int l, int i, int64_t &r0, int64_t &m) {
        r0 = h->bounds[(size_t)i << (L - l)];
        m = h->bounds[(size_t)(i + 1) << (L - l)] - r0;
    };
    const int rc = h->lv[c].rp;
    T *Uc = reinterpret_cast<T *>(h->Ul[c]);
    T *Dc = reinterpret_cast<T *>(h->Dl[c]);
    T *Vc = reinterpret_cast<T *>(h->Vl[c]);
    T *Ec = reinterpret_cast<T *>(h->El[c]);
    const T *Kinv = reinterpret_cast<const T *>(h->leafinv);
    // ---- workspace: per deeper level l the children's V^T d_c and its S^-1
    // image, then the cores of level c - 1 (one allocation)
    Arena ws;
    std::vector<size_t> oY(L), oYv(L);
    for (int l = L - 1; l >= c; --l) {
        const size_t bytes = (size_t)(1 << l) * 2 * h->lv[l + 1].rp * std::max(rc, 1) * sizeof(T);
        oY[l] = ws.take(bytes);
        oYv[l] = ws.take(bytes);
    }
    const int nn0 = 1 << (c - 1);
    const int64_t s2c = 2 * (int64_t)rc;
    const size_t oYo = ws.take((size_t)nn0 * s2c * std::max(rc, 1) * sizeof(T));
    const size_t oM = ws.take((size_t)nn0 * rc * rc * sizeof(T));
    const bool gwn = gj_needs_work<T>(rc);
    const size_t oGW = gwn ? ws.take((size_t)nn0 * 2 * rc * rc * sizeof(T)) : 0;
    // the FP64 re-inversion of the cores above the condition threshold (FP32 arithmetic)
    const bool redo = h->promote && sizeof(T) == 4 && rc > 0;
    const bool gwn64 = redo && gj_needs_work<double>(rc);
    const size_t oY64 = redo ? ws.take((size_t)nn0 * s2c * rc * sizeof(double)) : 0;
    const size_t oM64 = redo ? ws.take((size_t)nn0 * rc * rc * sizeof(double)) : 0;
    const size_t oGW64 = gwn64 ? ws.take((size_t)nn0 * 2 * rc * rc * sizeof(double)) : 0;
    Pl->work = dalloc(cx, ws.bytes, s);
    if (!Pl->work) {
        set_error("factor plan: out of device memory (%zu bytes)", ws.bytes);
        return HODLR_OUT_OF_MEMORY;
    }
    Pl->work_bytes = ws.bytes;
    char *wb = reinterpret_cast<char *>(Pl->work);
    Rec<T> rec{cx, Pl};
    // ---- zeros and identities this share starts from
    std::vector<FillDesc<T>> fills;
    if (rc > 0) {
        fills.push_back(FillDesc<T>{Dc, 0, ldn * rc, 1, INT_MAX, 1, 0});
        fills.push_back(FillDesc<T>{Ec, 0, ldn * 2 * rc, 1, INT_MAX, 1, 0});
        for (int l = L - 1; l >= c; --l) {
            const int64_t e = (int64_t)(1 << l) * 2 * h->lv[l + 1].rp * rc;
            if (e == 0) continue;
            fills.push_back(FillDesc<T>{reinterpret_cast<T *>(wb + oY[l]), 0, e, 1, INT_MAX, 1, 0});
            fills.push_back(FillDesc<T>{reinterpret_cast<T *>(wb + oYv[l]), 0, e, 1, INT_MAX, 1, 0});
        }
        fills.push_back(FillDesc<T>{reinterpret_cast<T *>(wb + oYo), 0, (int64_t)nn0 * s2c * rc, 1, INT_MAX, 1, 0});
        fills.push_back(FillDesc<T>{reinterpret_cast<T *>(wb + oM), rc, rc, rc, 0, nn0, (int64_t)rc * rc});   // I
        fills.push_back(FillDesc<T>{reinterpret_cast<T *>(h->Sinv[c - 1]), s2c, s2c, s2c, rc, nn0,
                                    s2c * s2c});   // [0 0; 0 I]
    }
    rec.fill(fills);
    if (rc > 0) {
        // ---- d_c = K_leaf^-1 U_c on every leaf
        {
            std::vector<GemmDesc<T>> gd(nleaf);
            for (int i = 0; i < nleaf; ++i) {
                int64_t r0, m;
                node_range(L, i, r0, m);
                gd[i] = GemmDesc<T>{Kinv + (size_t)i * bmax * bmax, Uc + r0, Dc + r0, bmax, ldn, ldn, (int)m, rc,
                                    (int)m};
            }
            rec.gemm(gd, 0, T(1));
        }
        // ---- the Woodbury update of every deeper level, deepest first: for
        // the parents of level l + 1, [y1; y2] = S^-1 [V_ba^T d_c(a); V_ab^T d_c(b)],
        // d_c(a) -= d_a y2, d_c(b) -= d_b y1
        for (int l = L - 1; l >= c; --l) {
            const int rl = h->lv[l + 1].rp;
            if (rl == 0) continue;
            const int nn = 1 << l;
            const int64_t s2 = 2 * (int64_t)rl;
            const T *Vn = reinterpret_cast<const T *>(h->Vl[l + 1]);
            const T *Dn = reinterpret_cast<const T *>(h->Dl[l + 1]);
            const T *Sn = reinterpret_cast<const T *>(h->Sinv[l]);
            Pl->waits.push_back({Pl->ops.size(), l + 1});
            T *Y = reinterpret_cast<T *>(wb + oY[l]);
            T *Yv = reinterpret_cast<T *>(wb + oYv[l]);
            std::vector<GemmDesc<T>> gy(2 * nn), gv(nn), gu(2 * nn);
            for (int ch = 0; ch < 2 * nn; ++ch) {
                int64_t r0, m;
                node_range(l + 1, ch, r0, m);
                gy[ch] = GemmDesc<T>{Vn + r0, Dc + r0, Y + (size_t)(ch / 2) * s2 * rc + (ch & 1) * rl, ldn, ldn, s2,
                                     rl, rc, (int)m};
            }
            for (int i = 0; i < nn; ++i)
                gv[i] = GemmDesc<T>{Sn + (size_t)i * s2 * s2, Y + (size_t)i * s2 * rc, Yv + (size_t)i * s2 * rc, s2, s2,
                                    s2, (int)s2, rc, (int)s2};
            for (int i = 0; i < nn; ++i) {
                int64_t ra, ma, rb, mb;
                node_range(l + 1, 2 * i, ra, ma);
                node_range(l + 1, 2 * i + 1, rb, mb);
                const T *yv = Yv + (size_t)i * s2 * rc;
                gu[2 * i] = GemmDesc<T>{Dn + ra, yv + rl, Dc + ra, ldn, s2, ldn, (int)ma, rc, rl};
                gu[2 * i + 1] = GemmDesc<T>{Dn + rb, yv, Dc + rb, ldn, s2, ldn, (int)mb, rc, rl};
            }
            rec.gemm(gy, 1, T(1));
            rec.gemm(gv, 0, T(1));
            rec.gemm(gu, 0, T(-1));
        }
        // ---- the cores of level c - 1: Y_i = [V_ba^T d_a; V_ab^T d_b] (2 rc x rc),
        // P = Y_a, Q = Y_b, S = [[I, P], [Q, I]], M = I - P Q,
        // S^-1 = [[M^-1, -M^-1 P], [-Q M^-1, I + Q M^-1 P]]
        T *Yo = reinterpret_cast<T *>(wb + oYo);
        T *M = reinterpret_cast<T *>(wb + oM);
        T *gw = gwn ? reinterpret_cast<T *>(wb + oGW) : nullptr;
        T *Sinv = reinterpret_cast<T *>(h->Sinv[c - 1]);
        auto Yi = [&](int i) { return Yo + (size_t)i * s2c * rc; };
        {
            std::vector<GemmDesc<T>> gd(2 * nn0);
            for (int ch = 0; ch < 2 * nn0; ++ch) {
                int64_t r0, m;
                node_range(c, ch, r0, m);
                gd[ch] = GemmDesc<T>{Vc + r0, Dc + r0, Yi(ch / 2) + (ch & 1) * rc, ldn, ldn, s2c, rc, rc, (int)m};
            }
            rec.gemm(gd, 1, T(1));
        }
        {
            std::vector<GemmDesc<T>> gd(nn0);
            for (int i = 0; i < nn0; ++i)
                gd[i] = GemmDesc<T>{Yi(i), Yi(i) + rc, M + (size_t)i * rc * rc, s2c, s2c, rc, rc, rc, rc};
            rec.gemm(gd, 0, T(-1));
        }
        {
            std::vector<GJDesc<T>> gd(nn0);
            for (int i = 0; i < nn0; ++i)
                gd[i] = GJDesc<T>{nullptr, 0, M + (size_t)i * rc * rc, rc, gw ? gw + (size_t)i * 2 * rc * rc : nullptr,
                                  Sinv + (size_t)i * s2c * s2c, s2c, rc};
            rec.gj(gd);
        }
        {
            std::vector<GemmDesc<T>> g12(2 * nn0), g3(nn0);
            for (int i = 0; i < nn0; ++i) {
                T *S = Sinv + (size_t)i * s2c * s2c;
                const T *P = Yi(i), *Q = Yi(i) + rc;
                g12[2 * i] = GemmDesc<T>{S, P, S + rc * s2c, s2c, s2c, s2c, rc, rc, rc};        // TR -= M^-1 P
                g12[2 * i + 1] = GemmDesc<T>{Q, S, S + rc, s2c, s2c, s2c, rc, rc, rc};          // BL -= Q M^-1
                g3[i] = GemmDesc<T>{Q, S + rc * s2c, S + rc + rc * s2c, s2c, s2c, s2c, rc, rc, rc};   // BR -= Q TR
            }
            rec.gemm(g12, 0, T(-1));
            rec.gemm(g3, 0, T(-1));
        }
        // ---- the condition guard: kappa_1(S) of every core; with FP32
        // arithmetic, the cores above the threshold are formed again from the
        // same stored factors with FP64 products (P, Q), inverted in FP64 and
        // rounded into the core array before E is formed from it.  Every step is
        // enqueued for all cores; the flag of a core decides on the device
        // whether its CTAs do any work.
        if (h->guard) {
            // the condition kernel: launched alone, or (FP32 arithmetic) as the
            // first node of the guard's graph built when the share is uploaded
            LevelPlan *PP = Pl;
            double *cond = h->core_cond[c - 1];
            int *flag = h->core_flag[c - 1];
            unsigned *counter = h->core_count[c - 1];
            const double thr = h->promote ? h->cond_thr : __builtin_inf();
            const int cnt = nn0;
            const int rcc = rc;
            hodlr_ctx *gcx = cx;
            rec.op([=](cudaStream_t st) {
                // the guard's graph is built here, on first use: its host cost
                // then overlaps the GPU work already enqueued for this share
                if (!PP->redo.empty() && !PP->gexec) HODLR_TRY(build_guard_graph(gcx, PP));
                if (PP->gexec) {
                    HODLR_TRY_CUDA(cudaGraphLaunch(PP->gexec, st));
                } else {
                    core_cond_kernel<T><<<cnt, CC_THREADS, 0, st>>>(Yo, Sinv, rcc, thr, cond, flag, counter, 0,
                                                                    cudaGraphConditionalHandle{});
                    HODLR_TRY_CUDA(cudaGetLastError());
                }
                note_launch();
                return HODLR_OK;
            });
            Pl->cond_args = {reinterpret_cast<const void *>(Yo), reinterpret_cast<const void *>(Sinv), rcc, thr, cond,
                             flag, counter, cnt, sizeof(T)};
        }
        if (redo) {
            Rec<T> rr{cx, Pl, &Pl->redo};
            const int *flag = h->core_flag[c - 1];
            double *Y64 = reinterpret_cast<double *>(wb + oY64);
            double *M64 = reinterpret_cast<double *>(wb + oM64);
            double *gw64 = gwn64 ? reinterpret_cast<double *>(wb + oGW64) : nullptr;
            double *S64 = h->Sinv64[c - 1];
            auto Y64i = [&](int i) { return Y64 + (size_t)i * s2c * rc; };
            rr.fill(std::vector<FillDesc<double>>{
                FillDesc<double>{Y64, 0, (int64_t)nn0 * s2c * rc, 1, INT_MAX, 1, 0},
                FillDesc<double>{M64, rc, rc, rc, 0, nn0, (int64_t)rc * rc},            // I
                FillDesc<double>{S64, s2c, s2c, s2c, rc, nn0, s2c * s2c}});             // [0 0; 0 I]
            std::vector<GemmDesc<double, T>> gy(2 * nn0);
            for (int ch = 0; ch < 2 * nn0; ++ch) {
                int64_t r0, m;
                node_range(c, ch, r0, m);
                gy[ch] = GemmDesc<double, T>{Vc + r0, Dc + r0, Y64i(ch / 2) + (ch & 1) * rc, ldn, ldn, s2c, rc, rc,
                                             (int)m, flag + ch / 2};
            }
            rr.gemm(gy, 1, 1.0);
            std::vector<GemmDesc<double>> gm(nn0), g12(2 * nn0), g3(nn0);
            std::vector<GJDesc<double>> gj(nn0);
            for (int i = 0; i < nn0; ++i) {
                double *S = S64 + (size_t)i * s2c * s2c;
                const double *P = Y64i(i), *Q = Y64i(i) + rc;
                gm[i] = GemmDesc<double>{P, Q, M64 + (size_t)i * rc * rc, s2c, s2c, rc, rc, rc, rc, flag + i};
                gj[i] = GJDesc<double>{nullptr, 0, M64 + (size_t)i * rc * rc, rc,
                                       gw64 ? gw64 + (size_t)i * 2 * rc * rc : nullptr, S, s2c, rc, flag + i};
                g12[2 * i] = GemmDesc<double>{S, P, S + rc * s2c, s2c, s2c, s2c, rc, rc, rc, flag + i};
                g12[2 * i + 1] = GemmDesc<double>{Q, S, S + rc, s2c, s2c, s2c, rc, rc, rc, flag + i};
                g3[i] = GemmDesc<double>{Q, S + rc * s2c, S + rc + rc * s2c, s2c, s2c, s2c, rc, rc, rc, flag + i};
            }
            rr.gemm(gm, 0, -1.0);
            rr.gj(gj);
            rr.gemm(g12, 0, -1.0);
            rr.gemm(g3, 0, -1.0);
            const int cnt = nn0;
            const int64_t per = s2c * s2c;
            float *S32 = reinterpret_cast<float *>(h->Sinv[c - 1]);
            const unsigned gx = (unsigned)std::max<int64_t>(1, std::min<int64_t>(64, (per + 1023) / 1024));
            rr.op([=](cudaStream_t st) {
                core_store_kernel<<<dim3(gx, cnt), 256, 0, st>>>(S64, S32, per, flag);
                note_launch();
                HODLR_TRY_CUDA(cudaGetLastError());
                return HODLR_OK;
            });
        }
        // ---- E = d_child S^-1(half, :) on every child's rows: the apply's
        // x_child -= d_child y_half with y = S^-1 w becomes x_child -= E w (the
        // first child takes the second half y2, the second child y1)
        {
            std::vector<GemmDesc<T>> gd(2 * nn0);
            for (int ch = 0; ch < 2 * nn0; ++ch) {
                int64_t r0, m;
                node_range(c, ch, r0, m);
                const T *Sh = Sinv + (size_t)(ch / 2) * s2c * s2c + ((ch & 1) ? 0 : rc);
                gd[ch] = GemmDesc<T>{Dc + r0, Sh, Ec + r0, ldn, s2c, ldn, (int)m, (int)s2c, rc};
            }
            rec.gemm(gd, 0, T(1));
        }
    }
    // ---- 16-bit copies of V_c and E_c for the apply (BF16 / FP16 storage)
    if constexpr (sizeof(T) == 4) {
        if ((h->store == HODLR_BF16 || h->store == HODLR_FP16) && rc > 0) {
            const int nn = 1 << c;
            const float *Vf = reinterpret_cast<const float *>(h->Vl[c]);
            const float *Ef = reinterpret_cast<const float *>(h->El[c]);
            const int64_t *bd = h->d_bounds;
            if (h->store == HODLR_BF16) {
                __nv_bfloat16 *Vq = reinterpret_cast<__nv_bfloat16 *>(h->Vql[c]);
                __nv_bfloat16 *Eq = reinterpret_cast<__nv_bfloat16 *>(h->Eql[c]);
                Pl->ops.push_back([=](cudaStream_t st) {
                    quantize_kernel<__nv_bfloat16><<<dim3(nn, rc), 256, 0, st>>>(Vf, Vq, ldn, 0, rc, bd, L, c, nullptr);
                    note_launch();
                    quantize_kernel<__nv_bfloat16><<<dim3(nn, 2 * rc), 256, 0, st>>>(Ef, Eq, ldn, 0, 2 * rc, bd, L, c,
                                                                                  nullptr);
                    note_launch();
                    HODLR_TRY_CUDA(cudaGetLastError());
                    return HODLR_OK;
                });
            } else {
                __half *Vq = reinterpret_cast<__half *>(h->Vql[c]);
                __half *Eq = reinterpret_cast<__half *>(h->Eql[c]);
                float *vs = h->vscale[c], *es = h->escale[c];
                Pl->ops.push_back([=](cudaStream_t st) {
                    quantize_kernel<__half><<<dim3(nn, rc), 256, 0, st>>>(Vf, Vq, ldn, 0, rc, bd, L, c, vs);
                    note_launch();
                    quantize_kernel<__half><<<dim3(nn, 2 * rc), 256, 0, st>>>(Ef, Eq, ldn, 0, 2 * rc, bd, L, c, es);
                    note_launch();
                    HODLR_TRY_CUDA(cudaGetLastError());
                    return HODLR_OK;
                });
            }
        }
    }
    // one upload of this share's descriptors
    Pl->dbytes = std::max<size_t>(Pl->blob.size(), 256);
    Pl->dblob = reinterpret_cast<char *>(dalloc(cx, Pl->dbytes, s));
    if (!Pl->dblob) {
        set_error("factor plan: out of device memory for descriptors");
        return HODLR_OUT_OF_MEMORY;
    }
    if (!Pl->blob.empty())
        HODLR_TRY_CUDA(cudaMemcpyAsync(Pl->dblob, Pl->blob.data(), Pl->blob.size(), cudaMemcpyHostToDevice, s));
    return HODLR_OK;
}

}  // namespace

template <typename T, typename TI>
hodlr_status gemm_batched(hodlr_ctx *c, const GemmDesc<T, TI> *d_desc, int nbatch, int maxM, int maxN,
                          int maxK, int transA, T alpha, cudaStream_t s) {
    if (nbatch > 65535) {
        hodlr::set_error("gemm_batched: too many batches (%d)", nbatch);
        return HODLR_RANGE;
    }
    const int64_t want = 2LL * std::max(1, c->num_sms);
    // 64-wide tiles unless that leaves most of the GPU idle
    int bm = 64;
    if ((int64_t)((maxM + 63) / 64) * ((maxN + 63) / 64) * nbatch < c->num_sms) bm = 32;
    const int tm = (maxM + bm - 1) / bm, tn = (maxN + bm - 1) / bm;
    const int64_t tiles = (int64_t)tm * tn * nbatch;
    int splitK = 1;
    if (tiles < want) splitK = (int)std::min<int64_t>((want + tiles - 1) / tiles, std::max(1, maxK / 64));
    splitK = std::max(1, std::min(splitK, 64));
    if ((int64_t)nbatch * splitK > 65535) splitK = std::max(1, 65535 / nbatch);
    dim3 grid(tn, tm, nbatch * splitK);
    if (bm == 64)
        gemm_batched_kernel<T, TI, 64><<<grid, GB_THREADS, 0, s>>>(d_desc, transA, alpha, splitK);
    else
        gemm_batched_kernel<T, TI, 32><<<grid, GB_THREADS, 0, s>>>(d_desc, transA, alpha, splitK);
    note_launch();
    HODLR_TRY_CUDA(cudaGetLastError());
    return HODLR_OK;
}

template hodlr_status gemm_batched<float, float>(hodlr_ctx *, const GemmDesc<float> *, int, int, int, int, int,
                                                 float, cudaStream_t);
template hodlr_status gemm_batched<double, double>(hodlr_ctx *, const GemmDesc<double> *, int, int, int, int, int,
                                                   double, cudaStream_t);
template hodlr_status gemm_batched<double, float>(hodlr_ctx *, const GemmDesc<double, float> *, int, int, int,
                                                  int, int, double, cudaStream_t);

namespace {

template <typename T>
hodlr_status leaf_inverses_typed(hodlr_t *h, cudaStream_t s) {
    const int L = h->L, nleaf = 1 << L;
    const int64_t bmax = h->bmax;
    T *Kinv = reinterpret_cast<T *>(h->leafinv);
    // work matrices are needed only by the global-memory variant (large leaves)
    T *work = nullptr;
    if (gj_needs_work<T>((int)bmax)) {
        work = reinterpret_cast<T *>(own(h, (size_t)nleaf * 2 * bmax * bmax * sizeof(T), s));
        if (!work) return HODLR_OUT_OF_MEMORY;
    }
    std::vector<GJDesc<T>> gd(nleaf);
    for (int i = 0; i < nleaf; ++i) {
        const int64_t r0 = h->bounds[i], m = h->bounds[i + 1] - r0;
        gd[i] = GJDesc<T>{h->A + r0 * h->lda + r0, h->lda, nullptr, 0,
                          work ? work + (size_t)i * 2 * bmax * bmax : nullptr, Kinv + (size_t)i * bmax * bmax,
                          bmax, (int)m};
    }
    GJDesc<T> *dd = reinterpret_cast<GJDesc<T> *>(own(h, gd.size() * sizeof(GJDesc<T>), s));
    if (!dd) return HODLR_OUT_OF_MEMORY;
    HODLR_TRY_CUDA(cudaMemcpyAsync(dd, gd.data(), gd.size() * sizeof(GJDesc<T>), cudaMemcpyHostToDevice, s));
    return launch_gj<T>(h->ctx, dd, nleaf, (int)bmax, s);
}

}  // namespace

hodlr_status leaf_inverses(hodlr_t *h, cudaStream_t s) {
    if (h->prec == HODLR_FP64) return leaf_inverses_typed<double>(h, s);
    return leaf_inverses_typed<float>(h, s);
}

hodlr_status plan_level(hodlr_t *h, int c, cudaStream_t s) {
    if (!h->plan) {
        h->plan = new FactorPlan();
        h->plan->lv.resize(h->L + 1);
    }
    LevelPlan *P = &h->plan->lv[c];
    if (!P->ops.empty()) return HODLR_OK;
    return (h->prec == HODLR_FP64) ? plan_level_typed<double>(h, P, c, s) : plan_level_typed<float>(h, P, c, s);
}

hodlr_status run_level(hodlr_t *h, int c, cudaStream_t s, const cudaEvent_t *share_done) {
    if (!h->plan || c >= (int)h->plan->lv.size()) {
        set_error("factor: level %d was not planned", c);
        return HODLR_INVALID_ARG;
    }
    const LevelPlan &P = h->plan->lv[c];
    size_t w = 0;
    for (size_t i = 0; i < P.ops.size(); ++i) {
        for (; w < P.waits.size() && P.waits[w].first == i; ++w)
            if (share_done) HODLR_TRY_CUDA(cudaStreamWaitEvent(s, share_done[P.waits[w].second], 0));
        HODLR_TRY(P.ops[i](s));
    }
    return HODLR_OK;
}

void free_plan(hodlr_t *h, cudaStream_t s) {
    if (!h->plan) return;
    for (auto &P : h->plan->lv) {
        if (P.gexec) cudaGraphExecDestroy(P.gexec);
        if (P.ggraph) cudaGraphDestroy(P.ggraph);
        if (P.work) dfree(h->ctx, P.work, P.work_bytes, s);
        if (P.dblob) dfree(h->ctx, P.dblob, P.dbytes, s);
    }
    delete h->plan;
    h->plan = nullptr;
}

hodlr_status factor_impl(hodlr_t *h, cudaStream_t s) {
    for (int c = h->L; c >= 1; --c) HODLR_TRY(run_level(h, c, s, nullptr));
    return HODLR_OK;
}

}  // namespace hodlr
