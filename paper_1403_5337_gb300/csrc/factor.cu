// Recursive Woodbury factorisation of a HODLR matrix, level-synchronous
// (Sec. 4.3, Factorize steps 2-5; Sec. 4.2 eqs. Schur and y).
//
// Layout: D and V are ldn x Wtot column-major; the columns of level l occupy
// [coff(l), coff(l) + rp(l)).  Row block "node" of level l in D first holds
// U_node (the Z stack of the paper: every row carries the U columns of all its
// ancestors' blocks), and after factorisation d_node = K_node^-1 U_node.
//
//  1. leaves:  D(leaf rows, :) <- K_leaf^-1 Z(leaf rows, :)          (explicit inverse)
//  2. for l = L-1 .. 0, children c = l + 1:
//       Y_child = V(child rows, blk c)^T D(child rows, 0 : coff(c)+rp(c))
//       S_node  = [[I, P], [Q, I]],  P = Y_alpha(:, blk c) = V_ba^T d_alpha,
//                                     Q = Y_beta (:, blk c) = V_ab^T d_beta
//       S^-1    = [[M^-1, -M^-1 P], [-Q M^-1, I + Q M^-1 P]],  M = I - P Q
//       (l >= 1) D(alpha, 0:coff(c)) -= d_alpha * (S^-1 [Y_alpha; Y_beta])(rp:2rp, :)
//                D(beta,  0:coff(c)) -= d_beta  * (S^-1 [Y_alpha; Y_beta])(0:rp, :)
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
constexpr int GB_M = 64, GB_N = 64, GB_K = 16, GB_THREADS = 256;

template <typename T>
__global__ void __launch_bounds__(GB_THREADS)
    gemm_batched_kernel(const GemmDesc<T> *__restrict__ descs, int transA, T alpha, int splitK) {
    const GemmDesc<T> d = descs[blockIdx.z / splitK];
    const int kz = blockIdx.z % splitK;
    const int m0 = blockIdx.y * GB_M, n0 = blockIdx.x * GB_N;
    if (m0 >= d.M || n0 >= d.N || d.K <= 0) return;
    const int kper = ((d.K + splitK - 1) / splitK + GB_K - 1) / GB_K * GB_K;
    const int kbeg = kz * kper;
    const int kend = min(d.K, kbeg + kper);
    if (kbeg >= kend) return;
    __shared__ T As[GB_K][GB_M + 1];
    __shared__ T Bs[GB_K][GB_N + 1];
    const int tid = threadIdx.x;
    const int ty = tid & 15, tx = tid >> 4;
    T acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
    for (int k0 = kbeg; k0 < kend; k0 += GB_K) {
        for (int e = tid; e < GB_M * GB_K; e += GB_THREADS) {
            int i, kk;
            T v = T(0);
            if (!transA) {
                i = e % GB_M;
                kk = e / GB_M;
                if (m0 + i < d.M && k0 + kk < kend) v = d.A[(int64_t)(m0 + i) + (int64_t)(k0 + kk) * d.lda];
            } else {
                kk = e % GB_K;
                i = e / GB_K;
                if (m0 + i < d.M && k0 + kk < kend) v = d.A[(int64_t)(k0 + kk) + (int64_t)(m0 + i) * d.lda];
            }
            As[kk][i] = v;
        }
        for (int e = tid; e < GB_N * GB_K; e += GB_THREADS) {
            int kk = e % GB_K, j = e / GB_K;
            T v = T(0);
            if (n0 + j < d.N && k0 + kk < kend) v = d.B[(int64_t)(k0 + kk) + (int64_t)(n0 + j) * d.ldb];
            Bs[kk][j] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GB_K; ++kk) {
            T a[4], b[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                a[q] = As[kk][ty + 16 * q];
                b[q] = Bs[kk][tx + 16 * q];
            }
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[p][q] = fma(a[p], b[q], acc[p][q]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int j = n0 + tx + 16 * q;
        if (j >= d.N) continue;
#pragma unroll
        for (int p = 0; p < 4; ++p) {
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
};

constexpr int GJ_THREADS = 512;

template <typename T>
__global__ void __launch_bounds__(GJ_THREADS) gj_inverse_kernel(const GJDesc<T> *__restrict__ descs,
                                                                int *status) {
    const GJDesc<T> g = descs[blockIdx.x];
    const int b = g.b, tid = threadIdx.x;
    if (b <= 0) return;
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

template <typename T>
__global__ void set_identity_kernel(T *M, int64_t ld, int n, int count, int64_t stride) {
    const int m = blockIdx.y;
    if (m >= count) return;
    T *P = M + m * stride;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)n * n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = e / n, i = e % n;
        P[i + j * ld] = (i == j) ? T(1) : T(0);
    }
}

template <typename T>
__global__ void zero_kernel(T *p, int64_t count) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count;
         e += (int64_t)gridDim.x * blockDim.x)
        p[e] = T(0);
}

template <typename T>
hodlr_status zero(T *p, int64_t count, cudaStream_t s) {
    if (count <= 0) return HODLR_OK;
    int blocks = (int)std::min<int64_t>((count + 255) / 256, 4096);
    zero_kernel<T><<<blocks, 256, 0, s>>>(p, count);
    HODLR_TRY_CUDA(cudaGetLastError());
    return HODLR_OK;
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
    if (b <= 0) return;
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

// Gauss-Jordan inversion with the matrix held in registers: 512 threads as a
// 16 x 32 grid, thread (ty, tx) owns rows ty + 16 p (p < MR) and columns
// tx + 32 q (q < MC).  Per step only pivot column k and pivot row k pass
// through shared memory (the row swap too), so each step costs MR + MC shared
// loads and MR * MC FMAs per thread.  Same pivot rule and the same in-place
// update as gj_inverse_smem_kernel.  Register slots are selected with unrolled
// predicated loops, never by a run-time index.
constexpr int GJR_TY = 16, GJR_TX = 32, GJR_THREADS = GJR_TY * GJR_TX;

template <typename T, int MR, int MC>
__global__ void __launch_bounds__(GJR_THREADS, 1) gj_inverse_reg_kernel(const GJDesc<T> *__restrict__ descs,
                                                                       int *status) {
    const GJDesc<T> g = descs[blockIdx.x];
    const int b = g.b;
    if (b <= 0) return;
    const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
    __shared__ T colk[MR * GJR_TY];
    __shared__ T rowk[MC * GJR_TX];
    __shared__ T rowa[MC * GJR_TX];
    __shared__ T rowb[MC * GJR_TX];
    __shared__ int orig[MR * GJR_TY];
    __shared__ int s_p, s_fail;
    T a[MR][MC];
#pragma unroll
    for (int p = 0; p < MR; ++p)
#pragma unroll
        for (int q = 0; q < MC; ++q) {
            const int i = ty + GJR_TY * p, j = tx + GJR_TX * q;
            T v = T(0);
            if (i < b && j < b)
                v = g.srcA ? dev::from_double<T>(g.srcA[(int64_t)i * g.lda + j]) : g.srcM[i + (int64_t)j * g.ldm];
            a[p][q] = v;
        }
    for (int i = tid; i < b; i += GJR_THREADS) orig[i] = i;
    if (tid == 0) s_fail = 0;
    __syncthreads();
    for (int k = 0; k < b; ++k) {
        const int kq = k / GJR_TX, kx = k % GJR_TX;
        // 1. column k to shared memory
        if (tx == kx) {
#pragma unroll
            for (int q = 0; q < MC; ++q)
                if (q == kq) {
#pragma unroll
                    for (int p = 0; p < MR; ++p) {
                        const int i = ty + GJR_TY * p;
                        if (i < b) colk[i] = a[p][q];
                    }
                }
        }
        __syncthreads();
        // 2. pivot row: argmax_{i >= k} |colk[i]|, lowest row on ties
        if (ty == 0) {
            T bv = T(-1);
            int bi = INT_MAX;
            for (int i = k + tx; i < b; i += 32) {
                const T v = fabs(colk[i]);
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
            if (tx == 0) {
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
        const int pr = s_p;
        // 3. swap rows k and pr through shared memory
        if (pr != k) {
            const int ky = k % GJR_TY, kp = k / GJR_TY, py = pr % GJR_TY, pp = pr / GJR_TY;
            if (ty == ky)
#pragma unroll
                for (int p = 0; p < MR; ++p)
                    if (p == kp)
#pragma unroll
                        for (int q = 0; q < MC; ++q) rowa[tx + GJR_TX * q] = a[p][q];
            if (ty == py)
#pragma unroll
                for (int p = 0; p < MR; ++p)
                    if (p == pp)
#pragma unroll
                        for (int q = 0; q < MC; ++q) rowb[tx + GJR_TX * q] = a[p][q];
            __syncthreads();
            if (ty == ky)
#pragma unroll
                for (int p = 0; p < MR; ++p)
                    if (p == kp)
#pragma unroll
                        for (int q = 0; q < MC; ++q) a[p][q] = rowb[tx + GJR_TX * q];
            if (ty == py)
#pragma unroll
                for (int p = 0; p < MR; ++p)
                    if (p == pp)
#pragma unroll
                        for (int q = 0; q < MC; ++q) a[p][q] = rowa[tx + GJR_TX * q];
            if (tid == 0) {
                const T t = colk[k];
                colk[k] = colk[pr];
                colk[pr] = t;
            }
        }
        __syncthreads();
        // 4. scaled pivot row to shared memory
        const T d = T(1) / colk[k];
        {
            const int ky = k % GJR_TY, kp = k / GJR_TY;
            if (ty == ky)
#pragma unroll
                for (int p = 0; p < MR; ++p)
                    if (p == kp)
#pragma unroll
                        for (int q = 0; q < MC; ++q) {
                            const int j = tx + GJR_TX * q;
                            rowk[j] = (j == k) ? d : a[p][q] * d;
                        }
        }
        __syncthreads();
        // 5. eliminate column k from every other row: a -= colk * rowk everywhere
        // (rows beyond b hold zeros and stay zero), then overwrite the pivot row
        // with rowk and the pivot column with -colk d.
        T rk[MC];
#pragma unroll
        for (int q = 0; q < MC; ++q) rk[q] = rowk[tx + GJR_TX * q];
#pragma unroll
        for (int p = 0; p < MR; ++p) {
            const int i = ty + GJR_TY * p;
            const T ci = (i < b) ? colk[i] : T(0);
#pragma unroll
            for (int q = 0; q < MC; ++q) a[p][q] = fma(-ci, rk[q], a[p][q]);
            if (tx == kx) {
#pragma unroll
                for (int q = 0; q < MC; ++q)
                    if (q == kq) a[p][q] = -ci * d;
            }
        }
        if (ty == k % GJR_TY) {
#pragma unroll
            for (int p = 0; p < MR; ++p)
                if (p == k / GJR_TY) {
#pragma unroll
                    for (int q = 0; q < MC; ++q) a[p][q] = rk[q];
                }
        }
        __syncthreads();
    }
    if (s_fail) {
        if (tid == 0) atomicOr(status, ST_SINGULAR);
        return;
    }
    // A^-1 = (PA)^-1 P: column q of the work matrix is column orig[q] of A^-1
#pragma unroll
    for (int p = 0; p < MR; ++p)
#pragma unroll
        for (int q = 0; q < MC; ++q) {
            const int i = ty + GJR_TY * p, j = tx + GJR_TX * q;
            if (i < b && j < b) g.out[i + (int64_t)orig[j] * g.ldo] = a[p][q];
        }
}

template <typename T, int MR, int MC>
hodlr_status launch_gj_reg(hodlr_ctx *c, const GJDesc<T> *dd, int count, cudaStream_t s) {
    gj_inverse_reg_kernel<T, MR, MC><<<count, GJR_THREADS, 0, s>>>(dd, c->d_status);
    HODLR_TRY_CUDA(cudaGetLastError());
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

// Which Gauss-Jordan variant launch_gj picks for matrices up to bmax: registers,
// shared memory, or the global-memory kernel (the only one that needs GJDesc::work).
template <typename T>
bool gj_needs_work(int bmax) {
    if (bmax <= 128) return false;
    if (sizeof(T) == 4 && bmax <= 192) return false;
    return gjs_smem<T>(bmax) > GJS_SMEM_MAX;
}

template <typename T>
hodlr_status launch_gj(hodlr_ctx *c, const GJDesc<T> *dd, int count, int bmax, cudaStream_t s) {
    if (bmax <= 32) return launch_gj_reg<T, 2, 1>(c, dd, count, s);
    if (bmax <= 64) return launch_gj_reg<T, 4, 2>(c, dd, count, s);
    if (bmax <= 96) return launch_gj_reg<T, 6, 3>(c, dd, count, s);
    if (bmax <= 128) return launch_gj_reg<T, 8, 4>(c, dd, count, s);
    if constexpr (sizeof(T) == 4) {   // FP64 tiles beyond 128 would spill registers
        if (bmax <= 160) return launch_gj_reg<T, 10, 5>(c, dd, count, s);
        if (bmax <= 192) return launch_gj_reg<T, 12, 6>(c, dd, count, s);
    }
    if (gjs_smem<T>(bmax) <= GJS_SMEM_MAX) {
        const size_t sm = gjs_smem<T>(bmax);
        HODLR_TRY_CUDA(cudaFuncSetAttribute(gj_inverse_smem_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)sm));
        gj_inverse_smem_kernel<T><<<count, GJS_THREADS, sm, s>>>(dd, c->d_status);
        HODLR_TRY_CUDA(cudaGetLastError());
        return HODLR_OK;
    }
    size_t sm = 3 * (size_t)bmax * sizeof(T);
    HODLR_TRY_CUDA(cudaFuncSetAttribute(gj_inverse_kernel<T>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    gj_inverse_kernel<T><<<count, GJ_THREADS, sm, s>>>(dd, c->d_status);
    HODLR_TRY_CUDA(cudaGetLastError());
    return HODLR_OK;
}

}  // namespace

// The factorisation is planned once, when the HODLR matrix is built: every
// launch of the level-synchronous sweep is recorded with its arguments, and all
// batched-GEMM and inversion descriptors are laid out in one blob that is
// uploaded in a single copy.  hodlr_factor then only replays the launches, with
// no host-device transfer on the stream.
struct FactorPlan {
    std::vector<std::function<hodlr_status(cudaStream_t)>> ops;
    std::vector<char> blob;
    char *dblob = nullptr;
    size_t dbytes = 0;
    void *work = nullptr;
    size_t work_bytes = 0;

    size_t put(const void *p, size_t bytes) {
        const size_t off = (blob.size() + 255) & ~size_t(255);
        blob.resize(off + bytes);
        std::memcpy(blob.data() + off, p, bytes);
        return off;
    }
};

namespace {

template <typename T>
struct Rec {
    hodlr_ctx *c;
    FactorPlan *P;
    void gj(const std::vector<GJDesc<T>> &hd) {
        if (hd.empty()) return;
        int bmax = 0;
        for (auto &g : hd) bmax = std::max(bmax, g.b);
        const size_t off = P->put(hd.data(), hd.size() * sizeof(GJDesc<T>));
        const int cnt = (int)hd.size();
        hodlr_ctx *cc = c;
        FactorPlan *PP = P;
        P->ops.push_back([=](cudaStream_t s) {
            return launch_gj<T>(cc, reinterpret_cast<const GJDesc<T> *>(PP->dblob + off), cnt, bmax, s);
        });
    }
    void gemm(const std::vector<GemmDesc<T>> &hd, int transA, T alpha) {
        if (hd.empty()) return;
        int maxM = 0, maxN = 0, maxK = 0;
        for (auto &g : hd) {
            maxM = std::max(maxM, g.M);
            maxN = std::max(maxN, g.N);
            maxK = std::max(maxK, g.K);
        }
        if (maxM == 0 || maxN == 0 || maxK == 0) return;
        const size_t off = P->put(hd.data(), hd.size() * sizeof(GemmDesc<T>));
        const int cnt = (int)hd.size();
        hodlr_ctx *cc = c;
        FactorPlan *PP = P;
        P->ops.push_back([=](cudaStream_t s) {
            return gemm_batched<T>(cc, reinterpret_cast<const GemmDesc<T> *>(PP->dblob + off), cnt, maxM, maxN,
                                   maxK, transA, alpha, s);
        });
    }
    void zero_(T *p, int64_t count) {
        P->ops.push_back([=](cudaStream_t s) { return zero<T>(p, count, s); });
    }
    void identity(T *M, int64_t ld, int n, int count, int64_t stride) {
        P->ops.push_back([=](cudaStream_t s) {
            dim3 grid(std::max(1, std::min(64, (n * n + 255) / 256)), count);
            set_identity_kernel<T><<<grid, 256, 0, s>>>(M, ld, n, count, stride);
            HODLR_TRY_CUDA(cudaGetLastError());
            return HODLR_OK;
        });
    }
    void memset2d(T *p, int64_t pitch_elems, int64_t width_elems, int64_t height) {
        P->ops.push_back([=](cudaStream_t s) {
            HODLR_TRY_CUDA(cudaMemset2DAsync(p, pitch_elems * sizeof(T), 0, width_elems * sizeof(T), height, s));
            return HODLR_OK;
        });
    }
    void copy(T *dst, const T *src, int64_t count) {
        P->ops.push_back([=](cudaStream_t s) {
            HODLR_TRY_CUDA(cudaMemcpyAsync(dst, src, count * sizeof(T), cudaMemcpyDeviceToDevice, s));
            return HODLR_OK;
        });
    }
};

template <typename T>
hodlr_status plan_typed(hodlr_t *h, FactorPlan *Pl, cudaStream_t s) {
    hodlr_ctx *c = h->ctx;
    const int L = h->L;
    const int64_t ldn = h->ldn, W = h->Wtot;
    T *D = reinterpret_cast<T *>(h->D);
    T *V = reinterpret_cast<T *>(h->V);
    const int nleaf = 1 << L;
    auto node_range = [&](int l, int i, int64_t &r0, int64_t &m) {
        r0 = h->bounds[(size_t)i << (L - l)];
        m = h->bounds[(size_t)(i + 1) << (L - l)] - r0;
    };
    // ---- workspace sizing
    const int64_t bmax = h->bmax;
    size_t need = 0;
    size_t lvl_max = 0;
    for (int l = 0; l < L; ++l) {
        const int cch = l + 1;
        const int rp = h->lv[cch].rp;
        const int64_t Wc = h->lv[cch].coff + rp;
        const int nn = 1 << l;
        size_t y = (size_t)(2 * nn) * rp * Wc;                   // Y per child
        size_t yv = (size_t)nn * 2 * rp * h->lv[cch].coff;       // S^-1 W per node
        size_t mm = (size_t)nn * rp * rp;                        // M per node
        size_t gw = (size_t)nn * 2 * rp * rp;                    // GJ work per node
        lvl_max = std::max(lvl_max, (y + yv + mm + gw) * sizeof(T) + 4096);
    }
    need += lvl_max + 4096;
    Pl->work = dalloc(c, need, s);
    if (!Pl->work) {
        set_error("factor plan: out of device memory (%zu bytes)", need);
        return HODLR_OUT_OF_MEMORY;
    }
    Pl->work_bytes = need;
    char *wp = reinterpret_cast<char *>(Pl->work);
    auto carve = [&](size_t bytes) {
        char *p = wp;
        wp += (bytes + 255) & ~size_t(255);
        return p;
    };
    char *lvl = carve(lvl_max);
    Rec<T> rec{c, Pl};
    const T *U = reinterpret_cast<const T *>(h->U);

    // ---- 1. leaf inverses: computed by hodlr_build (they depend on A only), while
    // the off-diagonal blocks are being compressed
    T *Kinv = reinterpret_cast<T *>(h->leafinv);
    // ---- 2. leaf stack: D = Kinv_leaf * U (all columns).  U is left intact, so
    // the factorisation can be repeated.
    if (W > 0) {
        rec.zero_(D, ldn * W);
        std::vector<GemmDesc<T>> gd(nleaf);
        for (int i = 0; i < nleaf; ++i) {
            int64_t r0, m;
            node_range(L, i, r0, m);
            gd[i] = GemmDesc<T>{Kinv + (size_t)i * bmax * bmax, U + r0, D + r0, bmax, ldn, ldn,
                                (int)m, (int)W, (int)m};
        }
        rec.gemm(gd, 0, T(1));
    }
    // ---- 3. levels, bottom-up
    for (int l = L - 1; l >= 0; --l) {
        const int cch = l + 1;
        const int rp = h->lv[cch].rp;
        const int64_t coffc = h->lv[cch].coff;
        const int64_t Wc = coffc + rp;
        const int nn = 1 << l;
        const int nch = 2 * nn;
        T *Sinv = reinterpret_cast<T *>(h->Sinv[l]);
        const int64_t s2 = 2 * (int64_t)rp;
        if (rp == 0) continue;
        char *lp = lvl;
        auto lcarve = [&](size_t bytes) {
            char *p = lp;
            lp += (bytes + 255) & ~size_t(255);
            return p;
        };
        T *Y = reinterpret_cast<T *>(lcarve((size_t)nch * rp * Wc * sizeof(T)));
        T *Yv = reinterpret_cast<T *>(lcarve((size_t)nn * s2 * std::max<int64_t>(coffc, 1) * sizeof(T)));
        T *M = reinterpret_cast<T *>(lcarve((size_t)nn * rp * rp * sizeof(T)));
        T *gw = reinterpret_cast<T *>(lcarve((size_t)nn * 2 * rp * rp * sizeof(T)));
        // (a) Y_child = V(child, blk c)^T D(child, 0:Wc)
        rec.zero_(Y, (int64_t)nch * rp * Wc);
        {
            std::vector<GemmDesc<T>> gd(nch);
            for (int i = 0; i < nch; ++i) {
                int64_t r0, m;
                node_range(cch, i, r0, m);
                gd[i] = GemmDesc<T>{V + coffc * ldn + r0, D + r0, Y + (size_t)i * rp * Wc, ldn, ldn,
                                    rp, rp, (int)Wc, (int)m};
            }
            rec.gemm(gd, 1, T(1));
        }
        // (b) M = I - P Q per node
        {
            rec.identity(M, rp, rp, nn, (int64_t)rp * rp);
            std::vector<GemmDesc<T>> gd(nn);
            for (int i = 0; i < nn; ++i) {
                const T *P = Y + (size_t)(2 * i) * rp * Wc + coffc * rp;
                const T *Q = Y + (size_t)(2 * i + 1) * rp * Wc + coffc * rp;
                gd[i] = GemmDesc<T>{P, Q, M + (size_t)i * rp * rp, rp, rp, rp, rp, rp, rp};
            }
            rec.gemm(gd, 0, T(-1));
        }
        // (c) M^-1 into the top-left block of S^-1
        {
            std::vector<GJDesc<T>> gd(nn);
            for (int i = 0; i < nn; ++i)
                gd[i] = GJDesc<T>{nullptr, 0, M + (size_t)i * rp * rp, rp, gw + (size_t)i * 2 * rp * rp,
                                  Sinv + (size_t)i * s2 * s2, s2, rp};
            rec.gj(gd);
        }
        // (d) the other three blocks of S^-1
        {
            // TR = -M^-1 P ; BL = -Q M^-1 (zeroed first), BR = I - Q TR
            for (int i = 0; i < nn; ++i) {
                T *S = Sinv + (size_t)i * s2 * s2;
                rec.memset2d(S + rp * s2, s2, rp, rp);
                rec.memset2d(S + rp, s2, rp, rp);
            }
            rec.identity(Sinv + rp + rp * s2, s2, rp, nn, s2 * s2);
            std::vector<GemmDesc<T>> g1(nn), g2(nn), g3(nn);
            for (int i = 0; i < nn; ++i) {
                T *S = Sinv + (size_t)i * s2 * s2;
                const T *P = Y + (size_t)(2 * i) * rp * Wc + coffc * rp;
                const T *Q = Y + (size_t)(2 * i + 1) * rp * Wc + coffc * rp;
                g1[i] = GemmDesc<T>{S, P, S + rp * s2, s2, rp, s2, rp, rp, rp};        // TR -= Minv P
                g2[i] = GemmDesc<T>{Q, S, S + rp, rp, s2, s2, rp, rp, rp};              // BL -= Q Minv
                g3[i] = GemmDesc<T>{Q, S + rp * s2, S + rp + rp * s2, rp, s2, s2, rp, rp, rp};  // BR -= Q TR
            }
            rec.gemm(g1, 0, T(-1));
            rec.gemm(g2, 0, T(-1));
            rec.gemm(g3, 0, T(-1));
        }
        // (e) update the ancestor columns (levels 1..l) for l >= 1
        if (l >= 1 && coffc > 0) {
            rec.zero_(Yv, (int64_t)nn * s2 * coffc);
            std::vector<GemmDesc<T>> ga(2 * nn);
            for (int i = 0; i < nn; ++i) {
                T *S = Sinv + (size_t)i * s2 * s2;
                const T *Ya = Y + (size_t)(2 * i) * rp * Wc;
                const T *Yb = Y + (size_t)(2 * i + 1) * rp * Wc;
                T *out = Yv + (size_t)i * s2 * coffc;
                ga[2 * i] = GemmDesc<T>{S, Ya, out, s2, rp, s2, (int)s2, (int)coffc, rp};
                ga[2 * i + 1] = GemmDesc<T>{S + rp * s2, Yb, out, s2, rp, s2, (int)s2, (int)coffc, rp};
            }
            // the two halves accumulate into the same output: run them as two launches
            std::vector<GemmDesc<T>> gA(nn), gB(nn);
            for (int i = 0; i < nn; ++i) {
                gA[i] = ga[2 * i];
                gB[i] = ga[2 * i + 1];
            }
            rec.gemm(gA, 0, T(1));
            rec.gemm(gB, 0, T(1));
            std::vector<GemmDesc<T>> gu(nch);
            for (int i = 0; i < nn; ++i) {
                int64_t ra, ma, rb, mb;
                node_range(cch, 2 * i, ra, ma);
                node_range(cch, 2 * i + 1, rb, mb);
                const T *yv = Yv + (size_t)i * s2 * coffc;
                // alpha rows: -= d_alpha * y2 ; beta rows: -= d_beta * y1
                gu[2 * i] = GemmDesc<T>{D + coffc * ldn + ra, yv + rp, D + ra, ldn, s2, ldn,
                                        (int)ma, (int)coffc, rp};
                gu[2 * i + 1] = GemmDesc<T>{D + coffc * ldn + rb, yv, D + rb, ldn, s2, ldn,
                                            (int)mb, (int)coffc, rp};
            }
            rec.gemm(gu, 0, T(-1));
        }
    }
    // 16-bit copies of V and d for the apply (BF16 / FP16 storage)
    if constexpr (sizeof(T) == 4) {
        if (h->store == HODLR_BF16 || h->store == HODLR_FP16) {
            for (int l = 1; l <= L; ++l) {
                const int rp = h->lv[l].rp;
                if (rp == 0) continue;
                const int64_t coff = h->lv[l].coff;
                const int nn = 1 << l;
                const float *Vf = reinterpret_cast<const float *>(h->V);
                const float *Df = reinterpret_cast<const float *>(h->D);
                const int64_t *bd = h->d_bounds;
                if (h->store == HODLR_BF16) {
                    __nv_bfloat16 *Vq = reinterpret_cast<__nv_bfloat16 *>(h->Vq);
                    __nv_bfloat16 *Dq = reinterpret_cast<__nv_bfloat16 *>(h->Dq);
                    Pl->ops.push_back([=](cudaStream_t s) {
                        quantize_kernel<__nv_bfloat16><<<dim3(nn, rp), 256, 0, s>>>(Vf, Vq, ldn, coff, rp, bd, L, l,
                                                                                     nullptr);
                        quantize_kernel<__nv_bfloat16><<<dim3(nn, rp), 256, 0, s>>>(Df, Dq, ldn, coff, rp, bd, L, l,
                                                                                     nullptr);
                        HODLR_TRY_CUDA(cudaGetLastError());
                        return HODLR_OK;
                    });
                } else {
                    __half *Vq = reinterpret_cast<__half *>(h->Vq);
                    __half *Dq = reinterpret_cast<__half *>(h->Dq);
                    float *vs = h->vscale[l], *ds = h->dscale[l];
                    Pl->ops.push_back([=](cudaStream_t s) {
                        quantize_kernel<__half><<<dim3(nn, rp), 256, 0, s>>>(Vf, Vq, ldn, coff, rp, bd, L, l, vs);
                        quantize_kernel<__half><<<dim3(nn, rp), 256, 0, s>>>(Df, Dq, ldn, coff, rp, bd, L, l, ds);
                        HODLR_TRY_CUDA(cudaGetLastError());
                        return HODLR_OK;
                    });
                }
            }
        }
    }
    // one upload of every descriptor (the caller synchronises before factor runs)
    Pl->dbytes = std::max<size_t>(Pl->blob.size(), 256);
    Pl->dblob = reinterpret_cast<char *>(dalloc(c, Pl->dbytes, s));
    if (!Pl->dblob) {
        set_error("factor plan: out of device memory for descriptors");
        return HODLR_OUT_OF_MEMORY;
    }
    if (!Pl->blob.empty())
        HODLR_TRY_CUDA(cudaMemcpyAsync(Pl->dblob, Pl->blob.data(), Pl->blob.size(), cudaMemcpyHostToDevice, s));
    return HODLR_OK;
}

}  // namespace

template <typename T>
hodlr_status gemm_batched(hodlr_ctx *c, const GemmDesc<T> *d_desc, int nbatch, int maxM, int maxN,
                          int maxK, int transA, T alpha, cudaStream_t s) {
    const int tm = (maxM + GB_M - 1) / GB_M, tn = (maxN + GB_N - 1) / GB_N;
    const int64_t tiles = (int64_t)tm * tn * nbatch;
    int splitK = 1;
    const int64_t want = 2LL * std::max(1, c->num_sms);
    if (tiles < want) splitK = (int)std::min<int64_t>((want + tiles - 1) / tiles, std::max(1, maxK / 128));
    splitK = std::max(1, std::min(splitK, 64));
    if ((int64_t)nbatch * splitK > 65535) splitK = std::max(1, 65535 / nbatch);
    if (nbatch > 65535) {
        hodlr::set_error("gemm_batched: too many batches (%d)", nbatch);
        return HODLR_RANGE;
    }
    dim3 grid(tn, tm, nbatch * splitK);
    gemm_batched_kernel<T><<<grid, GB_THREADS, 0, s>>>(d_desc, transA, alpha, splitK);
    HODLR_TRY_CUDA(cudaGetLastError());
    return HODLR_OK;
}

template hodlr_status gemm_batched<float>(hodlr_ctx *, const GemmDesc<float> *, int, int, int, int, int,
                                          float, cudaStream_t);
template hodlr_status gemm_batched<double>(hodlr_ctx *, const GemmDesc<double> *, int, int, int, int, int,
                                           double, cudaStream_t);

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

hodlr_status plan_factor(hodlr_t *h, cudaStream_t s) {
    if (h->plan) return HODLR_OK;
    FactorPlan *P = new FactorPlan();
    hodlr_status st = (h->prec == HODLR_FP64) ? plan_typed<double>(h, P, s) : plan_typed<float>(h, P, s);
    h->plan = P;   // owned even on failure, released by free_plan
    return st;
}

void free_plan(hodlr_t *h, cudaStream_t s) {
    if (!h->plan) return;
    if (h->plan->work) dfree(h->ctx, h->plan->work, h->plan->work_bytes, s);
    if (h->plan->dblob) dfree(h->ctx, h->plan->dblob, h->plan->dbytes, s);
    delete h->plan;
    h->plan = nullptr;
}

hodlr_status factor_impl(hodlr_t *h, cudaStream_t s) {
    HODLR_TRY(plan_factor(h, s));
    for (auto &op : h->plan->ops) HODLR_TRY(op(s));
    return HODLR_OK;
}

}  // namespace hodlr
