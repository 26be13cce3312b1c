// FP64-accurate W = A Z on the BF16 tensor cores, for many right-hand sides.
//
// GMRES (Sec. 3) needs the product with the FP64 front A to FP64 accuracy.
// With one to a few right-hand sides it is a matrix-vector stream (the
// double-float kernel in gmres.cu); with tens it is a GEMM of n x n x s, and
// the FP32 pipes that kernel runs on become the limit.  Here every FP64 entry
// is split exactly into base-256 digits relative to a power of two shared by
// its row of A (column of Z):
//   a = 2^(e_i - 8) sum_p d_p 2^(-8p),  p = 0..6,  |d_p| <= 256, e_i the least
//   exponent with max_k |A(i,k)| < 2^e_i, the last digit rounded to nearest,
// so each digit times its 2^(-8p) is a BF16 number (8 significant bits), and
//   (A Z)(i,j) = 2^(e_i + f_j - 16) sum_{p,q} (A_p Z_q)(i,j).
// The slice products A_p Z_q run on the tensor cores with FP32 accumulation.
// Pairs of one level t = p + q have the same scale.  For t <= 3 their sum over
// 64 values of k, for t = 4 over 32, stays below 2^24 units of that scale
// (level 3: 64 (2 * 256 * 255 + 2 * 255^2) = 16,679,040 < 2^24), so those FP32
// sums are exact whatever rounding the tensor cores' accumulation uses; each is
// moved into a float pair (TwoSum) after its 64 (32) values of k.  The levels
// t = 5, 6 (below 2^-40 of the leading level) share one FP32 accumulator,
// moved into the pair every 32 values of k; pairs with t >= 7 (below 2^-56)
// are dropped.  The result is accurate to a few units of
// 2^-56 max|A(i,:)| max|Z(:,j)| per term.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>

#include "internal.cuh"

namespace hodlr {
namespace {

constexpr int S = OZ_SLICES;
constexpr int OZ_BM = 128;      // rows of A per CTA: 8 warps x 16
constexpr int OZ_BN = 32;       // right-hand sides per CTA: 4 MMA tiles of 8
constexpr int OZ_BK = 32;       // k per pipeline stage (two MMA k-steps of 16)
constexpr int OZ_FLUSH = 64;    // k per exact FP32 sum of the levels 0..3 (level 4: one stage)
constexpr int OZ_THREADS = 256;
constexpr int OZ_LDS = 40;      // shared row stride in BF16 (80 bytes: the 8 rows of an ldmatrix hit distinct banks)

struct OzStage {
    __nv_bfloat16 a[S][OZ_BM][OZ_LDS];
    __nv_bfloat16 z[S][OZ_BN][OZ_LDS];
};
constexpr size_t OZ_SMEM = 2 * sizeof(OzStage);
static_assert(OZ_SMEM <= 227 * 1024, "two stages must fit in shared memory");

inline int64_t oz_np(int64_t n) { return (n + OZ_BM - 1) / OZ_BM * OZ_BM; }
inline int64_t oz_kp(int64_t n) { return (n + OZ_FLUSH - 1) / OZ_FLUSH * OZ_FLUSH; }
inline int oz_sp(int s) { return (s + OZ_BN - 1) / OZ_BN * OZ_BN; }

__device__ __forceinline__ int exp_field(double a) {
    return (int)((unsigned long long)__double_as_longlong(a) >> 52) & 0x7FF;
}

// The digits of a relative to 2^e (|a| < 2^e, or a not finite: all zero),
// each already multiplied by its 2^(-8p), as BF16 (exact).
__device__ __forceinline__ void digits(double a, int e, __nv_bfloat16 (&out)[S]) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(a);
    const int ex = (int)(u >> 52) & 0x7FF;
    unsigned long long F = 0;   // round(|a| 2^(56 - e)) < 2^56 + 1
    if (ex != 0 && ex != 0x7FF) {
        const unsigned long long mant = (u & 0xFFFFFFFFFFFFFull) | (1ull << 52);
        const int sh = 1019 + e - ex;   // |a| 2^(56 - e) = mant 2^(-sh); sh >= -3 as |a| < 2^e
        if (sh <= 0)
            F = mant << (-sh);
        else if (sh < 54)
            F = (mant + (1ull << (sh - 1))) >> sh;
    }
    const float sg = (u >> 63) ? -1.f : 1.f;
    out[0] = __float2bfloat16_rn(sg * (float)(F >> 48));
#pragma unroll
    for (int p = 1; p < S; ++p) {
        const float scale = __int_as_float((127 - 8 * p) << 23);   // 2^(-8p)
        out[p] = __float2bfloat16_rn(sg * (float)((F >> (48 - 8 * p)) & 255u) * scale);
    }
}

// One warp per row of the padded np x kp slices: the row's exponent, then its
// digits (zero outside the n x n matrix).
__global__ void __launch_bounds__(256) oz_split_rows_kernel(const double *__restrict__ A, int64_t n, int64_t lda,
                                                            int64_t np, int64_t kp, __nv_bfloat16 *__restrict__ sl,
                                                            int *__restrict__ ea, int *status) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t i = (int64_t)blockIdx.x * 8 + warp;
    if (i >= np) return;
    const double *row = A + i * lda;
    int mx = 0, bad = 0;
    if (i < n)
        for (int64_t k = lane; k < n; k += 32) {
            const int ex = exp_field(row[k]);
            if (ex == 0x7FF)
                bad = 1;
            else
                mx = max(mx, ex);
        }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    bad = __any_sync(0xffffffffu, bad);
    const int e = mx - 1022;
    if (lane == 0) {
        ea[i] = e;
        if (bad) atomicOr(status, ST_NONFINITE);
    }
    for (int64_t k = lane; k < kp; k += 32) {
        __nv_bfloat16 d[S];
        digits((i < n && k < n) ? row[k] : 0.0, e, d);
#pragma unroll
        for (int p = 0; p < S; ++p) sl[((int64_t)p * np + i) * kp + k] = d[p];
    }
}

// One CTA per column of the padded Z slices (sp columns of kp digits each).
__global__ void __launch_bounds__(256) oz_split_cols_kernel(const double *__restrict__ Z, int64_t ldz, int64_t n,
                                                            int s, int64_t kp, int sp, __nv_bfloat16 *__restrict__ zs,
                                                            int *__restrict__ ez, int *status) {
    __shared__ int s_max, s_bad;
    const int j = blockIdx.x;
    if (threadIdx.x == 0) {
        s_max = 0;
        s_bad = 0;
    }
    __syncthreads();
    const double *col = Z + (int64_t)j * ldz;
    int mx = 0, bad = 0;
    if (j < s)
        for (int64_t k = threadIdx.x; k < n; k += blockDim.x) {
            const int ex = exp_field(col[k]);
            if (ex == 0x7FF)
                bad = 1;
            else
                mx = max(mx, ex);
        }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    bad = __any_sync(0xffffffffu, bad);
    if ((threadIdx.x & 31) == 0) {
        atomicMax(&s_max, mx);
        if (bad) atomicOr(&s_bad, 1);
    }
    __syncthreads();
    const int e = s_max - 1022;
    if (threadIdx.x == 0) {
        ez[j] = e;
        if (s_bad) atomicOr(status, ST_NONFINITE);
    }
    for (int64_t k = threadIdx.x; k < kp; k += blockDim.x) {
        __nv_bfloat16 d[S];
        digits((j < s && k < n) ? col[k] : 0.0, e, d);
#pragma unroll
        for (int p = 0; p < S; ++p) zs[((int64_t)p * sp + j) * kp + k] = d[p];
    }
}

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

__device__ __forceinline__ void ldsm_x4(uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3, const void *p) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(a));
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// hi + lo += x (TwoSum; x exact)
__device__ __forceinline__ void df_add(float &hi, float &lo, float x) {
    const float s = hi + x;
    const float bb = s - hi;
    lo += (hi - (s - bb)) + (x - bb);
    hi = s;
}

// W(0:n, n0:n0+32) for 128 rows of A per CTA.  Warp w owns rows 16w..16w+15 of
// the tile and all 32 columns (4 MMA tiles of 16 x 8).  Two cp.async stages of
// k = 32 (every slice of A's 128 rows and of Z's 32 columns).
__global__ void __launch_bounds__(OZ_THREADS, 1)
    oz_gemm_kernel(const __nv_bfloat16 *__restrict__ sl, const int *__restrict__ ea, int64_t np, int64_t kp,
                   const __nv_bfloat16 *__restrict__ zs, const int *__restrict__ ez, int sp, int64_t n, int s,
                   double *__restrict__ W, int64_t ldw) {
    extern __shared__ __align__(16) unsigned char oz_smem[];
    OzStage *stg = reinterpret_cast<OzStage *>(oz_smem);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t m0 = (int64_t)blockIdx.x * OZ_BM;
    const int n0 = blockIdx.y * OZ_BN;
    const int nk = (int)(kp / OZ_BK);

    auto load = [&](int buf, int64_t k0) {
        OzStage &st = stg[buf];
        for (int c = tid; c < S * OZ_BM * 4; c += OZ_THREADS) {
            const int p = c / (OZ_BM * 4), r = (c >> 2) % OZ_BM, part = c & 3;
            cp_async16(&st.a[p][r][part * 8], sl + ((int64_t)p * np + m0 + r) * kp + k0 + part * 8);
        }
        for (int c = tid; c < S * OZ_BN * 4; c += OZ_THREADS) {
            const int p = c / (OZ_BN * 4), r = (c >> 2) % OZ_BN, part = c & 3;
            cp_async16(&st.z[p][r][part * 8], zs + ((int64_t)p * sp + n0 + r) * kp + k0 + part * 8);
        }
        cp_async_commit();
    };

    float lv[5][4][4], tail[4][4], hi[4][4], lo[4][4];
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
#pragma unroll
            for (int t = 0; t < 5; ++t) lv[t][nt][v] = 0.f;
            tail[nt][v] = hi[nt][v] = lo[nt][v] = 0.f;
        }

    // ldmatrix lane addresses: A tile rows (lane & 7) + 8 ((lane >> 3) & 1),
    // k offset 8 (lane >> 4); Z tile columns (lane & 7) + 8 (lane >> 4), k
    // offset 8 ((lane >> 3) & 1)
    const int a_row = warp * 16 + (lane & 7) + (((lane >> 3) & 1) << 3);
    const int a_col = (lane >> 4) << 3;
    const int z_row = (lane & 7) + ((lane >> 4) << 3);
    const int z_col = ((lane >> 3) & 1) << 3;

    load(0, 0);
    for (int kt = 0; kt < nk; ++kt) {
        if (kt + 1 < nk) {
            load((kt + 1) & 1, (int64_t)(kt + 1) * OZ_BK);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        const OzStage &st = stg[kt & 1];
#pragma unroll
        for (int ks = 0; ks < OZ_BK; ks += 16) {
            uint32_t a[S][4];
#pragma unroll
            for (int p = 0; p < S; ++p) ldsm_x4(a[p][0], a[p][1], a[p][2], a[p][3], &st.a[p][a_row][ks + a_col]);
#pragma unroll
            for (int q = 0; q < S; ++q) {
                uint32_t b[4][2];
#pragma unroll
                for (int h = 0; h < 2; ++h)
                    ldsm_x4(b[2 * h][0], b[2 * h][1], b[2 * h + 1][0], b[2 * h + 1][1],
                            &st.z[q][h * 16 + z_row][ks + z_col]);
#pragma unroll
                for (int p = 0; p + q < S; ++p)
#pragma unroll
                    for (int nt = 0; nt < 4; ++nt) {
                        if (p + q < 5)
                            mma_bf16(lv[p + q][nt], a[p], b[nt]);
                        else
                            mma_bf16(tail[nt], a[p], b[nt]);
                    }
            }
        }
        // level 4 and the tail after every stage, levels 0..3 after every 64 of k
        const bool all = (kt + 1) % (OZ_FLUSH / OZ_BK) == 0 || kt + 1 == nk;
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                df_add(hi[nt][v], lo[nt][v], lv[4][nt][v]);
                df_add(hi[nt][v], lo[nt][v], tail[nt][v]);
                lv[4][nt][v] = 0.f;
                tail[nt][v] = 0.f;
                if (all) {
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        df_add(hi[nt][v], lo[nt][v], lv[t][nt][v]);
                        lv[t][nt][v] = 0.f;
                    }
                }
            }
        __syncthreads();   // the next iteration's load overwrites this stage
    }

    // accumulator (nt, v): row 16 warp + (lane >> 2) + 8 (v >> 1), column
    // 8 nt + 2 (lane & 3) + (v & 1)
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int64_t i = m0 + warp * 16 + (lane >> 2) + ((v >> 1) << 3);
            const int j = n0 + nt * 8 + ((lane & 3) << 1) + (v & 1);
            if (i < n && j < s) {
                const double x = (double)hi[nt][v] + (double)lo[nt][v];
                W[(int64_t)j * ldw + i] = scalbn(x, ea[i] + ez[j] - 16);
            }
        }
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

}  // namespace

bool oz_eligible(int64_t n, int s) { return s >= OZ_MIN_RHS && n >= OZ_MIN_N; }

size_t oz_a_bytes(int64_t n) {
    const int64_t np = oz_np(n), kp = oz_kp(n);
    return align256((size_t)S * np * kp * sizeof(__nv_bfloat16)) + align256((size_t)np * sizeof(int));
}

size_t oz_z_bytes(int64_t n, int s) {
    const int64_t kp = oz_kp(n);
    const int sp = oz_sp(s);
    return align256((size_t)S * sp * kp * sizeof(__nv_bfloat16)) + align256((size_t)sp * sizeof(int));
}

hodlr_status oz_split_a(hodlr_ctx *c, const double *A, int64_t n, int64_t lda, void *abuf, cudaStream_t st) {
    const int64_t np = oz_np(n), kp = oz_kp(n);
    auto *sl = reinterpret_cast<__nv_bfloat16 *>(abuf);
    int *ea = reinterpret_cast<int *>(reinterpret_cast<char *>(abuf) +
                                      align256((size_t)S * np * kp * sizeof(__nv_bfloat16)));
    oz_split_rows_kernel<<<(unsigned)(np / 8), 256, 0, st>>>(A, n, lda, np, kp, sl, ea, c->d_status);
    note_launch();
    HODLR_TRY_CUDA(cudaGetLastError());
    return HODLR_OK;
}

hodlr_status oz_matvec(hodlr_ctx *c, const void *abuf, int64_t n, int s, const double *Z, int64_t ldz, double *W,
                       int64_t ldw, void *zbuf, cudaStream_t st) {
    if (n == 0 || s == 0) return HODLR_OK;
    const int64_t np = oz_np(n), kp = oz_kp(n);
    const int sp = oz_sp(s);
    if (np / OZ_BM > 0x7fffffff || sp / OZ_BN > 65535) {
        set_error("oz_matvec: size out of range (n %lld, s %d)", (long long)n, s);
        return HODLR_RANGE;
    }
    const auto *sl = reinterpret_cast<const __nv_bfloat16 *>(abuf);
    const int *ea = reinterpret_cast<const int *>(reinterpret_cast<const char *>(abuf) +
                                                  align256((size_t)S * np * kp * sizeof(__nv_bfloat16)));
    auto *zs = reinterpret_cast<__nv_bfloat16 *>(zbuf);
    int *ez = reinterpret_cast<int *>(reinterpret_cast<char *>(zbuf) +
                                      align256((size_t)S * sp * kp * sizeof(__nv_bfloat16)));
    oz_split_cols_kernel<<<(unsigned)sp, 256, 0, st>>>(Z, ldz, n, s, kp, sp, zs, ez, c->d_status);
    note_launch();
    HODLR_TRY_CUDA(cudaFuncSetAttribute(oz_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)OZ_SMEM));
    const dim3 grid((unsigned)(np / OZ_BM), (unsigned)(sp / OZ_BN));
    oz_gemm_kernel<<<grid, OZ_THREADS, OZ_SMEM, st>>>(sl, ea, np, kp, zs, ez, sp, n, s, W, ldw);
    note_launch();
    HODLR_TRY_CUDA(cudaGetLastError());
    return HODLR_OK;
}

}  // namespace hodlr
