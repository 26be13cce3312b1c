// FP64-accurate W = A Z on the BF16 tensor cores (tcgen05), for many
// right-hand sides.
//
// GMRES (Sec. 3) needs the product with the FP64 front A to FP64 accuracy.
// With one to a few right-hand sides it is a matrix-vector stream (the
// double-float kernel in gmres.cu); with tens it is a GEMM of n x n x s.  Here
// every FP64 entry is split exactly into balanced base-256 digits relative to a
// power of two shared by its row of A (column of Z):
//   a = 2^(e_i - 8) sum_p d_p 2^(-8p),  p = 0..6,  d_p integer, |d_p| <= 128,
// e_i the least exponent with max_k |A(i,k)| < 2^(e_i - 1), the last digit
// rounded to nearest (every digit is an exact BF16 number), so that
//   (A Z)(i,j) = 2^(e_i + f_j - 16) sum_t 2^(-8t) sum_{p+q=t} (A_p Z_q)(i,j).
// The 28 slice products of the levels t = 0..6 (the pairs with t >= 7 lie
// below 2^-56 of the leading level and are dropped) run on the tensor cores:
// for slice p of A one MMA multiplies it with the Z slices 0..6-p stacked along
// N, into the TMEM accumulators of the levels p..6 (level t at columns 32 t).
// Over one chunk of 32 values of k a level's sum is an integer of magnitude at
// most 32 (t + 1) 2^14 <= 7 * 2^19 < 2^22, so the FP32 accumulation is exact
// whatever rounding the tensor core applies.  After every chunk the epilogue
// warps read the 7 levels out of TMEM and add them, as integers, into two
// 64-bit sums per (row, rhs): hi = sum over t <= 2 of A_t 2^(8(2-t)) and lo =
// sum over t = 3..6 of A_t 2^(8(6-t)).  Integer sums are exact and
// order-independent, so split-K partial sums combine with integer atomics and
// the product is bitwise reproducible.  Finally
//   W(i,j) = 2^(e_i + f_j - 32) hi + 2^(e_i + f_j - 64) lo   (FP64).
// The error per term is at most about 2^-56 max|A(i,:)| max|Z(:,j)| (digit
// rounding) plus the final FP64 rounding.
//
// The GEMM kernel is warp-specialised: warp 0 streams 3 shared-memory stages
// of (7 slices of 128 rows of A, 7 slices of 32 columns of Z) x 32 values of k
// with TMA (64-byte swizzle); warp 1 allocates TMEM (two accumulator sets of
// 224 columns) and issues the MMAs (M = 128, N = 32 (7 - p), K = 16, two
// k-steps per chunk); warps 2..9 drain the accumulators (warp w reads the TMEM
// lanes of quarter w mod 4, i.e. 32 rows, and 16 of the 32 right-hand sides).
// Every wait on an mbarrier is bounded (about 2 s of global time): on timeout
// the status word gets ST_TIMEOUT, every role leaves its loop, the copies and
// MMAs already issued are waited for (bounded too), TMEM is freed and the
// kernel returns.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>
#include <mutex>

#include "internal.cuh"

namespace hodlr {
namespace {

constexpr int S = OZ_SLICES;        // 7 digit slices
constexpr int TC_BM = 128;          // rows of A per CTA (the MMA's M)
constexpr int TC_BN = 32;           // right-hand sides per CTA
constexpr int TC_BK = 32;           // k per chunk: one shared-memory stage, one exact flush
constexpr int TC_STAGES = 3;
constexpr int TC_THREADS = 320;     // warp 0 TMA, warp 1 MMA, warps 2..9 epilogue
constexpr int TC_EPI_WARPS = 8;
constexpr int TC_ACC_COLS = S * TC_BN;          // 224 TMEM columns per accumulator set
constexpr int TC_TMEM_COLS = 512;
constexpr uint32_t TC_A_BYTES = S * TC_BM * TC_BK * 2;   // 57344
constexpr uint32_t TC_Z_BYTES = S * TC_BN * TC_BK * 2;   // 14336
constexpr uint32_t TC_STAGE_BYTES = TC_A_BYTES + TC_Z_BYTES;
constexpr size_t TC_SMEM = (size_t)TC_STAGES * TC_STAGE_BYTES + 1024 /* alignment */ + 256 /* barriers */;
static_assert(TC_SMEM <= 227 * 1024, "three stages must fit in shared memory");
static_assert(TC_A_BYTES % 1024 == 0 && TC_Z_BYTES % 1024 == 0, "stages keep the swizzle alignment");
// the exact-flush bound: 32 values of k, 7 pairs, |digit products| <= 2^14
static_assert((long long)TC_BK * S * (1 << 14) < (1 << 22), "level sums of a chunk must stay below 2^22");

constexpr float MAGIC = 12582912.0f;            // 1.5 * 2^23: x + MAGIC has the bits 0x4B400000 + x
constexpr uint32_t MAGIC_BITS = 0x4B400000u;
constexpr unsigned long long GT_LIMIT_NS = 2000000000ull;   // bound of every wait

inline int64_t oz_np(int64_t n) { return (n + TC_BM - 1) / TC_BM * TC_BM; }
inline int64_t oz_kp(int64_t n) { return (n + TC_BK - 1) / TC_BK * TC_BK; }
inline int oz_sp(int s) { return (s + TC_BN - 1) / TC_BN * TC_BN; }
size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// ------------------------------------------------------------------ digit split
__device__ __forceinline__ int exp_field(double a) {
    return (int)((unsigned long long)__double_as_longlong(a) >> 52) & 0x7FF;
}

// The balanced digits of a relative to 2^e (|a| < 2^(e-1); a not finite or
// subnormal: all zero): F = round(|a| 2^(56 - e)) <= 2^55 written in base 256
// with the six lower digits in [-128, 128) (a digit of 128 or more becomes
// d - 256 with a carry into the next one) and the top digit, F's bits from 48
// on plus that carry, in [0, 128]; the sign of a on every digit.
__device__ __forceinline__ void balanced_digits(double a, int e, __nv_bfloat16 (&out)[S]) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(a);
    const int ex = (int)(u >> 52) & 0x7FF;
    unsigned long long F = 0;
    if (ex != 0 && ex != 0x7FF) {
        const unsigned long long mant = (u & 0xFFFFFFFFFFFFFull) | (1ull << 52);
        const int sh = 1019 + e - ex;   // F = mant 2^(-sh); sh >= -2 as |a| < 2^(e-1)
        if (sh <= 0)
            F = mant << (-sh);
        else if (sh < 56)
            F = (mant + (1ull << (sh - 1))) >> sh;
    }
    const bool neg = (u >> 63) != 0;
#pragma unroll
    for (int p = S - 1; p >= 0; --p) {
        int d = (int)(F & 255u);
        F >>= 8;
        if (p > 0 && d >= 128) {
            d -= 256;
            F += 1;
        }
        out[p] = __float2bfloat16_rn((float)(neg ? -d : d));
    }
}

// One warp per row of the padded np x kp slices: the row's exponent, then its
// digits (zero outside the n x n matrix).  Slices: [S][np][kp] BF16.
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
    const int e = mx - 1021;
    if (lane == 0) {
        ea[i] = e;
        if (bad) atomicOr(status, ST_NONFINITE);
    }
    for (int64_t k = lane; k < kp; k += 32) {
        __nv_bfloat16 d[S];
        balanced_digits((i < n && k < n) ? row[k] : 0.0, e, d);
#pragma unroll
        for (int p = 0; p < S; ++p) sl[((int64_t)p * np + i) * kp + k] = d[p];
    }
}

// One CTA per column of the padded Z slices: [S][sp][kp] BF16.
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
    const int e = s_max - 1021;
    if (threadIdx.x == 0) {
        ez[j] = e;
        if (s_bad) atomicOr(status, ST_NONFINITE);
    }
    for (int64_t k = threadIdx.x; k < kp; k += blockDim.x) {
        __nv_bfloat16 d[S];
        balanced_digits((j < s && k < n) ? col[k] : 0.0, e, d);
#pragma unroll
        for (int p = 0; p < S; ++p) zs[((int64_t)p * sp + j) * kp + k] = d[p];
    }
}

// ------------------------------------------------------------------ PTX wrappers
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the phase of `parity` to complete, giving up after GT_LIMIT_NS or
// when another role has given up (*abort set).  Returns false on give-up.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int *abort, int *status) {
    if (mbar_try(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (unsigned it = 1;; ++it) {
        if (mbar_try(bar, parity)) return true;
        if ((it & 63) == 0) {
            if (*abort) return false;
            if (global_ns() - t0 > GT_LIMIT_NS) {
                *abort = 1;
                atomicOr(status, ST_TIMEOUT);
                return false;
            }
        }
    }
}

// The same wait with no early exit on abort (draining what was issued), bounded.
__device__ __forceinline__ void mbar_drain(uint32_t bar, uint32_t parity, int *status) {
    const unsigned long long t0 = global_ns();
    for (unsigned it = 0;; ++it) {
        if (mbar_try(bar, parity)) return;
        if ((it & 63) == 63 && global_ns() - t0 > GT_LIMIT_NS) {
            atomicOr(status, ST_TIMEOUT);
            return;
        }
    }
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *map, int c0, int c1, int c2,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
        : "memory");
}

// Shared-memory matrix descriptor of a K-major tile with 64-byte swizzle: rows
// of 64 bytes (32 BF16 values of k), 8-row groups 512 bytes apart.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;              // leading byte offset (16 B; not used for swizzled K-major)
    d |= (uint64_t)(512 >> 4) << 32;     // stride byte offset: 8 rows x 64 B
    d |= (uint64_t)1 << 46;              // descriptor version
    d |= (uint64_t)4 << 61;              // 64-byte swizzle
    return d;
}

// Instruction descriptor of kind::f16: BF16 A and B (both K-major), FP32 D, M x N.
__device__ __forceinline__ uint32_t mma_idesc(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t dtmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            dtmem),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int c = 0; c < 16; ++c) v[c] = __uint_as_float(r[c]);
}

// ------------------------------------------------------------------ the GEMM
struct TcArgs {
    const int *ea, *ez;
    int64_t n;
    int s;
    int nchunks;          // kp / 32
    int chunks_per_cta;   // along the split of k (blockIdx.z)
    unsigned long long *Phi, *Plo;   // [sp][np] integer partial sums
    int64_t np;
    int *status;
};

__global__ void __launch_bounds__(TC_THREADS, 1)
    oz_tc_gemm_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapZ,
                      const TcArgs a) {
    extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
    // 1024-byte aligned stage area (the swizzled tiles' phase depends on the address)
    unsigned char *smem = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(tc_smem_raw) + 1023) & ~uintptr_t(1023));
    unsigned long long *bars = reinterpret_cast<unsigned long long *>(smem + TC_STAGES * TC_STAGE_BYTES);
    // bars: full[3], empty[3], acc_full[2], acc_empty[2], drain
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * TC_BM, j0 = blockIdx.y * TC_BN;
    const int c_begin = blockIdx.z * a.chunks_per_cta;
    const int c_end = min(a.nchunks, c_begin + a.chunks_per_cta);
    const int nch = max(0, c_end - c_begin);
    const uint32_t sbase = smem_u32(smem);
    const uint32_t bar0 = smem_u32(bars);
    auto full = [&](int st) { return bar0 + 8u * st; };
    auto empty = [&](int st) { return bar0 + 8u * (TC_STAGES + st); };
    auto accf = [&](int b) { return bar0 + 8u * (2 * TC_STAGES + b); };
    auto acce = [&](int b) { return bar0 + 8u * (2 * TC_STAGES + 2 + b); };
    const uint32_t drain = bar0 + 8u * (2 * TC_STAGES + 4);

    if (threadIdx.x == 0) {
        for (int st = 0; st < TC_STAGES; ++st) {
            mbar_init(full(st), 1);
            mbar_init(empty(st), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(accf(b), 1);
            mbar_init(acce(b), TC_EPI_WARPS);
        }
        mbar_init(drain, 1);
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {   // the MMA warp owns the TMEM allocation
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(TC_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;
    volatile int *abort = &s_abort;

    if (warp == 0) {
        // ---------------- TMA producer
        if (lane == 0 && nch > 0) {
            int issued = 0;
            for (int c = 0; c < nch; ++c) {
                const int st = c % TC_STAGES;
                const uint32_t ph = (uint32_t)((c / TC_STAGES) & 1);
                if (!mbar_wait(empty(st), ph ^ 1u, abort, a.status)) break;
                const uint32_t sa = sbase + st * TC_STAGE_BYTES;
                mbar_expect_tx(full(st), TC_STAGE_BYTES);
                const int k0 = (c_begin + c) * TC_BK;
                tma_load_3d(sa, &mapA, k0, m0, 0, full(st));
                tma_load_3d(sa + TC_A_BYTES, &mapZ, k0, j0, 0, full(st));
                ++issued;
            }
            // copies still in flight when the pipeline stopped early: wait for
            // them (bounded) before the CTA may leave
            if (*abort)
                for (int c = max(0, issued - TC_STAGES); c < issued; ++c)
                    mbar_drain(full(c % TC_STAGES), (uint32_t)((c / TC_STAGES) & 1), a.status);
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer
        if (lane == 0 && nch > 0) {
            for (int c = 0; c < nch; ++c) {
                const int st = c % TC_STAGES;
                const uint32_t ph = (uint32_t)((c / TC_STAGES) & 1);
                const int b = c & 1;
                const uint32_t aph = (uint32_t)((c >> 1) & 1);
                if (!mbar_wait(full(st), ph, abort, a.status)) break;
                if (!mbar_wait(acce(b), aph ^ 1u, abort, a.status)) break;
                tc_fence_after();
                const uint32_t sa = sbase + st * TC_STAGE_BYTES;
                const uint32_t sz = sa + TC_A_BYTES;
                const uint32_t dcol = tmem + (uint32_t)(b * TC_ACC_COLS);
#pragma unroll
                for (int ks = 0; ks < TC_BK / 16; ++ks) {
#pragma unroll
                    for (int p = 0; p < S; ++p) {
                        const uint64_t ad = smem_desc(sa + p * (TC_BM * TC_BK * 2) + ks * 32);
                        const uint64_t bd = smem_desc(sz + ks * 32);
                        mma_bf16(dcol + 32u * p, ad, bd, mma_idesc(TC_BM, TC_BN * (S - p)),
                                 (ks == 0 && p == 0) ? 0u : 1u);
                    }
                }
                mma_commit(empty(st));   // the stage is free once these MMAs have read it
                mma_commit(accf(b));     // the accumulators are complete
            }
            // every MMA issued is complete before TMEM is released
            mma_commit(drain);
            mbar_drain(drain, 0, a.status);
        }
    } else {
        // ---------------- epilogue: warp w drains TMEM lanes 32 (w mod 4).., rhs 16 h..
        const int q = warp & 3, h = (warp - 2) >> 2;
        const uint32_t lane_base = (uint32_t)(32 * q) << 16;
        unsigned long long hi[16], lo[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) hi[c] = lo[c] = 0ull;
        int done = 0;
        for (int c = 0; c < nch; ++c) {
            const int b = c & 1;
            const uint32_t aph = (uint32_t)((c >> 1) & 1);
            // one lane waits, the warp follows it (tcgen05.ld needs the whole warp)
            int ok = 0;
            if (lane == 0) ok = mbar_wait(accf(b), aph, abort, a.status) ? 1 : 0;
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) break;
            tc_fence_after();
            const uint32_t t0 = tmem + lane_base + (uint32_t)(b * TC_ACC_COLS + 16 * h);
            float v[16];
            // levels 0..2 into hi (units of level 2), 3..6 into lo (units of level 6)
#pragma unroll
            for (int t = 0; t < S; ++t) {
                tmem_ld16(t0 + 32u * t, v);
                const unsigned long long m = (t <= 2) ? (1ull << (8 * (2 - t))) : (1ull << (8 * (6 - t)));
#pragma unroll
                for (int col = 0; col < 16; ++col) {
                    const unsigned long long bits = __float_as_uint(v[col] + MAGIC);
                    if (t <= 2)
                        hi[col] += bits * m;
                    else
                        lo[col] += bits * m;
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(acce(b));
            ++done;
        }
        // remove the conversion's bias (modular arithmetic: exact whenever the
        // true sums fit in 64 bits, which they do)
        const unsigned long long bh = (unsigned long long)done * MAGIC_BITS * (65536ull + 256ull + 1ull);
        const unsigned long long bl =
            (unsigned long long)done * MAGIC_BITS * ((1ull << 24) + (1ull << 16) + (1ull << 8) + 1ull);
        const int64_t row = m0 + 32 * q + lane;
        if (!*abort && done > 0 && row < a.n) {
#pragma unroll
            for (int col = 0; col < 16; ++col) {
                const int j = j0 + 16 * h + col;
                if (j < a.s) {
                    atomicAdd(a.Phi + (int64_t)j * a.np + row, hi[col] - bh);
                    atomicAdd(a.Plo + (int64_t)j * a.np + row, lo[col] - bl);
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS)
                     : "memory");
    }
}

// W(i, j) = 2^(e_i + f_j - 32) hi + 2^(e_i + f_j - 64) lo
__global__ void oz_finalize_kernel(const unsigned long long *__restrict__ Phi, const unsigned long long *__restrict__ Plo,
                                   const int *__restrict__ ea, const int *__restrict__ ez, int64_t n, int s, int64_t np,
                                   double *__restrict__ W, int64_t ldw) {
    const int j = blockIdx.y;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int e = ea[i] + ez[j];
        const double hi = (double)(long long)Phi[(int64_t)j * np + i];
        const double lo = (double)(long long)Plo[(int64_t)j * np + i];
        W[(int64_t)j * ldw + i] = scalbn(hi, e - 32) + scalbn(lo, e - 64);
    }
}

// ------------------------------------------------------------------ tensor maps
using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                 const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encode_fn() {
    static EncodeTiled fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiled>(p);
        cudaGetLastError();
    });
    return fn;
}

// [slices][rows][kp] BF16 slices, boxes of 32 k x `box_rows` rows x 7 slices, 64-byte swizzle
hodlr_status make_map(CUtensorMap *m, const void *base, int64_t rows, int64_t kp, int box_rows) {
    EncodeTiled fn = encode_fn();
    if (!fn) {
        set_error("oz: cuTensorMapEncodeTiled is not available from the driver");
        return HODLR_CUDA_ERROR;
    }
    const cuuint64_t dims[3] = {(cuuint64_t)kp, (cuuint64_t)rows, (cuuint64_t)S};
    const cuuint64_t strides[2] = {(cuuint64_t)kp * 2, (cuuint64_t)rows * kp * 2};
    const cuuint32_t box[3] = {(cuuint32_t)TC_BK, (cuuint32_t)box_rows, (cuuint32_t)S};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void *>(base), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("oz: cuTensorMapEncodeTiled failed (%d)", (int)r);
        return HODLR_CUDA_ERROR;
    }
    return HODLR_OK;
}

}  // namespace

bool oz_eligible(int64_t n, int s) { return s >= OZ_MIN_RHS && n >= OZ_MIN_N; }

size_t oz_a_bytes(int64_t n) {
    const int64_t np = oz_np(n), kp = oz_kp(n);
    return align256((size_t)S * np * kp * sizeof(__nv_bfloat16)) + align256((size_t)np * sizeof(int));
}

size_t oz_z_bytes(int64_t n, int s) {
    const int64_t np = oz_np(n), kp = oz_kp(n);
    const int sp = oz_sp(s);
    return align256((size_t)S * sp * kp * sizeof(__nv_bfloat16)) + align256((size_t)sp * sizeof(int)) +
           2 * align256((size_t)sp * np * sizeof(unsigned long long));
}

hodlr_status oz_split_a(hodlr_ctx *c, const double *A, int64_t n, int64_t lda, void *abuf, cudaStream_t st) {
    const int64_t np = oz_np(n), kp = oz_kp(n);
    auto *sl = reinterpret_cast<__nv_bfloat16 *>(abuf);
    int *ea = reinterpret_cast<int *>(reinterpret_cast<char *>(abuf) +
                                      align256((size_t)S * np * kp * sizeof(__nv_bfloat16)));
    {
        ProfScope ps("oz_split_rows_kernel", st);
        oz_split_rows_kernel<<<(unsigned)(np / 8), 256, 0, st>>>(A, n, lda, np, kp, sl, ea, c->d_status);
    }
    note_launch();
    HODLR_TRY_CUDA(cudaGetLastError());
    return HODLR_OK;
}

hodlr_status oz_matvec(hodlr_ctx *c, const void *abuf, int64_t n, int s, const double *Z, int64_t ldz, double *W,
                       int64_t ldw, void *zbuf, cudaStream_t st) {
    if (n == 0 || s == 0) return HODLR_OK;
    const int64_t np = oz_np(n), kp = oz_kp(n);
    const int sp = oz_sp(s);
    if (np / TC_BM > 0x7fffffff || sp / TC_BN > 65535 || np > 0x7fffffff || kp > 0x7fffffff) {
        set_error("oz_matvec: size out of range (n %lld, s %d)", (long long)n, s);
        return HODLR_RANGE;
    }
    const auto *sl = reinterpret_cast<const __nv_bfloat16 *>(abuf);
    const int *ea = reinterpret_cast<const int *>(reinterpret_cast<const char *>(abuf) +
                                                  align256((size_t)S * np * kp * sizeof(__nv_bfloat16)));
    char *zp = reinterpret_cast<char *>(zbuf);
    auto *zs = reinterpret_cast<__nv_bfloat16 *>(zp);
    zp += align256((size_t)S * sp * kp * sizeof(__nv_bfloat16));
    int *ez = reinterpret_cast<int *>(zp);
    zp += align256((size_t)sp * sizeof(int));
    auto *Phi = reinterpret_cast<unsigned long long *>(zp);
    zp += align256((size_t)sp * np * sizeof(unsigned long long));
    auto *Plo = reinterpret_cast<unsigned long long *>(zp);
    {
        ProfScope ps("oz_split_cols_kernel", st);
        oz_split_cols_kernel<<<(unsigned)sp, 256, 0, st>>>(Z, ldz, n, s, kp, sp, zs, ez, c->d_status);
    }
    note_launch();
    HODLR_TRY_CUDA(cudaMemsetAsync(Phi, 0, 2 * align256((size_t)sp * np * sizeof(unsigned long long)), st));
    CUtensorMap mA, mZ;
    HODLR_TRY(make_map(&mA, sl, np, kp, TC_BM));
    HODLR_TRY(make_map(&mZ, zs, sp, kp, TC_BN));
    // split k so that the grid holds about four CTAs per SM (one resident at a time)
    const int tiles = (int)(np / TC_BM) * (sp / TC_BN);
    const int nchunks = (int)(kp / TC_BK);
    int ksplit = std::max(1, (4 * std::max(1, c->num_sms) + tiles - 1) / tiles);
    ksplit = std::min(ksplit, std::max(1, nchunks / 8));
    ksplit = std::min(ksplit, 65535);
    const int per = (nchunks + ksplit - 1) / ksplit;
    ksplit = (nchunks + per - 1) / per;
    TcArgs ta{ea, ez, n, s, nchunks, per, Phi, Plo, np, c->d_status};
    HODLR_TRY_CUDA(cudaFuncSetAttribute(oz_tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM));
    const dim3 grid((unsigned)(np / TC_BM), (unsigned)(sp / TC_BN), (unsigned)ksplit);
    {
        ProfScope ps("oz_tc_gemm_kernel", st);
        oz_tc_gemm_kernel<<<grid, TC_THREADS, TC_SMEM, st>>>(mA, mZ, ta);
    }
    note_launch();
    HODLR_TRY_CUDA(cudaGetLastError());
    const unsigned gx = (unsigned)std::min<int64_t>((n + 255) / 256, 1024);
    oz_finalize_kernel<<<dim3(gx, (unsigned)s), 256, 0, st>>>(Phi, Plo, ea, ez, n, s, np, W, ldw);
    note_launch();
    HODLR_TRY_CUDA(cudaGetLastError());
    return HODLR_OK;
}

}  // namespace hodlr
