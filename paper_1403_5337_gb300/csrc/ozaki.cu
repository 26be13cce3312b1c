// FP64-accurate W = A Z on the FP16 tensor cores (tcgen05), for many
// right-hand sides.
//
// GMRES (Sec. 3) needs the product with the FP64 front A to FP64 accuracy.
// With one to a few right-hand sides it is a matrix-vector stream (the
// double-float kernel in gmres.cu); with tens it is a GEMM of n x n x s.  Here
// every FP64 entry is split exactly into balanced base-256 digits relative to a
// power of two shared by its row of A (column of Z):
//   a = 2^(e_i - 8) sum_p d_p 2^(-8p),  p = 0..6,  d_p integer, |d_p| <= 128,
// the last digit rounded to nearest, so that
//   (A Z)(i,j) = 2^(e_i + f_j - 16) sum_t 2^(-8t) sum_{p+q=t} (A_p Z_q)(i,j).
// The 28 slice products of the levels t = 0..6 (the pairs with t >= 7 lie
// below 2^-56 of the leading level and are dropped) run on the tensor cores:
// for slice p of A one MMA multiplies it with the Z slices 0..6-p stacked along
// N, into the TMEM accumulators of the levels p..6 (level t at columns 32 t).
// Every digit is an exact FP16 number, and over one chunk of 32 values of k a
// level's sum is an integer of magnitude at most 32 (t + 1) 2^14 <= 7 * 2^19 <
// 2^22, so the FP32 accumulation is exact whatever rounding the tensor core
// applies.
//
// A's digits live in HBM as bytes (7 n^2 bytes, made once per A): byte p of
// entry (i, k) is d_p + 128.  They are the two's-complement balanced digits of
// the signed integer round(a 2^(56 - e_i)), which lies strictly inside
// (-2^55 + B, 2^55 - B) for B = sum_{p<6} 128 * 256^p, so that the top digit
// stays in [-128, 127] as well: e_i is the least exponent with that property
// for the row's largest entry.  The GEMM kernel turns the bytes of a tile into
// FP16 digits in shared memory (two byte permutes and two FP16x2 adds per four
// digits) for the MMAs.  Z's digits (sign and magnitude, the top digit in
// [0, 128]) are written as FP16 slices per product.
//
// The GEMM kernel is persistent: one CTA per SM walks a contiguous range of
// (row tile, rhs tile, chunk of 32 k) units, the split of the work over SMs
// balanced to one unit.  Both operands are stored unit by unit (one unit of A
// is 28 KB of bytes, one of Z 14 KB of FP16 already in the shared-memory
// operand's 64-byte-swizzled order), so each arrives by one bulk copy.  Warp 0
// streams A's units (3 stages); warps 4-7 convert them into the FP16 slices of
// one of 2 MMA stages and fetch Z's unit into it; warp 1 allocates TMEM
// (two accumulator sets of 224 columns) and issues the MMAs (M = 128, N =
// 32 (7 - p), K = 16, two k-steps per chunk); warps 8-15 drain the accumulators
// after every chunk (warp w reads the TMEM lanes of quarter w mod 4, i.e. 32
// rows, and 16 of the 32 right-hand sides), adding each level's integer into a
// 32-bit sum (exact for 512 chunks), and at the end of a tile's run of units
// (or after 512 chunks) add, as 64-bit integers,
//   hi = sum_{t <= 2} x_t 2^(8(2-t)),  lo = sum_{t = 3..6} x_t 2^(8(6-t))
// into the tile's partial sums with atomics.  Integer sums are exact and
// order-independent, so the product is bitwise reproducible.  Finally
//   W(i,j) = 2^(e_i + f_j - 32) hi + 2^(e_i + f_j - 64) lo   (FP64).
// The error per term is at most about 2^-55 max|A(i,:)| max|Z(:,j)| (digit
// rounding) plus the final FP64 rounding.
//
// Every wait on an mbarrier is bounded (about 2 s of global time): on timeout
// the status word gets ST_TIMEOUT, every role leaves its loop, the copies and
// MMAs already issued are waited for (bounded too), TMEM is freed and the
// kernel returns.
#include <cuda_fp16.h>

#include <algorithm>
#include <cstdint>

#include "internal.cuh"

namespace hodlr {
namespace {

constexpr int S = OZ_SLICES;        // 7 digit slices
constexpr int TC_BM = 128;          // rows of A per unit (the MMA's M)
constexpr int TC_BN = 32;           // right-hand sides per unit
constexpr int TC_BK = 32;           // k per unit: one exact flush of TMEM
constexpr int TC_TSTAGES = 3;       // stages of A's bytes
constexpr int TC_MSTAGES = 2;       // MMA stages (FP16 slices of A and Z)
constexpr int TC_THREADS = 512;     // warp 0 loads, 1 MMA, 4-7 convert, 8-15 drain (2-3 idle)
constexpr int TC_CONV_WARP0 = 4;
constexpr int TC_CONV_WARPS = 4;
constexpr int TC_EPI_WARP0 = 8;
// registers per thread: 128 at launch (65536 / 512); the first two warpgroups
// (loads, MMA, converters) give up 48 each, the drain's two take 48 more each
constexpr int TC_REGS_LAUNCH = 128, TC_REGS_LOW = 80, TC_REGS_HIGH = 176;
static_assert(TC_REGS_LOW * 256 + TC_REGS_HIGH * 256 == TC_REGS_LAUNCH * TC_THREADS,
              "the register split must add up to the CTA's allocation");
constexpr int TC_EPI_WARPS = 8;
constexpr int TC_ACC_COLS = S * TC_BN;          // 224 TMEM columns per accumulator set
constexpr int TC_TMEM_COLS = 512;
constexpr uint32_t TC_AB_BYTES = S * TC_BM * TC_BK;           // 28672: A's bytes of a unit
constexpr uint32_t TC_AH_BYTES = S * TC_BM * TC_BK * 2;       // 57344: A's FP16 slices
constexpr uint32_t TC_Z_BYTES = S * TC_BN * TC_BK * 2;        // 14336: Z's FP16 slices
constexpr uint32_t TC_MSTAGE_BYTES = TC_AH_BYTES + TC_Z_BYTES;
constexpr size_t TC_SMEM = (size_t)TC_MSTAGES * TC_MSTAGE_BYTES + (size_t)TC_TSTAGES * TC_AB_BYTES +
                           1024 /* alignment */ + 256 /* barriers */;
static_assert(TC_SMEM <= 227 * 1024, "the stages must fit in shared memory");
static_assert(TC_AB_BYTES % 1024 == 0 && TC_AH_BYTES % 1024 == 0 && TC_Z_BYTES % 1024 == 0,
              "stages keep the swizzle alignment");
// the exact-flush bound: 32 values of k, 7 pairs, |digit products| <= 2^14
static_assert((long long)TC_BK * S * (1 << 14) < (1 << 22), "level sums of a chunk must stay below 2^22");
// 32-bit level sums over TC_FLUSH chunks stay below 2^31 in magnitude
constexpr int TC_FLUSH = 512;
static_assert((long long)TC_FLUSH * TC_BK * S * (1 << 14) < (1ll << 31), "32-bit level sums must not overflow");

constexpr float MAGIC = 12582912.0f;            // 1.5 * 2^23: x + MAGIC has the bits 0x4B400000 + x
constexpr uint32_t MAGIC_BITS = 0x4B400000u;
constexpr unsigned long long GT_LIMIT_NS = 2000000000ull;   // bound of every wait
// the six lower digits' bias: sum_{p<6} 128 * 256^p
constexpr unsigned long long DIGIT_BIAS = 0x808080808080ull;

inline int64_t oz_np(int64_t n) { return (n + TC_BM - 1) / TC_BM * TC_BM; }
inline int64_t oz_kp(int64_t n) { return (n + TC_BK - 1) / TC_BK * TC_BK; }
inline int oz_sp(int s) { return (s + TC_BN - 1) / TC_BN * TC_BN; }
size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// ------------------------------------------------------------------ digit split
__device__ __forceinline__ int exp_field(double a) {
    return (int)((unsigned long long)__double_as_longlong(a) >> 52) & 0x7FF;
}

// round(|a| 2^(56 - e)) (ties away from zero) for an entry a of the row or
// column whose exponent is e, so that sh = 1019 + e - ex >= -2; zero for a
// zero, subnormal or non-finite a.
__device__ __forceinline__ unsigned long long scaled_magnitude(unsigned long long u, int e) {
    const int ex = (int)(u >> 52) & 0x7FF;
    if (ex == 0 || ex == 0x7FF) return 0ull;
    const unsigned long long mant = (u & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const int sh = 1019 + e - ex;
    if (sh <= 0) return mant << (-sh);
    if (sh < 56) return (mant + (1ull << (sh - 1))) >> sh;
    return 0ull;
}

// Z's balanced digits relative to 2^e (|a| < 2^(e-1); a not finite or
// subnormal: all zero): F = round(|a| 2^(56 - e)) <= 2^55 written in base 256
// with the six lower digits in [-128, 128) (a digit of 128 or more becomes
// d - 256 with a carry into the next one) and the top digit, F's bits from 48
// on plus that carry, in [0, 128]; the sign of a on every digit.
__device__ __forceinline__ void balanced_digits(double a, int e, __half (&out)[S]) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(a);
    unsigned long long F = scaled_magnitude(u, e);
    const bool neg = (u >> 63) != 0;
#pragma unroll
    for (int p = S - 1; p >= 0; --p) {
        int d = (int)(F & 255u);
        F >>= 8;
        if (p > 0 && d >= 128) {
            d -= 256;
            F += 1;
        }
        out[p] = __int2half_rn(neg ? -d : d);
    }
}

// A's digit bytes of one entry relative to 2^e, packed: byte 6 - p of the
// result is d_p + 128.  G = round(a 2^(56-e)) + DIGIT_BIAS (two's complement)
// holds d_p + 128 in its bytes 0..5 (p = 6..1) and the top digit d_0 in its
// bits 48..63, which e keeps in [-128, 127].
__device__ __forceinline__ unsigned long long digit_bytes(double a, int e) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(a);
    unsigned long long F = scaled_magnitude(u, e);
    if (u >> 63) F = 0ull - F;
    const unsigned long long G = F + DIGIT_BIAS;
    return (G & 0xFFFFFFFFFFFFull) | ((((G >> 48) & 0xFFull) ^ 0x80ull) << 48);
}

// The row exponent of A: the least e with |a| < 2^(e-1) for the row's largest
// entry M whose scaled value also leaves the top digit below 128:
// round(M 2^(56-e)) + DIGIT_BIAS < 2^55.  M = 0 gives e = -1021 (all digits 0).
__device__ __forceinline__ int row_exponent(unsigned long long mbits) {
    const int ex = (int)(mbits >> 52) & 0x7FF;
    if (ex == 0) return -1021;
    int e = ex - 1021;
    const unsigned long long top = (((mbits & 0xFFFFFFFFFFFFFull) | (1ull << 52)) << 2);   // round(M 2^(56-e))
    if (top + DIGIT_BIAS >= (1ull << 55)) e += 1;
    return e;
}

// One warp per 4 rows of the padded np x kp matrix (8 lanes per row): each
// row's exponent from its largest magnitude, then its digit bytes (zero outside
// the n x n matrix), in units of 128 rows x 32 k: unit (row tile, chunk) is one
// block of 7 x 128 x 32 bytes ([slice][row][k]) at (row tile * chunks + chunk)
// * 28672, so that the GEMM fetches a unit with one bulk copy.  A lane takes 4
// consecutive k of its row, so the warp writes 128 contiguous bytes of every
// slice of a unit per chunk.
__global__ void __launch_bounds__(256) oz_split_rows_kernel(const double *__restrict__ A, int64_t n, int64_t lda,
                                                            int64_t np, int64_t kp, uint8_t *__restrict__ sl,
                                                            int *__restrict__ ea, int *status) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t i = ((int64_t)blockIdx.x * 8 + warp) * 4 + (lane >> 3);
    const int sub = lane & 7;
    if (i >= np) return;   // the grid covers np rows exactly: whole warps only
    const double *row = A + i * lda;
    unsigned long long mx = 0ull;
    int bad = 0;
    if (i < n)
        for (int64_t k = sub; k < n; k += 8) {
            const unsigned long long u = (unsigned long long)__double_as_longlong(row[k]) & 0x7FFFFFFFFFFFFFFFull;
            if ((u >> 52) == 0x7FF)
                bad = 1;
            else
                mx = u > mx ? u : mx;
        }
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) {
        const unsigned long long t = __shfl_xor_sync(0xffffffffu, mx, o);
        mx = t > mx ? t : mx;
        bad |= __shfl_xor_sync(0xffffffffu, bad, o);
    }
    const int e = row_exponent(mx);
    if (sub == 0) {
        ea[i] = e;
        if (bad) atomicOr(status, ST_NONFINITE);
    }
    const int64_t nchunks = kp / TC_BK;
    uint8_t *u0 = sl + (i >> 7) * nchunks * (int64_t)TC_AB_BYTES + (i & 127) * TC_BK + sub * 4;
    for (int64_t c = 0; c < nchunks; ++c) {
        const int64_t k0 = c * TC_BK + sub * 4;
        uint32_t w[S];
#pragma unroll
        for (int p = 0; p < S; ++p) w[p] = 0u;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int64_t k = k0 + q;
            const unsigned long long g = digit_bytes((i < n && k < n) ? row[k] : 0.0, e);
#pragma unroll
            for (int p = 0; p < S; ++p) w[p] |= (uint32_t)((g >> (8 * (S - 1 - p))) & 0xFFu) << (8 * q);
        }
        uint8_t *u = u0 + c * TC_AB_BYTES;
#pragma unroll
        for (int p = 0; p < S; ++p) *reinterpret_cast<uint32_t *>(u + p * (TC_BM * TC_BK)) = w[p];
    }
}

// One CTA per column of the padded Z: FP16 digit slices in units of 32
// columns x 32 k, unit (rhs tile, chunk) one block of 7 x 32 x 32 halves
// ([slice][column][k]) at (rhs tile * chunks + chunk) * 14336 bytes, each
// 64-byte row already in the 64-byte-swizzled order of the shared-memory
// operand (16-byte piece c of row r at piece c ^ ((r / 2) mod 4)), so that a
// bulk copy of the unit is the MMA's B operand.
__global__ void __launch_bounds__(256) oz_split_cols_kernel(const double *__restrict__ Z, int64_t ldz, int64_t n,
                                                            int s, int64_t kp, int sp, __half *__restrict__ zs,
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
        __half d[S];
        balanced_digits((j < s && k < n) ? col[k] : 0.0, e, d);
        const int jr = j & 31, kk = (int)(k & 31);
        __half *u = zs + ((int64_t)(j >> 5) * (kp / TC_BK) + (k >> 5)) * (TC_Z_BYTES / 2) + jr * TC_BK +
                    (((kk >> 3) ^ ((jr >> 1) & 3)) << 3) + (kk & 7);
#pragma unroll
        for (int p = 0; p < S; ++p) u[p * (TC_BN * TC_BK)] = d[p];
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

// One contiguous block of `bytes` (a multiple of 16, both addresses 16-byte
// aligned) from global to shared memory, completing on `bar`.
__device__ __forceinline__ void bulk_load(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
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

// Instruction descriptor of kind::f16: FP16 A and B (both K-major; format
// code 0 in bits 7-9 and 10-12), FP32 D (bit 4), M x N.
__device__ __forceinline__ uint32_t mma_idesc(int M, int N) {
    return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Shared-memory writes of this thread made visible to the async proxy (the
// tensor core's operand reads).
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mma_f16(uint32_t dtmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
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

// Issue a load of 16 columns without waiting for it (tmem_wait() completes it).
__device__ __forceinline__ void tmem_ld16_issue(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
}

// Wait for this thread's TMEM loads; the registers they wrote pass through an
// empty asm so that no use of them is scheduled before the wait.
__device__ __forceinline__ void tmem_wait(uint32_t (&a)[16], uint32_t (&b)[16]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int c = 0; c < 16; ++c) asm volatile("" : "+r"(a[c]), "+r"(b[c]));
}

__device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t b, uint32_t sel) {
    uint32_t d;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(sel));
    return d;
}

__device__ __forceinline__ uint32_t hadd2(uint32_t a, uint32_t b) {
    uint32_t d;
    asm("add.rn.f16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}

__device__ __forceinline__ uint4 ld_shared_v4(uint32_t addr) {
    uint4 v;
    asm volatile("ld.shared.v4.b32 {%0, %1, %2, %3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(addr));
    return v;
}

__device__ __forceinline__ void st_shared_v4(uint32_t addr, uint32_t x, uint32_t y, uint32_t z, uint32_t w) {
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(x), "r"(y), "r"(z), "r"(w));
}

// Four digit bytes u (one word) as two FP16x2 words of d = u - 128: a byte
// permute puts each u under the FP16 exponent of 1024 (0x64uu = 1024 + u,
// exact), and one FP16x2 add of -1152 (0xE480) leaves u - 128, exact.
__device__ __forceinline__ void bytes_to_half2(uint32_t w, uint32_t &lo, uint32_t &hi) {
    constexpr uint32_t E1024 = 0x64646464u, BIAS = 0xE480E480u;
    lo = hadd2(prmt(w, E1024, 0x4140u), BIAS);
    hi = hadd2(prmt(w, E1024, 0x4342u), BIAS);
}

// ------------------------------------------------------------------ the GEMM
struct TcArgs {
    int64_t n;
    int s;
    int nchunks;                     // kp / 32
    int ntn;                         // tiles of 32 right-hand sides
    long long units;                 // row tiles x rhs tiles x chunks
    unsigned long long *Phi, *Plo;   // [sp][np] integer partial sums
    int64_t np;
    int *status;
};

// A position in the unit sequence, advanced one unit at a time (no divisions
// in the roles' loops): units run over the chunks of a tile, then the next
// tile; tile = row tile * ntn + rhs tile.
struct Cursor {
    int tile, chunk;
    __device__ __forceinline__ void next(int nchunks) {
        if (++chunk == nchunks) {
            chunk = 0;
            ++tile;
        }
    }
};

__device__ __forceinline__ Cursor cursor_at(const TcArgs &a, long long u) {
    const long long tile = u / a.nchunks;
    return Cursor{(int)tile, (int)(u - tile * a.nchunks)};
}

__global__ void __launch_bounds__(TC_THREADS, 1)
    oz_tc_gemm_kernel(const uint8_t *__restrict__ Ab, const __half *__restrict__ Zb, const TcArgs a) {
    extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
    // 1024-byte aligned stage area (the swizzled tiles' phase depends on the address):
    // [MMA stage 0][MMA stage 1][byte stage 0..2][barriers]
    unsigned char *smem = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(tc_smem_raw) + 1023) & ~uintptr_t(1023));
    unsigned char *tsm = smem + TC_MSTAGES * TC_MSTAGE_BYTES;
    unsigned long long *bars = reinterpret_cast<unsigned long long *>(tsm + TC_TSTAGES * TC_AB_BYTES);
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // this CTA's units: [u0, u0 + nu), the split balanced to one unit
    const long long u0 = a.units * blockIdx.x / gridDim.x;
    const int nu = (int)(a.units * (blockIdx.x + 1) / gridDim.x - u0);
    const uint32_t mbase = smem_u32(smem);
    const uint32_t tbase = smem_u32(tsm);
    const uint32_t bar0 = smem_u32(bars);
    auto tfull = [&](int st) { return bar0 + 8u * st; };
    auto tempty = [&](int st) { return bar0 + 8u * (3 + st); };
    auto cfull = [&](int ms) { return bar0 + 8u * (6 + ms); };
    auto zfull = [&](int ms) { return bar0 + 8u * (8 + ms); };
    auto mempty = [&](int ms) { return bar0 + 8u * (10 + ms); };
    auto accf = [&](int b) { return bar0 + 8u * (12 + b); };
    auto acce = [&](int b) { return bar0 + 8u * (14 + b); };
    const uint32_t drain = bar0 + 8u * 16;
    static_assert(TC_TSTAGES == 3 && TC_MSTAGES == 2, "barrier layout");

    if (threadIdx.x == 0) {
        for (int st = 0; st < TC_TSTAGES; ++st) {
            mbar_init(tfull(st), 1);
            mbar_init(tempty(st), TC_CONV_WARPS);
        }
        for (int ms = 0; ms < TC_MSTAGES; ++ms) {
            mbar_init(cfull(ms), TC_CONV_WARPS);
            mbar_init(zfull(ms), 1);
            mbar_init(mempty(ms), 1);
            mbar_init(accf(ms), 1);
            mbar_init(acce(ms), TC_EPI_WARPS);
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
    // Each warpgroup changes its registers at the top of its own branch (the
    // host launches only when the kernel was compiled with TC_REGS_LAUNCH per
    // thread): warpgroup 0 holds the loads and the MMA warp, 1 the converters,
    // 2-3 the drain.
    if (warp < TC_CONV_WARP0) {
        asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(TC_REGS_LOW));
        if (warp == 0) {
            // ---------------- producer of A's digit bytes (bulk copies)
            if (lane == 0 && nu > 0) {
                int issued = 0;
                Cursor cu = cursor_at(a, u0);
                for (int i = 0; i < nu; ++i, cu.next(a.nchunks)) {
                    const int st = i % TC_TSTAGES;
                    const uint32_t ph = (uint32_t)((i / TC_TSTAGES) & 1);
                    if (!mbar_wait(tempty(st), ph ^ 1u, abort, a.status)) break;
                    const long long ua = (long long)(cu.tile / a.ntn) * a.nchunks + cu.chunk;
                    mbar_expect_tx(tfull(st), TC_AB_BYTES);
                    bulk_load(tbase + st * TC_AB_BYTES, Ab + ua * TC_AB_BYTES, TC_AB_BYTES, tfull(st));
                    ++issued;
                }
                // copies still in flight when the pipeline stopped early: wait for
                // them (bounded) before the CTA may leave
                if (*abort)
                    for (int i = max(0, issued - TC_TSTAGES); i < issued; ++i)
                        mbar_drain(tfull(i % TC_TSTAGES), (uint32_t)((i / TC_TSTAGES) & 1), a.status);
            }
        } else if (warp == 1) {
            // ---------------- MMA issuer
            if (lane == 0 && nu > 0) {
                for (int i = 0; i < nu; ++i) {
                    const int ms = i & 1;
                    const uint32_t ph = (uint32_t)((i >> 1) & 1);
                    if (!mbar_wait(cfull(ms), ph, abort, a.status)) break;
                    if (!mbar_wait(zfull(ms), ph, abort, a.status)) break;
                    if (!mbar_wait(acce(ms), ph ^ 1u, abort, a.status)) break;
                    tc_fence_after();
                    const uint32_t sa = mbase + ms * TC_MSTAGE_BYTES;
                    const uint32_t sz = sa + TC_AH_BYTES;
                    const uint32_t dcol = tmem + (uint32_t)(ms * TC_ACC_COLS);
    #pragma unroll
                    for (int ks = 0; ks < TC_BK / 16; ++ks) {
    #pragma unroll
                        for (int p = 0; p < S; ++p) {
                            const uint64_t ad = smem_desc(sa + p * (TC_BM * TC_BK * 2) + ks * 32);
                            const uint64_t bd = smem_desc(sz + ks * 32);
                            mma_f16(dcol + 32u * p, ad, bd, mma_idesc(TC_BM, TC_BN * (S - p)),
                                    (ks == 0 && p == 0) ? 0u : 1u);
                        }
                    }
                    mma_commit(mempty(ms));   // the stage is free once these MMAs have read it
                    mma_commit(accf(ms));     // the accumulators are complete
                }
                // every MMA issued is complete before TMEM is released
                mma_commit(drain);
                mbar_drain(drain, 0, a.status);
            }
        }
    } else if (warp < TC_EPI_WARP0) {
        asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(TC_REGS_LOW));
        // ---------------- converters: warp wc turns rows 32 wc.. of every slice
        // of A's byte unit into FP16 digits in the MMA stage; warp 4 also fetches
        // Z's unit into that stage
        const int wc = warp - TC_CONV_WARP0;
        int zissued = 0;
        Cursor cu = cursor_at(a, u0);
        // 7 slices x 32 rows x 2 halves of 16 values of k: 14 pieces per lane;
        // lane l takes row 32 wc + 16 jj + l / 2, half l mod 2, of every slice p
        // and jj = 0..1, so that its offsets are constants plus a lane term, and
        // row r's 64-byte swizzle (r / 2) mod 4 = (l / 4) mod 4 is the lane's own
        constexpr int JJ = TC_BM / TC_CONV_WARPS / 16;
        const uint32_t src_lane = (uint32_t)((wc * (TC_BM / TC_CONV_WARPS) + (lane >> 1)) * TC_BK + (lane & 1) * 16);
        const uint32_t dst_lane = (uint32_t)((wc * (TC_BM / TC_CONV_WARPS) + (lane >> 1)) * (TC_BK * 2));
        const int sw = (lane >> 2) & 3, hh = lane & 1;
        const uint32_t c0 = (uint32_t)(((2 * hh) ^ sw) << 4), c1 = (uint32_t)(((2 * hh + 1) ^ sw) << 4);
        constexpr int NP = S * JJ, G = (NP + 1) / 2;   // pieces, and pieces loaded before any is converted
        for (int i = 0; i < nu; ++i, cu.next(a.nchunks)) {
            const int st = i % TC_TSTAGES;
            const uint32_t ph = (uint32_t)((i / TC_TSTAGES) & 1);
            const int ms = i & 1;
            const uint32_t mph = (uint32_t)((i >> 1) & 1);
            int ok = 1;
            if (lane == 0)
                ok = (mbar_wait(tfull(st), ph, abort, a.status) && mbar_wait(mempty(ms), mph ^ 1u, abort, a.status))
                         ? 1
                         : 0;
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) break;
            // every lane acquires both completed phases itself (neither can move
            // on before this warp arrives below)
            mbar_try(tfull(st), ph);
            mbar_try(mempty(ms), mph ^ 1u);
            const uint32_t sa = mbase + ms * TC_MSTAGE_BYTES;
            if (wc == 0 && lane == 0) {
                const long long uz = (long long)(cu.tile % a.ntn) * a.nchunks + cu.chunk;
                mbar_expect_tx(zfull(ms), TC_Z_BYTES);
                bulk_load(sa + TC_AH_BYTES, Zb + uz * (TC_Z_BYTES / 2), TC_Z_BYTES, zfull(ms));
                ++zissued;
            }
            const uint32_t src = tbase + st * TC_AB_BYTES + src_lane;
            const uint32_t dst = sa + dst_lane;
            // half of the pieces' loads in flight before their conversion (one
            // load at a time stalled each warp on shared-memory latency)
#pragma unroll
            for (int g0 = 0; g0 < NP; g0 += G) {
                uint4 b[G];
#pragma unroll
                for (int t = 0; t < G; ++t)
                    if (g0 + t < NP)
                        b[t] = ld_shared_v4(src + ((g0 + t) / JJ) * (TC_BM * TC_BK) + ((g0 + t) % JJ) * 16 * TC_BK);
#pragma unroll
                for (int t = 0; t < G; ++t) {
                    if (g0 + t >= NP) continue;
                    const int p = (g0 + t) / JJ, jj = (g0 + t) % JJ;
                    uint32_t o[8];
                    bytes_to_half2(b[t].x, o[0], o[1]);
                    bytes_to_half2(b[t].y, o[2], o[3]);
                    bytes_to_half2(b[t].z, o[4], o[5]);
                    bytes_to_half2(b[t].w, o[6], o[7]);
                    const uint32_t row = dst + (uint32_t)(p * (TC_BM * TC_BK * 2) + jj * 16 * (TC_BK * 2));
                    st_shared_v4(row + c0, o[0], o[1], o[2], o[3]);
                    st_shared_v4(row + c1, o[4], o[5], o[6], o[7]);
                }
            }
            fence_proxy_async();
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(cfull(ms));
                mbar_arrive(tempty(st));
            }
        }
        if (*abort && wc == 0 && lane == 0)
            for (int i = max(0, zissued - TC_MSTAGES); i < zissued; ++i)
                mbar_drain(zfull(i & 1), (uint32_t)((i >> 1) & 1), a.status);
    } else {
        asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(TC_REGS_HIGH));
        // ---------------- epilogue: warp w drains TMEM lanes 32 (w mod 4).., rhs 16 h..
        const int q = warp & 3, h = (warp - TC_EPI_WARP0) >> 2;
        const uint32_t lane_base = (uint32_t)(32 * q) << 16;
        Cursor cu = cursor_at(a, u0);
        int i = 0;
        bool ok = true;
        while (ok && i < nu) {
            // one run of units of the same tile (at most TC_FLUSH of them)
            const int tile = cu.tile;
            uint32_t acc[S][16];
#pragma unroll
            for (int t = 0; t < S; ++t)
#pragma unroll
                for (int c = 0; c < 16; ++c) acc[t][c] = 0u;
            int cnt = 0;
            do {
                const int b = i & 1;
                const uint32_t aph = (uint32_t)((i >> 1) & 1);
                // one lane waits, the warp follows it (tcgen05.ld needs the whole warp)
                int w = 0;
                if (lane == 0) w = mbar_wait(accf(b), aph, abort, a.status) ? 1 : 0;
                ok = __shfl_sync(0xffffffffu, w, 0) != 0;
                if (!ok) break;
                tc_fence_after();
                const uint32_t t0 = tmem + lane_base + (uint32_t)(b * TC_ACC_COLS + 16 * h);
                // two levels' loads in flight per wait
#pragma unroll
                for (int t = 0; t < S; t += 2) {
                    uint32_t va[16], vb[16];
                    tmem_ld16_issue(t0 + 32u * t, va);
                    if (t + 1 < S)
                        tmem_ld16_issue(t0 + 32u * (t + 1), vb);
                    else
#pragma unroll
                        for (int c = 0; c < 16; ++c) vb[c] = 0u;
                    tmem_wait(va, vb);
#pragma unroll
                    for (int c = 0; c < 16; ++c) acc[t][c] += __float_as_uint(__uint_as_float(va[c]) + MAGIC);
                    if (t + 1 < S) {
#pragma unroll
                        for (int c = 0; c < 16; ++c)
                            acc[t + 1][c] += __float_as_uint(__uint_as_float(vb[c]) + MAGIC);
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(acce(b));
                ++cnt;
                ++i;
                cu.next(a.nchunks);
            } while (i < nu && cu.tile == tile && cnt < TC_FLUSH);
            if (!ok || *abort) break;
            // remove the conversion's bias (modular: exact while the true sums
            // stay below 2^31 in magnitude) and add the levels as 64-bit
            // integers into the tile's partial sums
            const uint32_t bias = (uint32_t)cnt * MAGIC_BITS;
            const int tm = tile / a.ntn, tn = tile - tm * a.ntn;
            const int64_t row = (int64_t)tm * TC_BM + 32 * q + lane;
            if (row < a.n) {
                const int j0 = tn * TC_BN + 16 * h;
                const int ncol = a.s - j0;   // columns of this lane's 16 that exist
                unsigned long long *ph = a.Phi + (int64_t)j0 * a.np + row;
                unsigned long long *pl = a.Plo + (int64_t)j0 * a.np + row;
#pragma unroll
                for (int c = 0; c < 16; ++c) {
                    if (c < ncol) {
                        const long long hi = (long long)(int)(acc[0][c] - bias) * 65536ll +
                                             (long long)(int)(acc[1][c] - bias) * 256ll +
                                             (long long)(int)(acc[2][c] - bias);
                        const long long lo = (long long)(int)(acc[3][c] - bias) * 16777216ll +
                                             (long long)(int)(acc[4][c] - bias) * 65536ll +
                                             (long long)(int)(acc[5][c] - bias) * 256ll +
                                             (long long)(int)(acc[6][c] - bias);
                        atomicAdd(ph, (unsigned long long)hi);
                        atomicAdd(pl, (unsigned long long)lo);
                    }
                    ph += a.np;
                    pl += a.np;
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

}  // namespace

bool oz_eligible(int64_t n, int s) { return s >= OZ_MIN_RHS && n >= OZ_MIN_N; }

size_t oz_a_bytes(int64_t n) {
    const int64_t np = oz_np(n), kp = oz_kp(n);
    return align256((size_t)S * np * kp) + align256((size_t)np * sizeof(int));
}

size_t oz_z_bytes(int64_t n, int s) {
    const int64_t np = oz_np(n), kp = oz_kp(n);
    const int sp = oz_sp(s);
    return align256((size_t)S * sp * kp * sizeof(__half)) + align256((size_t)sp * sizeof(int)) +
           2 * align256((size_t)sp * np * sizeof(unsigned long long));
}

hodlr_status oz_split_a(hodlr_ctx *c, const double *A, int64_t n, int64_t lda, void *abuf, cudaStream_t st) {
    const int64_t np = oz_np(n), kp = oz_kp(n);
    auto *sl = reinterpret_cast<uint8_t *>(abuf);
    int *ea = reinterpret_cast<int *>(reinterpret_cast<char *>(abuf) + align256((size_t)S * np * kp));
    {
        ProfScope ps("oz_split_rows_kernel", st);
        oz_split_rows_kernel<<<(unsigned)(np / 32), 256, 0, st>>>(A, n, lda, np, kp, sl, ea, c->d_status);
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
    if (sp / TC_BN > 65535 || np / TC_BM > 0x7fffffff / 2 || kp > 0x7fffffff) {
        set_error("oz_matvec: size out of range (n %lld, s %d)", (long long)n, s);
        return HODLR_RANGE;
    }
    const auto *sl = reinterpret_cast<const uint8_t *>(abuf);
    const int *ea = reinterpret_cast<const int *>(reinterpret_cast<const char *>(abuf) + align256((size_t)S * np * kp));
    char *zp = reinterpret_cast<char *>(zbuf);
    auto *zs = reinterpret_cast<__half *>(zp);
    zp += align256((size_t)S * sp * kp * sizeof(__half));
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
    // persistent: one CTA per SM over all (row tile, rhs tile, chunk) units
    const int nchunks = (int)(kp / TC_BK);
    const long long tiles = (np / TC_BM) * (long long)(sp / TC_BN);
    if (tiles > 0x7fffffffll) {
        set_error("oz_matvec: size out of range (n %lld, s %d)", (long long)n, s);
        return HODLR_RANGE;
    }
    const long long units = tiles * nchunks;
    const int grid = (int)std::min<long long>(std::max(1, c->num_sms), units);
    TcArgs ta{n, s, nchunks, sp / TC_BN, units, Phi, Plo, np, c->d_status};
    HODLR_TRY_CUDA(cudaFuncSetAttribute(oz_tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM));
    {
        // the warpgroups' register changes assume this allocation per thread:
        // with any other, the drain warps' increase could never be granted
        cudaFuncAttributes fa;
        HODLR_TRY_CUDA(cudaFuncGetAttributes(&fa, oz_tc_gemm_kernel));
        if (fa.numRegs != TC_REGS_LAUNCH) {
            set_error("oz_matvec: the product kernel was compiled with %d registers per thread, not %d", fa.numRegs,
                      TC_REGS_LAUNCH);
            return HODLR_CUDA_ERROR;
        }
    }
    {
        ProfScope ps("oz_tc_gemm_kernel", st);
        oz_tc_gemm_kernel<<<grid, TC_THREADS, TC_SMEM, st>>>(sl, zs, ta);
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
