// FP64-accurate GMRES on the device (Sec. 3: GMRES with the HODLR direct solve
// as preconditioner), right-preconditioned in the flexible form:
//   z_j = P^-1 v_j (stored),  w = A z_j,  classical Gram-Schmidt twice,
//   Givens rotations on the Hessenberg column, estimate |g_{j+1}| / ||b||,
//   x = x0 + Z_j y once the estimate meets tol, then the true residual.
// Each right-hand side is an independent system with its own Krylov basis.
//
// The matvec with the FP64 front A is the dominant data stream.  GB300's FP64
// pipe is ~1/64 of its FP32 rate, so the product is formed on the FP32 pipes
// in double-float arithmetic: every FP64 entry a is split exactly into
// a = a_hi + a_lo + (a 5-bit tail) by integer operations on its bits (a_hi =
// the leading 24 significand bits, a_lo = the next 29 rounded to 24), z is
// split likewise, the product a_hi z_hi is made exact with an FMA
// (TwoProduct), cross terms are added in FP32, and the row sum is accumulated
// as an unevaluated float pair with TwoSum.  The relative error per term is
// about 2^-48, comparable to an FP64 dot product's accumulated rounding.
// With 16 or more right-hand sides the product is a GEMM and takes the exact
// digit-slice product on the FP16 tensor cores instead (ozaki.cu).
#include <algorithm>
#include <cmath>
#include <memory>
#include <mutex>
#include <vector>

#include "internal.cuh"

namespace hodlr {
namespace {

// ------------------------------------------------------------------ double-float matvec
struct DF {
    float s, c;
};

__device__ __forceinline__ void split_entry(double a, float &hi, float &lo, int &bad) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(a);
    const unsigned h32 = (unsigned)(u >> 32), l32 = (unsigned)u;
    const unsigned ex = (h32 >> 20) & 0x7FFu;
    const unsigned sgn = h32 & 0x80000000u;
    if (ex < 897u) {            // zero, FP64 subnormal, or below FP32's normal range
        hi = 0.f;
        lo = 0.f;
        return;
    }
    if (ex > 1150u) {           // >= 2^128, Inf or NaN
        bad = 1;
        hi = 0.f;
        lo = 0.f;
        return;
    }
    hi = __uint_as_float(sgn | ((ex - 896u) << 23) | ((h32 & 0xFFFFFu) << 3) | (l32 >> 29));
    if (ex >= 949u) {
        const float rem = __uint2float_rn(l32 & 0x1FFFFFFFu);
        const float scale = __uint_as_float((ex - 948u) << 23);   // 2^(ex - 1075)
        lo = __uint_as_float(__float_as_uint(rem * scale) | sgn);
    } else {
        lo = 0.f;
    }
}

__device__ __forceinline__ void df_acc(DF &acc, float ah, float al, float zh, float zl) {
    const float p = ah * zh;
    const float e = fmaf(ah, zh, -p);
    const float t = fmaf(ah, zl, fmaf(al, zh, e));
    const float s = acc.s + p;
    const float bp = s - acc.s;
    const float err = (acc.s - (s - bp)) + (p - bp);
    acc.s = s;
    acc.c += err + t;
}

// The same with zl = 0 (z exactly an FP32 value: the output of an FP32 apply).
__device__ __forceinline__ void df_acc_z(DF &acc, float ah, float al, float zh) {
    const float p = ah * zh;
    const float t = fmaf(al, zh, fmaf(ah, zh, -p));
    const float s = acc.s + p;
    const float bp = s - acc.s;
    const float err = (acc.s - (s - bp)) + (p - bp);
    acc.s = s;
    acc.c += err + t;
}

template <bool ZF>
__device__ __forceinline__ void df_term(DF &acc, float ah, float al, float zh, float zl) {
    if constexpr (ZF)
        df_acc_z(acc, ah, al, zh);
    else
        df_acc(acc, ah, al, zh, zl);
}

constexpr int MV_THREADS = 256;
constexpr int MV_WARPS = MV_THREADS / 32;
constexpr int MV_RPW = 2;            // rows per warp
constexpr int MV_ROWS = MV_WARPS * MV_RPW;
constexpr int MV_KC = 1024;          // columns per CTA (one column split)
constexpr int MV_S = 4;              // right-hand sides per pass
constexpr int MV_U = 2;              // 16-byte loads in flight per lane and row

__global__ void split_vec_kernel(const double *__restrict__ Z, int64_t ldz, int64_t n, int s,
                                 float2 *__restrict__ zs) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * s;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e % n, r = e / n;
        const double z = Z[i + r * ldz];
        const float h = __double2float_rn(z);
        const float l = __double2float_rn(z - (double)h);
        zs[r * n + i] = make_float2(h, l);
    }
}

// W(:, r0:r0+sr) += A(:, k0:k0+KC) Z(k0:k0+KC, r0:r0+sr) for the column split
// k0 = blockIdx.y * KC; zs = split Z (n x s, column-major float2); W zeroed
// beforehand, the splits are combined with FP64 atomics.  Each lane sums at
// most 32 terms per row in the float pair before it is converted to FP64, so
// the compensation term's own FP32 rounding never accumulates further.
// VEC: A rows are 16-byte aligned (even lda, aligned base) -> double2 loads.
// With a split buffer Asp (n x n FP32 pairs, ld n, VEC only): while *split_state
// is 0 the kernel splits A as usual and also stores the pairs to Asp; once it
// is 1 (set by the Arnoldi step that follows the first product of a solve)
// it reads the pairs instead of A and skips the split -- the same FP32 parts,
// so the same products.
// ZF: every z of this launch has a zero low part (z is exactly FP32).
template <bool VEC, bool ZF>
__global__ void __launch_bounds__(MV_THREADS, 4)
    df_matvec_kernel(const double *__restrict__ A, int64_t n, int64_t lda, const float2 *__restrict__ zs,
                     int s, int r0, double *__restrict__ W, int64_t ldw, int *status, float2 *__restrict__ Asp,
                     const int *__restrict__ split_state) {
    __shared__ __align__(16) float2 zsm[MV_S][MV_KC];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t k0 = (int64_t)blockIdx.y * MV_KC;
    const int kc = (n - k0 < (int64_t)MV_KC) ? (int)(n - k0) : MV_KC;
    const int sr = min(MV_S, s - r0);
    for (int e = threadIdx.x; e < MV_S * MV_KC; e += MV_THREADS) {
        const int q = e / MV_KC, kk = e % MV_KC;
        zsm[q][kk] = (q < sr && kk < kc) ? zs[(int64_t)(r0 + q) * n + k0 + kk] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    const int64_t row0 = (int64_t)blockIdx.x * MV_ROWS + warp * MV_RPW;
    DF acc[MV_RPW][MV_S];
#pragma unroll
    for (int a = 0; a < MV_RPW; ++a)
#pragma unroll
        for (int q = 0; q < MV_S; ++q) acc[a][q] = DF{0.f, 0.f};
    int bad = 0;
    // 1: write the pairs, 2: read them (a later launch of the same product reads
    // what the launch for the first right-hand sides wrote)
    const int smode = (VEC && Asp) ? ((*split_state || r0 > 0) ? 2 : 1) : 0;
    if (VEC && smode == 2) {
        const int np = kc >> 1;
        for (int p0 = lane; p0 < np; p0 += 32 * MV_U) {
            float4 hv[MV_RPW][MV_U];   // (h0, l0, h1, l1) of a column pair
#pragma unroll
            for (int u = 0; u < MV_U; ++u) {
                const int p = p0 + 32 * u;
#pragma unroll
                for (int a = 0; a < MV_RPW; ++a) {
                    const int64_t row = row0 + a;
                    hv[a][u] = (p < np && row < n) ? __ldg(reinterpret_cast<const float4 *>(Asp + row * n + k0) + p)
                                                   : make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
#pragma unroll
            for (int u = 0; u < MV_U; ++u) {
                const int p = p0 + 32 * u;
                if (p >= np) break;
#pragma unroll
                for (int q = 0; q < MV_S; ++q) {
                    const float4 z = reinterpret_cast<const float4 *>(zsm[q])[p];
#pragma unroll
                    for (int a = 0; a < MV_RPW; ++a) {
                        df_term<ZF>(acc[a][q], hv[a][u].x, hv[a][u].y, z.x, z.y);
                        df_term<ZF>(acc[a][q], hv[a][u].z, hv[a][u].w, z.z, z.w);
                    }
                }
            }
        }
        if ((kc & 1) && lane == 0) {   // odd tail column
            const int kk = kc - 1;
#pragma unroll
            for (int a = 0; a < MV_RPW; ++a) {
                const int64_t row = row0 + a;
                if (row >= n) continue;
                const float2 hl = Asp[row * n + k0 + kk];
#pragma unroll
                for (int q = 0; q < MV_S; ++q) df_term<ZF>(acc[a][q], hl.x, hl.y, zsm[q][kk].x, zsm[q][kk].y);
            }
        }
    } else if (VEC) {
        const int np = kc >> 1;   // column pairs
        for (int p0 = lane; p0 < np; p0 += 32 * MV_U) {
            double2 av[MV_RPW][MV_U];
#pragma unroll
            for (int u = 0; u < MV_U; ++u) {
                const int p = p0 + 32 * u;
#pragma unroll
                for (int a = 0; a < MV_RPW; ++a) {
                    const int64_t row = row0 + a;
                    av[a][u] = (p < np && row < n)
                                   ? __ldg(reinterpret_cast<const double2 *>(A + row * lda + k0) + p)
                                   : make_double2(0.0, 0.0);
                }
            }
#pragma unroll
            for (int u = 0; u < MV_U; ++u) {
                const int p = p0 + 32 * u;
                if (p >= np) break;
#pragma unroll
                for (int a = 0; a < MV_RPW; ++a) {
                    float h0, l0, h1, l1;
                    split_entry(av[a][u].x, h0, l0, bad);
                    split_entry(av[a][u].y, h1, l1, bad);
                    if (smode == 1 && row0 + a < n)
                        reinterpret_cast<float4 *>(Asp + (row0 + a) * n + k0)[p] = make_float4(h0, l0, h1, l1);
#pragma unroll
                    for (int q = 0; q < MV_S; ++q) {
                        const float4 z = reinterpret_cast<const float4 *>(zsm[q])[p];
                        df_term<ZF>(acc[a][q], h0, l0, z.x, z.y);
                        df_term<ZF>(acc[a][q], h1, l1, z.z, z.w);
                    }
                }
            }
        }
        if ((kc & 1) && lane == 0) {   // odd tail column
            const int kk = kc - 1;
#pragma unroll
            for (int a = 0; a < MV_RPW; ++a) {
                const int64_t row = row0 + a;
                if (row >= n) continue;
                float h0, l0;
                split_entry(A[row * lda + k0 + kk], h0, l0, bad);
                if (smode == 1) Asp[row * n + k0 + kk] = make_float2(h0, l0);
#pragma unroll
                for (int q = 0; q < MV_S; ++q) df_term<ZF>(acc[a][q], h0, l0, zsm[q][kk].x, zsm[q][kk].y);
            }
        }
    } else {
        for (int kk0 = lane; kk0 < kc; kk0 += 32 * MV_U) {
            double av[MV_RPW][MV_U];
#pragma unroll
            for (int u = 0; u < MV_U; ++u)
#pragma unroll
                for (int a = 0; a < MV_RPW; ++a) {
                    const int kk = kk0 + 32 * u;
                    const int64_t row = row0 + a;
                    av[a][u] = (kk < kc && row < n) ? __ldg(A + row * lda + k0 + kk) : 0.0;
                }
#pragma unroll
            for (int u = 0; u < MV_U; ++u) {
                const int kk = kk0 + 32 * u;
                if (kk >= kc) break;
#pragma unroll
                for (int a = 0; a < MV_RPW; ++a) {
                    float h0, l0;
                    split_entry(av[a][u], h0, l0, bad);
#pragma unroll
                    for (int q = 0; q < MV_S; ++q) df_term<ZF>(acc[a][q], h0, l0, zsm[q][kk].x, zsm[q][kk].y);
                }
            }
        }
    }
    if (bad) atomicOr(status, ST_NONFINITE);
    // Warp sums of the float pairs (TwoSum on the leading parts; after the xor
    // butterfly every lane holds every sum), then lane a MV_S + q converts sum
    // (a, q) to FP64 and adds it to W: three FP64 instructions per warp.
    float rs = 0.f, rc = 0.f;
#pragma unroll
    for (int a = 0; a < MV_RPW; ++a)
#pragma unroll
        for (int q = 0; q < MV_S; ++q) {
            DF p = acc[a][q];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float oh = __shfl_xor_sync(0xffffffffu, p.s, o);
                const float ol = __shfl_xor_sync(0xffffffffu, p.c, o);
                const float t = p.s + oh;
                const float bp = t - p.s;
                const float err = (p.s - (t - bp)) + (oh - bp);
                p.s = t;
                p.c = (p.c + ol) + err;
            }
            if (lane == a * MV_S + q) {
                rs = p.s;
                rc = p.c;
            }
        }
    if (lane < MV_RPW * MV_S) {
        const int a = lane / MV_S, q = lane % MV_S;
        const int64_t row = row0 + a;
        if (row < n && q < sr) atomicAdd(&W[row + (int64_t)(r0 + q) * ldw], (double)rs + (double)rc);
    }
}

// ------------------------------------------------------------------ Krylov kernels
constexpr int KT = 256;

// The Arnoldi step index of every kernel below is the per-rhs device counter
// jcur[r] (all active right-hand sides advance together), so one recorded
// iteration can be replayed by a device-side loop.

struct GState {
    double *H;       // (m+1) x m per rhs
    double *cs, *sn, *g;
    double *bnorm, *est;
    int *iters, *jcur, *active, *nactive;
};

// y = H(0:j,0:j)^-1 g(0:j) by back substitution, then X_r += Z_r y.  Grid
// (row chunks, rhs): every CTA solves the small triangular system itself (j is
// at most the restart length) and updates its own rows.
__global__ void __launch_bounds__(KT)
    backsolve_kernel(GState st, int m, const double *__restrict__ Zk, int64_t zstride, int64_t n, double *__restrict__ X,
                     int64_t ldx) {
    const int r = blockIdx.y;
    const int j = st.jcur[r];
    if (j <= 0) return;
    extern __shared__ double ys[];
    const double *H = st.H + (int64_t)r * (m + 1) * m;
    const double *g = st.g + (int64_t)r * (m + 1);
    if (threadIdx.x == 0) {
        for (int i = j - 1; i >= 0; --i) {
            double v = g[i];
            for (int k = i + 1; k < j; ++k) v -= H[i + (int64_t)k * (m + 1)] * ys[k];
            ys[i] = v / H[i + (int64_t)i * (m + 1)];
        }
    }
    __syncthreads();
    const double *Z = Zk + r * zstride;
    for (int64_t q = blockIdx.x * (int64_t)KT + threadIdx.x; q < n; q += (int64_t)gridDim.x * KT) {
        double v = X[q + r * ldx];
        for (int k = 0; k < j; ++k) v = fma(Z[(int64_t)k * n + q], ys[k], v);
        X[q + r * ldx] = v;
    }
}

// R = B - R (R holds A X), accumulate ||R||^2 per rhs.
__global__ void residual_kernel(const double *__restrict__ B, int64_t ldb, double *__restrict__ R, int64_t ldr, int64_t n,
                                double *__restrict__ nrm2) {
    const int r = blockIdx.y;
    double local = 0.0;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        const double v = B[q + r * ldb] - R[q + r * ldr];
        R[q + r * ldr] = v;
        local = fma(v, v, local);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(0xffffffffu, local, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(&nrm2[r], local);
}

// Start a cycle: v_0 = r / ||r||, g = ||r|| e_1, jcur = 0, activity from the residual.
__global__ void start_cycle_kernel(GState st, int m, int s, double *__restrict__ R, int64_t ldr, int64_t n,
                                   const double *__restrict__ nrm2, double *__restrict__ Vk, int64_t vstride, double tol,
                                   int max_iter, int first, double *__restrict__ Zc) {
    // Every block decides activity from values no block of this launch writes:
    // iters was zeroed before the first cycle, and bnorm is only written (by
    // block 0) on the first cycle, when every block uses beta instead.
    const int r = blockIdx.y;
    if (r >= s) return;
    const double beta = sqrt(nrm2[r]);
    if (first && blockIdx.x == 0 && threadIdx.x == 0) st.bnorm[r] = beta;
    const double bn = first ? beta : st.bnorm[r];
    const int act = (bn > 0.0) && (beta > tol * bn) && (st.iters[r] < max_iter);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st.active[r] = act;
        st.jcur[r] = 0;
        st.g[(int64_t)r * (m + 1)] = beta;
        if (!act) st.est[r] = bn > 0.0 ? beta / bn : 0.0;
    }
    if (!act) return;
    double *v0 = Vk + r * vstride;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        const double v = R[q + r * ldr] / beta;
        v0[q] = v;
        Zc[q + r * n] = v;     // the first vector to precondition
        R[q + r * ldr] = 0.0;  // the first product accumulates into R
    }
}

__global__ void count_active_kernel(const int *active, int s, int *nactive) {
    int c = 0;
    for (int r = 0; r < s; ++r) c += active[r];
    *nactive = c;
}

// The host's view of a cycle, gathered for one copy: ints [active rhs, device
// status word (read and cleared), replays of the last cycle's iteration, iters
// per rhs], then from report_doff(s) on doubles [est, ||r||^2, ||b||] per rhs.
__host__ __device__ inline size_t report_doff(int s) { return ((size_t)(3 + s) * sizeof(int) + 7) & ~size_t(7); }
__host__ __device__ inline size_t report_bytes(int s) { return report_doff(s) + (size_t)3 * s * sizeof(double); }

__global__ void cycle_report_kernel(GState st, int s, const double *nrm, int *status, const int *loops, char *rep) {
    if (threadIdx.x != 0) return;
    int c = 0;
    for (int r = 0; r < s; ++r) c += st.active[r];
    *st.nactive = c;
    int *ri = reinterpret_cast<int *>(rep);
    ri[0] = c;
    ri[1] = atomicExch(status, 0);
    ri[2] = *loops;
    for (int r = 0; r < s; ++r) ri[3 + r] = st.iters[r];
    double *rd = reinterpret_cast<double *>(rep + report_doff(s));
    for (int r = 0; r < s; ++r) {
        rd[r] = st.est[r];
        rd[s + r] = nrm[r];
        rd[2 * s + r] = st.bnorm[r];
    }
}

// First node of a cycle's graph: the while loop runs only if some right-hand
// side is active (so the host need not wait for the count before launching).
__global__ void cond_init_kernel(const int *nactive, cudaGraphConditionalHandle handle) {
    cudaGraphSetConditional(handle, *nactive > 0 ? 1u : 0u);
}

// ------------------------------------------------------------------ fused Arnoldi step
// After w = A z_j: classical Gram-Schmidt twice against v_0..v_j, the new basis
// vector, the Givens update of the Hessenberg column and the loop test, in one
// cooperative kernel with two software grid barriers (bounded waits).
// Work units are (128-row chunk, rhs); thread t of a unit owns one row.
//   P1  Z(:, j) = z_j; h1 = V^T w                      (partial sums, atomics)
//   P2  w -= V h1; h2 = V^T w; ||w||^2
//   P3  w -= V h2; v_{j+1} = w / ||w|| (also the next apply's input), w = 0
//       (the next product accumulates into it), with ||w - V h2||^2 =
//       ||w||^2 - ||h2||^2 (V orthonormal to working precision after the first
//       pass; ||h2|| << ||w||, so the difference loses nothing); CTA 0 first
//       H(:, j) = h1 + h2, h1 = 0, then the Givens rotation of H(:, j), the
//       residual estimate, activity and the loop condition
// nrm and h2 are cleared by CTA 0 in P1 (they are only accumulated in P2).  The
// step j and the activity of every rhs are fixed until CTA 0 advances them at
// the end.
constexpr int TT = 128;   // one warp per SM sub-partition: the FP64 reductions are pipe-bound
constexpr int TW = TT / 32;
constexpr unsigned long long TAIL_SPIN_LIMIT = 1ull << 26;

struct TailArgs {
    double *Vk;
    int64_t vstride, n;
    double *w;          // n x s (ld n)
    double *Zc;         // n x s
    double *Zk;
    int64_t zstride;
    double *h1, *h2, *nrm;
    int hstride;
    GState gs;
    int m, s, max_iter;
    double tol;
    unsigned *bar;
    int *status;
    int *loops;
    int limit;
    int *split_state;   // set to 1: A's FP32 pairs are in place for the next products
    cudaGraphConditionalHandle handle;
};

__device__ void tail_grid_sync(unsigned *bar, int *status) {
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *vgen = bar + 1;
        const unsigned gen = *vgen;
        __threadfence();
        if (atomicAdd(bar, 1u) == gridDim.x - 1) {
            bar[0] = 0;
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            unsigned long long spins = 0;
            while (*vgen == gen) {
                if (++spins > TAIL_SPIN_LIMIT) {
                    atomicOr(status, ST_TIMEOUT);
                    break;
                }
                __nanosleep(32);
            }
        }
        __threadfence();
    }
    __syncthreads();
}

// Butterfly sum of G values per lane over the warp (G = 8, 16 or 32): rounds
// with an xor distance of at least G add the partner's values; the later rounds
// each keep the half of the values selected by one bit of the lane index.  Lane
// L ends with the warp total of value L mod G, after 31 (G = 32), 31 (16) or
// 23 (8) FP64 additions instead of five per value.
template <int G>
__device__ __forceinline__ double warp_transpose_sum(double (&v)[G], int lane) {
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        if (o >= G) {
#pragma unroll
            for (int k = 0; k < G; ++k) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
        } else {
            const bool up = (lane & o) != 0;
#pragma unroll
            for (int k = 0; k < o; ++k) {
                const double send = up ? v[k] : v[k + o];
                const double keep = up ? v[k + o] : v[k];
                v[k] = keep + __shfl_xor_sync(0xffffffffu, send, o);
            }
        }
    }
    return v[0];
}

// h[i] += sum over the unit's rows of V(q, i) x(q), i in [g0, g0 + G) and i <= j.
template <int G>
__device__ __forceinline__ void unit_gram_group(const double *V, int64_t n, int64_t q, bool own, double x, int g0,
                                                int j, double *h, double *part, int lane, int warp) {
    double v[G];
#pragma unroll
    for (int k = 0; k < G; ++k) v[k] = (own && g0 + k <= j) ? V[(int64_t)(g0 + k) * n + q] * x : 0.0;
    const double t = warp_transpose_sum<G>(v, lane);
    if (lane < G) part[warp * 32 + lane] = t;
    __syncthreads();
    if (threadIdx.x < G && g0 + (int)threadIdx.x <= j) {
        double u = 0.0;
#pragma unroll
        for (int wv = 0; wv < TW; ++wv) u += part[wv * 32 + threadIdx.x];
        atomicAdd(h + g0 + threadIdx.x, u);
    }
    __syncthreads();
}

// h[i] += sum over the unit's rows of V(q, i) x(q), i <= j (one atomic per i).
__device__ void unit_gram(const double *V, int64_t n, int64_t q, bool own, double x, int j, double *h,
                          double *part, int lane, int warp) {
    for (int g0 = 0; g0 <= j; g0 += 32) {
        const int left = j + 1 - g0;
        if (left <= 8)
            unit_gram_group<8>(V, n, q, own, x, g0, j, h, part, lane, warp);
        else if (left <= 16)
            unit_gram_group<16>(V, n, q, own, x, g0, j, h, part, lane, warp);
        else
            unit_gram_group<32>(V, n, q, own, x, g0, j, h, part, lane, warp);
    }
}

__global__ void __launch_bounds__(TT) arnoldi_tail_kernel(TailArgs a) {
    extern __shared__ double hs[];                      // [m + 1]: the coefficients of the unit's rhs
    int *sj = reinterpret_cast<int *>(hs + a.m + 1);    // [s]: j of every rhs at entry
    int *sa = sj + a.s;                                 // [s]: its activity at entry
    __shared__ double part[TW * 32];
    __shared__ double s_inv;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t chunks = (a.n + TT - 1) / TT;
    const int64_t units = chunks * a.s;
    for (int r = threadIdx.x; r < a.s; r += TT) {
        sj[r] = a.gs.jcur[r];
        sa[r] = a.gs.active[r];
    }
    __syncthreads();
    // ---- P1: Z(:, j) = z_j; h1 = V^T w
    if (blockIdx.x == 0) {
        for (int r = threadIdx.x; r < a.s; r += TT) a.nrm[r] = 0.0;
        for (int r = 0; r < a.s; ++r)
            for (int i = threadIdx.x; i <= sj[r]; i += TT) a.h2[(int64_t)r * a.hstride + i] = 0.0;
    }
    for (int64_t u = blockIdx.x; u < units; u += gridDim.x) {
        const int r = (int)(u / chunks);
        if (!sa[r]) continue;
        const int j = sj[r];
        const int64_t q = (u % chunks) * TT + threadIdx.x;
        const bool own = q < a.n;
        double x = 0.0;
        if (own) {
            x = a.w[q + r * a.n];
            a.Zk[r * a.zstride + (int64_t)j * a.n + q] = a.Zc[q + r * a.n];
        }
        unit_gram(a.Vk + r * a.vstride, a.n, q, own, x, j, a.h1 + (int64_t)r * a.hstride, part, lane, warp);
    }
    tail_grid_sync(a.bar, a.status);
    // ---- P2: w -= V h1; h2 = V^T w; ||w||^2
    for (int64_t u = blockIdx.x; u < units; u += gridDim.x) {
        const int r = (int)(u / chunks);
        if (!sa[r]) continue;
        const int j = sj[r];
        const int64_t q = (u % chunks) * TT + threadIdx.x;
        const bool own = q < a.n;
        const double *V = a.Vk + r * a.vstride;
        for (int i = threadIdx.x; i <= j; i += TT) hs[i] = __ldcg(a.h1 + (int64_t)r * a.hstride + i);
        __syncthreads();
        double x = 0.0;
        if (own) {
            x = a.w[q + r * a.n];
            for (int i = 0; i <= j; ++i) x = fma(-hs[i], V[(int64_t)i * a.n + q], x);
            a.w[q + r * a.n] = x;
        }
        unit_gram(V, a.n, q, own, x, j, a.h2 + (int64_t)r * a.hstride, part, lane, warp);
        double p = x * x;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) p += __shfl_xor_sync(0xffffffffu, p, o);
        if (lane == 0) part[warp] = p;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
#pragma unroll
            for (int wv = 0; wv < TW; ++wv) t += part[wv];
            atomicAdd(a.nrm + r, t);
        }
        __syncthreads();
    }
    tail_grid_sync(a.bar, a.status);
    if (blockIdx.x == 0) {
        // H(:, j) = h1 + h2 (both complete); h1 is no longer read
        for (int r = 0; r < a.s; ++r) {
            if (!sa[r]) continue;
            const int j = sj[r];
            double *Hc = a.gs.H + (int64_t)r * (a.m + 1) * a.m + (int64_t)j * (a.m + 1);
            for (int i = threadIdx.x; i <= j; i += TT) {
                Hc[i] = __ldcg(a.h1 + (int64_t)r * a.hstride + i) + __ldcg(a.h2 + (int64_t)r * a.hstride + i);
                a.h1[(int64_t)r * a.hstride + i] = 0.0;
            }
        }
    }
    // ---- P3: w -= V h2; v_{j+1} = w / ||w||; w = 0
    for (int64_t u = blockIdx.x; u < units; u += gridDim.x) {
        const int r = (int)(u / chunks);
        if (!sa[r]) continue;
        const int j = sj[r];
        const int64_t q = (u % chunks) * TT + threadIdx.x;
        const double *V = a.Vk + r * a.vstride;
        for (int i = threadIdx.x; i <= j; i += TT) hs[i] = __ldcg(a.h2 + (int64_t)r * a.hstride + i);
        __syncthreads();
        if (threadIdx.x == 0) {
            double h2n = 0.0;
            for (int i = 0; i <= j; ++i) h2n += hs[i] * hs[i];
            const double nw2 = __ldcg(a.nrm + r) - h2n;
            s_inv = nw2 > 0.0 ? 1.0 / sqrt(nw2) : 0.0;
        }
        __syncthreads();
        const double inv = s_inv;
        if (q < a.n) {
            double x = a.w[q + r * a.n];
            for (int i = 0; i <= j; ++i) x = fma(-hs[i], V[(int64_t)i * a.n + q], x);
            if (inv > 0.0) {
                const double v = x * inv;
                a.Vk[r * a.vstride + (int64_t)(j + 1) * a.n + q] = v;
                a.Zc[q + r * a.n] = v;
            }
            a.w[q + r * a.n] = 0.0;
        }
        __syncthreads();
    }
    if (blockIdx.x != 0) return;
    // ---- CTA 0: Givens rotation of H(:, j), residual estimate, activity, loop test
    __shared__ int s_cnt;
    if (threadIdx.x == 0) s_cnt = 0;
    __syncthreads();
    for (int r = threadIdx.x; r < a.s; r += TT) {
        if (!sa[r]) continue;
        const int j = sj[r];
        const double *h2r = a.h2 + (int64_t)r * a.hstride;
        double h2n = 0.0;
        for (int i = 0; i <= j; ++i) h2n += __ldcg(h2r + i) * __ldcg(h2r + i);
        double *Hc = a.gs.H + (int64_t)r * (a.m + 1) * a.m + (int64_t)j * (a.m + 1);
        double *cs = a.gs.cs + (int64_t)r * a.m, *sn = a.gs.sn + (int64_t)r * a.m;
        double *g = a.gs.g + (int64_t)r * (a.m + 1);
        const double nw2 = __ldcg(a.nrm + r) - h2n;
        const double hn = nw2 > 0.0 ? sqrt(nw2) : 0.0;
        Hc[j + 1] = hn;
        for (int i = 0; i < j; ++i) {
            const double t = cs[i] * Hc[i] + sn[i] * Hc[i + 1];
            Hc[i + 1] = -sn[i] * Hc[i] + cs[i] * Hc[i + 1];
            Hc[i] = t;
        }
        const double rho = hypot(Hc[j], Hc[j + 1]);
        if (rho == 0.0) {
            cs[j] = 1.0;
            sn[j] = 0.0;
        } else {
            cs[j] = Hc[j] / rho;
            sn[j] = Hc[j + 1] / rho;
        }
        Hc[j] = rho;
        Hc[j + 1] = 0.0;
        g[j + 1] = -sn[j] * g[j];
        g[j] = cs[j] * g[j];
        a.gs.iters[r] += 1;
        a.gs.jcur[r] = j + 1;
        const double est = fabs(g[j + 1]) / a.gs.bnorm[r];
        a.gs.est[r] = est;
        if (est <= a.tol || rho == 0.0 || hn == 0.0 || j + 1 >= a.m || a.gs.iters[r] >= a.max_iter)
            a.gs.active[r] = 0;
        else
            atomicAdd(&s_cnt, 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        *a.gs.nactive = s_cnt;
        if (a.split_state) *a.split_state = 1;
        const int it = ++(*a.loops);
        cudaGraphSetConditional(a.handle, (s_cnt > 0 && it < a.limit) ? 1u : 0u);
    }
}

}  // namespace

hodlr_status matvec_impl(hodlr_ctx *c, const double *A, int64_t n, int64_t lda, int s, const double *Z, int64_t ldz,
                         double *W, int64_t ldw, cudaStream_t st, void *work, bool w_zeroed, float2 *Asp,
                         const int *split_state, bool z_split, bool z_fp32) {
    if (n == 0 || s == 0) return HODLR_OK;
    float2 *zs = work ? reinterpret_cast<float2 *>(work)
                      : reinterpret_cast<float2 *>(dalloc(c, (size_t)n * s * sizeof(float2), st));
    if (!zs) return HODLR_OUT_OF_MEMORY;
    if (!(z_split && work)) {
        int blocks = (int)std::min<int64_t>((n * s + 255) / 256, 4096);
        split_vec_kernel<<<blocks, 256, 0, st>>>(Z, ldz, n, s, zs);
        note_launch();
    }
    cudaError_t e = w_zeroed ? cudaSuccess : cudaMemset2DAsync(W, ldw * sizeof(double), 0, n * sizeof(double), s, st);
    const dim3 grid((unsigned)((n + MV_ROWS - 1) / MV_ROWS), (unsigned)((n + MV_KC - 1) / MV_KC));
    const bool vec = (lda % 2 == 0) && ((reinterpret_cast<uintptr_t>(A) & 15) == 0);
    if (!vec || n % 2 != 0) Asp = nullptr;   // the split buffer is read as 16-byte pairs of columns
    for (int r0 = 0; r0 < s && e == cudaSuccess; r0 += MV_S) {
        ProfScope ps("df_matvec_kernel", st);
        if (vec)
            if (z_fp32)
                df_matvec_kernel<true, true><<<grid, MV_THREADS, 0, st>>>(A, n, lda, zs, s, r0, W, ldw, c->d_status,
                                                                          Asp, split_state);
            else
                df_matvec_kernel<true, false><<<grid, MV_THREADS, 0, st>>>(A, n, lda, zs, s, r0, W, ldw, c->d_status,
                                                                           Asp, split_state);
        else
            df_matvec_kernel<false, false><<<grid, MV_THREADS, 0, st>>>(A, n, lda, zs, s, r0, W, ldw, c->d_status,
                                                                        nullptr, nullptr);
        note_launch();
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    if (!work) dfree(c, zs, (size_t)n * s * sizeof(float2), st);
    if (e != cudaSuccess) {
        set_error("matvec launch: %s", cudaGetErrorString(e));
        return HODLR_CUDA_ERROR;
    }
    return HODLR_OK;
}

// ------------------------------------------------------------------ allocation-free matvec
// Scratch of hodlr_matvec_noalloc: the FP32 (hi, lo) split of Z lives in a
// file-scope device array instead of memory obtained from an allocator.  The
// array exists on every GPU that loads this library, for the life of the
// process.  Its device address is looked up once per device (host code may not
// use the symbol itself: on the host it only names a stand-in object).
namespace {

constexpr int64_t NOALLOC_MAX_ELEMS = int64_t(1) << 19;   // n * s <= 524288 (4 MiB of float2)
constexpr int NOALLOC_MAX_DEVICES = 64;

static __device__ __align__(256) float2 g_noalloc_split[NOALLOC_MAX_ELEMS];
static __device__ __align__(256) int g_noalloc_status[64];

struct NoallocSlot {
    float2 *split = nullptr;
    int *status = nullptr;
    bool ready = false;
};
NoallocSlot g_noalloc_slots[NOALLOC_MAX_DEVICES];
std::mutex g_noalloc_mu;

}  // namespace

}  // namespace hodlr

using namespace hodlr;

// W = A Z without allocating device memory: the same double-float kernels as
// hodlr_matvec, with the split of Z in the static array above.  Sizes with
// n * s above NOALLOC_MAX_ELEMS are refused with HODLR_RANGE.  The first call on
// a device resolves the array's device address (cudaGetSymbolAddress) with that
// device current.  Concurrent calls share the array and must not overlap on the
// GPU.  The call synchronises `stream` to report non-finite entries of A.
extern "C" hodlr_status hodlr_matvec_noalloc(const hodlr_matrix *A, int s, const double *Z, int64_t ldz, double *W,
                                             int64_t ldw, hodlr_stream stream) {
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (!A || !A->data || A->n <= 0 || A->ld < A->n || !Z || !W || s <= 0 || ldz < A->n || ldw < A->n) {
        set_error("hodlr_matvec_noalloc: invalid argument");
        return HODLR_INVALID_ARG;
    }
    const int64_t n = A->n;
    if (n * s > NOALLOC_MAX_ELEMS) {
        set_error("hodlr_matvec_noalloc: n * s = %lld exceeds the static scratch limit %lld",
                  (long long)(n * s), (long long)NOALLOC_MAX_ELEMS);
        return HODLR_RANGE;
    }
    int dev = 0;
    HODLR_TRY_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) {
        set_error("hodlr_matvec_noalloc: device %d beyond %d", dev, NOALLOC_MAX_DEVICES);
        return HODLR_RANGE;
    }
    NoallocSlot slot;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        NoallocSlot &sl = g_noalloc_slots[dev];
        if (!sl.ready) {
            void *p = nullptr, *q = nullptr;
            HODLR_TRY_CUDA(cudaGetSymbolAddress(&p, g_noalloc_split));
            HODLR_TRY_CUDA(cudaGetSymbolAddress(&q, g_noalloc_status));
            sl.split = reinterpret_cast<float2 *>(p);
            sl.status = reinterpret_cast<int *>(q);
            sl.ready = true;
        }
        slot = sl;
    }
    // the array keeps the previous call's contents: the status word and W start
    // at zero, the split is rewritten in full before it is read
    HODLR_TRY_CUDA(cudaMemsetAsync(slot.status, 0, sizeof(int), st));
    HODLR_TRY_CUDA(cudaMemset2DAsync(W, ldw * sizeof(double), 0, n * sizeof(double), s, st));
    const int blocks = (int)std::min<int64_t>((n * s + 255) / 256, 4096);
    split_vec_kernel<<<blocks, 256, 0, st>>>(Z, ldz, n, s, slot.split);
    note_launch();
    const dim3 grid((unsigned)((n + MV_ROWS - 1) / MV_ROWS), (unsigned)((n + MV_KC - 1) / MV_KC));
    const bool vec = (A->ld % 2 == 0) && ((reinterpret_cast<uintptr_t>(A->data) & 15) == 0);
    for (int r0 = 0; r0 < s; r0 += MV_S) {
        if (vec)
            df_matvec_kernel<true, false><<<grid, MV_THREADS, 0, st>>>(A->data, n, A->ld, slot.split, s, r0, W, ldw,
                                                                       slot.status, nullptr, nullptr);
        else
            df_matvec_kernel<false, false><<<grid, MV_THREADS, 0, st>>>(A->data, n, A->ld, slot.split, s, r0, W, ldw,
                                                                        slot.status, nullptr, nullptr);
        note_launch();
    }
    HODLR_TRY_CUDA(cudaGetLastError());
    int hstat = 0;
    HODLR_TRY_CUDA(cudaMemcpyAsync(&hstat, slot.status, sizeof(int), cudaMemcpyDeviceToHost, st));
    HODLR_TRY_CUDA(cudaStreamSynchronize(st));
    if (hstat) {
        set_error("hodlr_matvec_noalloc: non-finite or out-of-range entry in A");
        return status_from_word(hstat);
    }
    return HODLR_OK;
}

namespace {

struct IterGraph {
    hodlr_ctx *c = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    ~IterGraph() {   // handed to the context: torn down by the next solve
        if (exec || graph) {
            std::lock_guard<std::mutex> lock(c->cache_mu);
            c->graph_trash.push_back({exec, graph});
        }
    }
};

void empty_graph_trash(hodlr_ctx *c) {
    std::vector<std::pair<cudaGraphExec_t, cudaGraph_t>> t;
    {
        std::lock_guard<std::mutex> lock(c->cache_mu);
        t.swap(c->graph_trash);
    }
    for (auto &g : t) {
        if (g.first) cudaGraphExecDestroy(g.first);
        if (g.second) cudaGraphDestroy(g.second);
    }
}

struct GmresBufs {
    hodlr_ctx *c = nullptr;
    cudaStream_t st = nullptr;
    std::vector<std::pair<void *, size_t>> list;
    void *get(size_t bytes) {
        void *p = dalloc(c, bytes, st);
        if (p) list.push_back({p, bytes});
        return p;
    }
    ~GmresBufs() {
        for (auto &q : list) dfree(c, q.first, q.second, st);
    }
};

// One GMRES solve (one front): its buffers, the recorded iteration graph and
// the host's view of the last cycle report.  setup() validates and launches
// nothing that depends on the host; first_cycle() and next_cycle() enqueue a
// cycle and its report without waiting, take_report() reads the report once
// the stream has passed it, finish() fills the info and gives the result.
struct GmresJob {
    hodlr_ctx *c = nullptr;
    const hodlr_matrix *A = nullptr;
    int s = 0;
    const double *B = nullptr;
    int64_t ldb = 0;
    double *X = nullptr;
    int64_t ldx = 0;
    const hodlr_t *P = nullptr;
    double tol = 0.0;
    int max_iter = 0, m = 0;
    cudaStream_t st = nullptr;

    int64_t n = 0, vstride = 0, zstride = 0;
    int hstride = 0;
    GmresBufs bufs;
    IterGraph iter;
    GState gs{};
    TailArgs ta{};
    double *Vk = nullptr, *Zk = nullptr, *Wv = nullptr, *nrm = nullptr, *Zc = nullptr;
    void *zsw = nullptr;
    int *loops = nullptr, *split_state = nullptr;
    char *rep_dev = nullptr;
    float2 *Asp = nullptr;
    // tensor-core product (many right-hand sides): A's digit slices, Z's
    void *oza = nullptr, *ozz = nullptr;
    dim3 vgrid;
    int tail_grid = 0;
    size_t tail_smem = 0;
    long long body_kernels = 0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    size_t rbytes = 0;
    std::vector<char> rep_pageable;
    char *rep_host = nullptr;
    int restarts = 0;

    ~GmresJob() {
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    }
    const int *rep_i() const { return reinterpret_cast<const int *>(rep_host); }
    const double *rep_d() const { return reinterpret_cast<const double *>(rep_host + report_doff(s)); }

    // Work-buffer bytes of a solve of order n with s right-hand sides and
    // restart length m (the stored split of A included).
    static size_t device_bytes(int64_t n, int s, int m) {
        const double prod = oz_eligible(n, s) ? (double)oz_a_bytes(n) + (double)oz_z_bytes(n, s) : (double)n * n * 8;
        const double v = (double)n * (m + 1) * s * 8 + (double)n * m * s * 8 + (double)n * s * 24 +
                         (double)s * (m + 1) * (m + 8) * 8 + 8192.0 + prod;
        return (size_t)std::min(v, 1e18);
    }

    hodlr_status setup(char *host_slot) {
        if (!c || !A || !A->data || !B || !X || s <= 0 || A->n <= 0 || A->ld < A->n || ldb < A->n || ldx < A->n ||
            max_iter <= 0 || !(tol > 0.0) || m < 0) {
            set_error("gmres_solve: invalid argument");
            return HODLR_INVALID_ARG;
        }
        if (P && (P->n != A->n)) {
            set_error("gmres_solve: preconditioner size %lld != %lld", (long long)P->n, (long long)A->n);
            return HODLR_INVALID_ARG;
        }
        if (P && !P->factored) {
            set_error("gmres_solve: preconditioner not factored");
            return HODLR_NOT_FACTORED;
        }
        HODLR_TRY_CUDA(cudaSetDevice(c->device));
        n = A->n;
        m = m > 0 ? std::min(m, max_iter) : max_iter;
        vstride = n * (m + 1);
        zstride = n * m;
        hstride = m + 1;
        // every work buffer in one allocation
        Arena ar;
        // W, h1, h2, nrm, the integer block and the split flag are adjacent:
        // one memset clears them
        const size_t oVk = ar.take((size_t)vstride * s * 8), oZk = ar.take((size_t)zstride * s * 8),
                     oWv = ar.take((size_t)n * s * 8), oh1 = ar.take((size_t)s * hstride * 8),
                     oh2 = ar.take((size_t)s * hstride * 8), onrm = ar.take((size_t)s * 8),
                     oib = ar.take((size_t)(4 * s + 4) * sizeof(int)), osst = ar.take(256), ozero_end = ar.bytes,
                     oH = ar.take((size_t)s * (m + 1) * m * 8), ocs = ar.take((size_t)s * m * 8),
                     osn = ar.take((size_t)s * m * 8), og = ar.take((size_t)s * (m + 1) * 8),
                     obn = ar.take((size_t)s * 8), oest = ar.take((size_t)s * 8),
                     ozs = ar.take((size_t)n * s * sizeof(float2)), oZc = ar.take((size_t)n * s * 8),
                     olp = ar.take(256), orep = ar.take(report_bytes(s));
        bufs.c = c;
        bufs.st = st;
        iter.c = c;
        char *base = (char *)bufs.get(ar.bytes);
        if (!base) {
            set_error("gmres_solve: out of device memory (%zu bytes)", ar.bytes);
            return HODLR_OUT_OF_MEMORY;
        }
        Vk = (double *)(base + oVk);
        Zk = (double *)(base + oZk);
        Wv = (double *)(base + oWv);
        double *h1 = (double *)(base + oh1);
        double *h2 = (double *)(base + oh2);
        nrm = (double *)(base + onrm);
        gs.H = (double *)(base + oH);
        gs.cs = (double *)(base + ocs);
        gs.sn = (double *)(base + osn);
        gs.g = (double *)(base + og);
        gs.bnorm = (double *)(base + obn);
        gs.est = (double *)(base + oest);
        int *ibuf = (int *)(base + oib);
        zsw = base + ozs;
        Zc = (double *)(base + oZc);
        loops = (int *)(base + olp);
        // A's FP32 (hi, lo) pairs for the products after the first (ld n; skipped
        // when A's rows are not 16-byte aligned, n is odd, the buffer would exceed
        // 16 GiB or cannot be allocated: the products then split A every time)
        split_state = (int *)(base + osst);
        rep_dev = base + orep;
        if (oz_eligible(n, s)) {
            oza = bufs.get(oz_a_bytes(n));
            ozz = oza ? bufs.get(oz_z_bytes(n, s)) : nullptr;
            if (!ozz) oza = nullptr;   // the double-float product instead
            cudaGetLastError();
        }
        if (!oza && n % 2 == 0 && A->ld % 2 == 0 && (reinterpret_cast<uintptr_t>(A->data) & 15) == 0 &&
            (double)n * (double)n * 8.0 <= 16.0 * 1024 * 1024 * 1024) {
            Asp = reinterpret_cast<float2 *>(bufs.get((size_t)n * n * sizeof(float2)));
            cudaGetLastError();
        }
        gs.iters = ibuf;
        gs.jcur = ibuf + s;
        gs.active = ibuf + 2 * s;
        gs.nactive = ibuf + 3 * s;
        HODLR_TRY_CUDA(cudaEventCreate(&e0));
        HODLR_TRY_CUDA(cudaEventCreate(&e1));
        HODLR_TRY_CUDA(cudaEventRecord(e0, st));

        vgrid = dim3((unsigned)std::min<int64_t>((n + KT - 1) / KT, 1024), s);
        // x0 = 0; W, h1, h2, nrm, the iteration counters, per-rhs state and
        // the split flag start at zero
        HODLR_TRY_CUDA(cudaMemset2DAsync(X, ldx * 8, 0, n * 8, s, st));
        HODLR_TRY_CUDA(cudaMemsetAsync(base + oWv, 0, ozero_end - oWv, st));
        // R := B - 0 and nrm = ||R||^2
        residual_kernel<<<vgrid, KT, 0, st>>>(B, ldb, Wv, n, n, nrm);
        note_launch();
        if (oza) HODLR_TRY(oz_split_a(c, A->data, n, A->ld, oza, st));
        // ---- one Arnoldi iteration, recorded once and replayed by a device-side
        // while loop (a conditional graph node) until no right-hand side is active:
        // z = P^-1 v_j, w = A z, then the fused Gram-Schmidt / Givens step
        if (P) HODLR_TRY(solve_prepare(P, s, st));
        ta.Vk = Vk;
        ta.vstride = vstride;
        ta.n = n;
        ta.w = Wv;
        ta.Zc = Zc;
        ta.Zk = Zk;
        ta.zstride = zstride;
        ta.h1 = h1;
        ta.h2 = h2;
        ta.nrm = nrm;
        ta.hstride = hstride;
        ta.gs = gs;
        ta.m = m;
        ta.s = s;
        ta.max_iter = max_iter;
        ta.tol = tol;
        ta.bar = reinterpret_cast<unsigned *>(ibuf + 3 * s + 2);
        ta.status = c->d_status;
        ta.loops = loops;
        ta.limit = m + 1;
        ta.split_state = Asp ? split_state : nullptr;
        tail_smem = (size_t)(m + 1) * sizeof(double) + 2 * (size_t)s * sizeof(int);
        HODLR_TRY_CUDA(cudaFuncSetAttribute(arnoldi_tail_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)tail_smem));
        {
            int per_sm = 0;
            HODLR_TRY_CUDA(
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, arnoldi_tail_kernel, TT, tail_smem));
            if (per_sm <= 0) {
                set_error("gmres_solve: restart length %d needs too much shared memory", m);
                return HODLR_INVALID_ARG;
            }
            const int64_t units = ((n + TT - 1) / TT) * s;
            tail_grid = (int)std::max<int64_t>(1, std::min<int64_t>(units, (int64_t)c->num_sms * per_sm));
        }
        HODLR_TRY(record_graph());
        // the host's view of each cycle comes in one copy (pinned unless the
        // caller's slot is missing or too small)
        rbytes = report_bytes(s);
        rep_host = host_slot;
        if (!rep_host) {
            rep_pageable.resize(rbytes);
            rep_host = rep_pageable.data();
        }
        return HODLR_OK;
    }

    hodlr_status record_graph() {
        cudaStream_t cs = c->side[HODLR_SIDE_STREAMS - 1];
        HODLR_TRY_CUDA(cudaGraphCreate(&iter.graph, 0));
        cudaGraphConditionalHandle handle;
        HODLR_TRY_CUDA(cudaGraphConditionalHandleCreate(&handle, iter.graph, 1, cudaGraphCondAssignDefault));
        cudaGraphNodeParams cp = {};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = handle;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        cudaGraphNode_t knode, cnode;
        {
            const int *na = gs.nactive;
            void *kargs[] = {(void *)&na, (void *)&handle};
            cudaKernelNodeParams kp = {};
            kp.func = (void *)cond_init_kernel;
            kp.gridDim = dim3(1);
            kp.blockDim = dim3(1);
            kp.kernelParams = kargs;
            HODLR_TRY_CUDA(cudaGraphAddKernelNode(&knode, iter.graph, nullptr, 0, &kp));
        }
        HODLR_TRY_CUDA(cudaGraphAddNode(&cnode, iter.graph, &knode, nullptr, 1, &cp));
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        HODLR_TRY_CUDA(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
        auto record = [&]() -> hodlr_status {
            if (oza) {
                if (P) HODLR_TRY(solve_impl(P, s, Zc, n, cs));
                HODLR_TRY(oz_matvec(c, oza, n, s, Zc, n, Wv, n, ozz, cs));
            } else {
                // the apply also leaves z split into FP32 pairs for the product
                if (P) HODLR_TRY(solve_impl(P, s, Zc, n, cs, reinterpret_cast<float2 *>(zsw)));
                HODLR_TRY(matvec_impl(c, A->data, n, A->ld, s, Zc, n, Wv, n, cs, zsw, true, Asp, split_state,
                                      P != nullptr, P != nullptr && P->prec != HODLR_FP64));
            }
            ta.handle = handle;
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3((unsigned)tail_grid);
            cfg.blockDim = dim3(TT);
            cfg.dynamicSmemBytes = tail_smem;
            cfg.stream = cs;
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeCooperative;
            attr[0].val.cooperative = 1;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            HODLR_TRY_CUDA(cudaLaunchKernelEx(&cfg, arnoldi_tail_kernel, ta));
            note_launch();
            return HODLR_OK;
        };
        hodlr_status rs;
        {
            LaunchCapture cap;
            rs = record();
            body_kernels = cap.captured;
        }
        cudaGraph_t captured = nullptr;
        const cudaError_t ce = cudaStreamEndCapture(cs, &captured);
        if (rs != HODLR_OK) return rs;
        if (ce != cudaSuccess) {
            set_error("gmres_solve: graph capture failed: %s", cudaGetErrorString(ce));
            return HODLR_CUDA_ERROR;
        }
        HODLR_TRY_CUDA(cudaGraphInstantiate(&iter.exec, iter.graph, 0));
        return HODLR_OK;
    }

    // One cycle from the current start vector: the Arnoldi iterations (graph),
    // x += Z y and the true residual R = B - A X.
    hodlr_status launch_cycle(bool first) {
        if (first) {
            count_active_kernel<<<1, 1, 0, st>>>(gs.active, s, gs.nactive);
            note_launch();
        }
        HODLR_TRY_CUDA(cudaMemsetAsync(loops, 0, sizeof(int), st));
        HODLR_TRY_CUDA(cudaGraphLaunch(iter.exec, st));
        note_launch();   // the graph's test of the count
        if (first) empty_graph_trash(c);   // earlier solves' graphs, while this one runs
        // x += Z y
        backsolve_kernel<<<dim3((unsigned)std::min<int64_t>((n + KT - 1) / KT, 64), s), KT, (size_t)m * 8, st>>>(
            gs, m, Zk, zstride, n, X, ldx);
        note_launch();
        HODLR_TRY_CUDA(cudaGetLastError());
        if (oza)
            HODLR_TRY(oz_matvec(c, oza, n, s, X, ldx, Wv, n, ozz, st));
        else
            HODLR_TRY(matvec_impl(c, A->data, n, A->ld, s, X, ldx, Wv, n, st, zsw, false, Asp, split_state));
        HODLR_TRY_CUDA(cudaMemsetAsync(nrm, 0, (size_t)s * 8, st));
        residual_kernel<<<vgrid, KT, 0, st>>>(B, ldb, Wv, n, n, nrm);
        note_launch();
        HODLR_TRY_CUDA(cudaGetLastError());
        return HODLR_OK;
    }

    // The first cycle (the graph tests the count itself, so it is launched
    // without a host round trip), then the restart test and its report.
    hodlr_status first_cycle() {
        start_cycle_kernel<<<vgrid, KT, 0, st>>>(gs, m, s, Wv, n, n, nrm, Vk, vstride, tol, max_iter, true, Zc);
        note_launch();
        HODLR_TRY(launch_cycle(true));
        return enqueue_report();
    }
    hodlr_status next_cycle() {
        ++restarts;
        HODLR_TRY(launch_cycle(false));
        return enqueue_report();
    }
    // Restart test from the true residual (a right-hand side stays active
    // while its residual is above tol), then the report copy.
    hodlr_status enqueue_report() {
        start_cycle_kernel<<<vgrid, KT, 0, st>>>(gs, m, s, Wv, n, n, nrm, Vk, vstride, tol, max_iter, false, Zc);
        note_launch();
        HODLR_TRY_CUDA(cudaEventRecord(e1, st));
        cycle_report_kernel<<<1, 32, 0, st>>>(gs, s, nrm, c->d_status, loops, rep_dev);
        note_launch();
        HODLR_TRY_CUDA(cudaMemcpyAsync(rep_host, rep_dev, rbytes, cudaMemcpyDeviceToHost, st));
        return HODLR_OK;
    }
    // After the stream has passed the report: false once every rhs is done.
    hodlr_status take_report(bool &more) {
        note_launch((long long)rep_i()[2] * body_kernels);   // replays of the last cycle
        HODLR_TRY(status_word(rep_i()[1]));
        more = rep_i()[0] != 0 && restarts < 10000;
        return HODLR_OK;
    }

    hodlr_status finish(hodlr_gmres_info *info) {
        hodlr_status result = HODLR_OK;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        const int *ri = rep_i();
        const double *rd = rep_d();
        for (int r = 0; r < s; ++r) {
            const double bn = rd[2 * s + r];
            const double tr = bn > 0.0 ? std::sqrt(rd[s + r]) / bn : 0.0;
            if (!(tr <= tol)) result = HODLR_NOT_CONVERGED;
            if (info) {
                if (info->iters) info->iters[r] = ri[3 + r];
                if (info->est_relres) info->est_relres[r] = rd[r];
                if (info->true_relres) info->true_relres[r] = tr;
            }
        }
        if (info) {
            info->restarts = restarts;
            info->ms_total = ms;
        }
        if (result == HODLR_NOT_CONVERGED) set_error("gmres_solve: not converged within %d iterations", max_iter);
        return result;
    }

    // Restarted cycles, each waited for, until every rhs is done.
    hodlr_status run_to_end(hodlr_gmres_info *info) {
        bool more = false;
        HODLR_TRY(take_report(more));
        while (more) {
            HODLR_TRY(next_cycle());
            HODLR_TRY_CUDA(cudaStreamSynchronize(st));
            HODLR_TRY(take_report(more));
        }
        return finish(info);
    }
};

size_t report_slot(int s) { return (report_bytes(s) + 63) & ~size_t(63); }

}  // namespace

extern "C" hodlr_status gmres_solve(hodlr_ctx *c, const hodlr_matrix *A, int s, const double *B, int64_t ldb,
                                    double *X, int64_t ldx, const hodlr_t *P, double tol, int max_iter, int restart,
                                    hodlr_gmres_info *info, hodlr_stream stream) {
    if (!c) {
        set_error("gmres_solve: invalid argument");
        return HODLR_INVALID_ARG;
    }
    GmresJob j;
    j.c = c;
    j.A = A;
    j.s = s;
    j.B = B;
    j.ldb = ldb;
    j.X = X;
    j.ldx = ldx;
    j.P = P;
    j.tol = tol;
    j.max_iter = max_iter;
    j.m = restart;
    j.st = reinterpret_cast<cudaStream_t>(stream);
    const bool pinned = s > 0 && report_bytes(s) <= HODLR_REPORT_BYTES;
    HODLR_TRY(j.setup(pinned ? reinterpret_cast<char *>(c->h_report) : nullptr));
    HODLR_TRY(j.first_cycle());
    HODLR_TRY_CUDA(cudaStreamSynchronize(j.st));
    return j.run_to_end(info);
}

// Fronts are taken in windows: every front of a window is set up and its first
// cycle and report enqueued without a host wait (each report in its own slot of
// the context's pinned buffer), the fronts spread over several streams so that
// their small dependent kernels overlap; one synchronisation then covers the
// window, and only fronts that need a restart wait again.  A window holds
// at most HODLR_REPORT_BYTES of reports, about 8 GiB of work buffers and each
// preconditioner once.
extern "C" hodlr_status gmres_solve_batched(hodlr_ctx *c, int nf, const hodlr_matrix *A, const int *s,
                                            const double *const *B, const int64_t *ldb, double *const *X,
                                            const int64_t *ldx, const hodlr_t *const *P, double tol, int max_iter,
                                            int restart, hodlr_gmres_info *info, hodlr_stream stream) {
    using namespace hodlr;
    if (!c || nf < 0 || (nf > 0 && (!A || !s || !B || !ldb || !X || !ldx))) {
        set_error("gmres_solve_batched: invalid argument");
        return HODLR_INVALID_ARG;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    HODLR_TRY_CUDA(cudaSetDevice(c->device));
    const size_t mem_window = (size_t)8 << 30;
    // fronts are independent: they go round-robin onto the context's side
    // streams (all but the one graphs are captured on), which start after the
    // work already on `stream` and are waited for by the host before return
    constexpr int NS = HODLR_SIDE_STREAMS - 1;
    cudaEvent_t ready = nullptr;
    HODLR_TRY_CUDA(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
    struct EventGuard {
        cudaEvent_t e;
        ~EventGuard() { cudaEventDestroy(e); }
    } ready_guard{ready};
    HODLR_TRY_CUDA(cudaEventRecord(ready, st));
    for (int q = 0; q < NS; ++q) HODLR_TRY_CUDA(cudaStreamWaitEvent(c->side[q], ready, 0));
    auto sync_side = [&]() -> hodlr_status {
        for (int q = 0; q < NS; ++q) HODLR_TRY_CUDA(cudaStreamSynchronize(c->side[q]));
        return HODLR_OK;
    };
    hodlr_status result = HODLR_OK;
    for (int f0 = 0; f0 < nf;) {
        std::vector<std::unique_ptr<GmresJob>> jobs;
        std::vector<const hodlr_t *> seen;
        size_t rep_used = 0, mem_used = 0;
        int f = f0;
        for (; f < nf; ++f) {
            const int sf = s[f] > 0 ? s[f] : 1;
            const int64_t nn = A[f].n > 0 ? A[f].n : 1;
            const int mf = restart > 0 ? std::min(restart, std::max(max_iter, 1)) : std::max(max_iter, 1);
            const size_t rb = report_slot(sf), mb = GmresJob::device_bytes(nn, sf, mf);
            // a preconditioner met again in the window ends it: its work buffers
            // may be resized for the new front while an earlier graph uses them
            const hodlr_t *pf = P ? P[f] : nullptr;
            if (f > f0 && (rep_used + rb > HODLR_REPORT_BYTES || mem_used + mb > mem_window ||
                           (pf && std::find(seen.begin(), seen.end(), pf) != seen.end())))
                break;
            if (pf) seen.push_back(pf);
            auto j = std::make_unique<GmresJob>();
            j->c = c;
            j->A = &A[f];
            j->s = s[f];
            j->B = B[f];
            j->ldb = ldb[f];
            j->X = X[f];
            j->ldx = ldx[f];
            j->P = pf;
            j->tol = tol;
            j->max_iter = max_iter;
            j->m = restart;
            j->st = c->side[(f - f0) % NS];
            char *slot = rep_used + rb <= HODLR_REPORT_BYTES ? reinterpret_cast<char *>(c->h_report) + rep_used
                                                             : nullptr;
            rep_used += rb;
            mem_used += mb;
            hodlr_status r = j->setup(slot);
            if (r == HODLR_OK) r = j->first_cycle();
            if (r != HODLR_OK) {
                sync_side();
                return r;
            }
            jobs.push_back(std::move(j));
        }
        HODLR_TRY(sync_side());
        for (size_t k = 0; k < jobs.size(); ++k) {
            const hodlr_status r = jobs[k]->run_to_end(info ? &info[f0 + k] : nullptr);
            if (r == HODLR_NOT_CONVERGED)
                result = HODLR_NOT_CONVERGED;
            else if (r != HODLR_OK) {
                sync_side();
                return r;
            }
        }
        f0 = f;
    }
    // every side stream idle on return: work queued next on `stream` sees X
    HODLR_TRY(sync_side());
    if (result == HODLR_NOT_CONVERGED) set_error("gmres_solve_batched: some front did not converge");
    return result;
}
