// Applying the factored HODLR inverse, X <- K~^-1 X (Sec. 4.3, Solve):
//   leaves:  x_leaf <- K_leaf^-1 x_leaf
//   for c = L .. 1 (children level), every parent node (alpha, beta):
//       w = [V_ba^T x_alpha ; V_ab^T x_beta]         (segmented reductions)
//       y = S^-1 w                                   (one GEMV per node)
//       x_alpha -= d_alpha y2,  x_beta -= d_beta y1  (rank-rp updates)
// X is FP64 in and out; the arithmetic runs in the factor's precision T on a
// private copy of X.  Memory-bound: each level streams V and d once.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>

#include "internal.cuh"

namespace hodlr {
namespace {

constexpr int AP_THREADS = 256;
constexpr int MAX_RHS_CHUNK = 8;

// Storage -> arithmetic type of the streamed factors (V, d): FP64, FP32, or a
// 16-bit copy (BF16, or FP16 scaled per node and column by a power of two).
template <typename T>
__device__ __forceinline__ T to_t(double x) { return (T)x; }
template <typename T>
__device__ __forceinline__ T to_t(float x) { return (T)x; }
template <typename T>
__device__ __forceinline__ T to_t(__nv_bfloat16 x) { return (T)__bfloat162float(x); }
template <typename T>
__device__ __forceinline__ T to_t(__half x) { return (T)__half2float(x); }

// x_T(leaf rows, r) = Kinv_leaf * X(leaf rows, r).  One CTA per (leaf, rhs).
template <typename T>
__global__ void __launch_bounds__(AP_THREADS)
    leaf_apply_kernel(const T *__restrict__ Kinv, int bmax, const int64_t *__restrict__ bounds,
                      const double *__restrict__ X, int64_t ldx, T *__restrict__ xt, int64_t ldt) {
    const int leaf = blockIdx.x, r = blockIdx.y;
    const int64_t r0 = bounds[leaf], b = bounds[leaf + 1] - r0;
    extern __shared__ __align__(16) unsigned char smem[];
    T *xs = reinterpret_cast<T *>(smem);
    for (int64_t i = threadIdx.x; i < b; i += AP_THREADS) xs[i] = dev::from_double<T>(X[r0 + i + r * ldx]);
    __syncthreads();
    const T *K = Kinv + (size_t)leaf * bmax * bmax;
    for (int64_t i = threadIdx.x; i < b; i += AP_THREADS) {
        T acc = T(0);
        for (int64_t k = 0; k < b; ++k) acc = fma(K[i + k * bmax], xs[k], acc);
        xt[r0 + i + r * ldt] = acc;
    }
}

// w(child, col, r) += sum_{rows of child} V(row, coff+col) x(row, r).
// Grid: (child * row-chunks, column groups); one warp per column.  vscale (or
// NULL) holds the dequantisation factor of each (child, column).
template <typename T, typename S>
__global__ void __launch_bounds__(AP_THREADS)
    vtx_kernel(const S *__restrict__ V, int64_t ldn, int64_t coff, int rp, const int64_t *__restrict__ bounds,
               int L, int c, int chunks, int64_t chunk_rows, const T *__restrict__ xt, int64_t ldt,
               int s, T *__restrict__ w, const float *__restrict__ vscale) {
    const int child = blockIdx.x / chunks, ch = blockIdx.x % chunks;
    const int64_t n0 = bounds[(size_t)child << (L - c)];
    const int64_t n1 = bounds[(size_t)(child + 1) << (L - c)];
    const int64_t a = n0 + ch * chunk_rows;
    const int64_t e = (a + chunk_rows < n1) ? a + chunk_rows : n1;
    if (a >= e) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int col = blockIdx.y * (AP_THREADS / 32) + warp;
    if (col >= rp) return;
    const S *vc = V + (coff + col) * ldn;
    const T sc = vscale ? (T)vscale[(size_t)child * rp + col] : T(1);
    T acc[MAX_RHS_CHUNK];
    for (int r0 = 0; r0 < s; r0 += MAX_RHS_CHUNK) {
        const int rr = (s - r0) < MAX_RHS_CHUNK ? (s - r0) : MAX_RHS_CHUNK;
#pragma unroll
        for (int q = 0; q < MAX_RHS_CHUNK; ++q) acc[q] = T(0);
        for (int64_t i = a + lane; i < e; i += 32) {
            const T v = to_t<T>(vc[i]);
#pragma unroll
            for (int q = 0; q < MAX_RHS_CHUNK; ++q)
                if (q < rr) acc[q] = fma(v, xt[i + (r0 + q) * ldt], acc[q]);
        }
#pragma unroll
        for (int q = 0; q < MAX_RHS_CHUNK; ++q) {
            if (q >= rr) break;
            T v = acc[q];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) atomicAdd(&w[((size_t)child * rp + col) * s + r0 + q], v * sc);
        }
    }
}

// y(node) = S^-1 [w(alpha); w(beta)] for every RHS.  Grid (node, 32-row tiles of
// S^-1): lane = output row, the 8 warps split the inner dimension, partial sums
// are reduced in shared memory.
constexpr int TR = 32;   // rows per CTA in the row-tiled apply kernels

template <typename T>
__global__ void __launch_bounds__(AP_THREADS)
    core_apply_kernel(const T *__restrict__ Sinv, int rp, const T *__restrict__ w, int s, T *__restrict__ y) {
    const int node = blockIdx.x;
    const int s2 = 2 * rp;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int i = blockIdx.y * TR + lane;
    extern __shared__ __align__(16) unsigned char smem[];
    T *ws = reinterpret_cast<T *>(smem);          // s2 * s
    T *part = ws + (size_t)s2 * s;                // 8 warps * TR * MAX_RHS_CHUNK
    const T *wn = w + (size_t)node * s2 * s;      // children 2 node, 2 node + 1 are contiguous
    for (int e = threadIdx.x; e < s2 * s; e += AP_THREADS) ws[e] = wn[e];
    __syncthreads();
    const T *S = Sinv + (size_t)node * s2 * s2;
    const int kper = (s2 + 7) / 8, kb = warp * kper, ke = min(s2, kb + kper);
    for (int r0 = 0; r0 < s; r0 += MAX_RHS_CHUNK) {
        const int rr = (s - r0) < MAX_RHS_CHUNK ? (s - r0) : MAX_RHS_CHUNK;
        T acc[MAX_RHS_CHUNK];
#pragma unroll
        for (int q = 0; q < MAX_RHS_CHUNK; ++q) acc[q] = T(0);
        if (i < s2) {
#pragma unroll 4
            for (int k = kb; k < ke; ++k) {
                const T sv = S[i + (size_t)k * s2];
#pragma unroll
                for (int q = 0; q < MAX_RHS_CHUNK; ++q)
                    if (q < rr) acc[q] = fma(sv, ws[k * s + r0 + q], acc[q]);
            }
        }
#pragma unroll
        for (int q = 0; q < MAX_RHS_CHUNK; ++q) part[(warp * TR + lane) * MAX_RHS_CHUNK + q] = acc[q];
        __syncthreads();
        for (int e = threadIdx.x; e < TR * rr; e += AP_THREADS) {
            const int li = e % TR, q = e / TR;
            T v = T(0);
            for (int wv = 0; wv < AP_THREADS / 32; ++wv) v += part[(wv * TR + li) * MAX_RHS_CHUNK + q];
            const int ii = blockIdx.y * TR + li;
            if (ii < s2) y[((size_t)node * s2 + ii) * s + r0 + q] = v;
        }
        __syncthreads();
    }
}

// x(child rows, r) -= d(child rows, coff:coff+rp) * y_sib(:, r), y_sib = y2 for the
// first child (alpha) and y1 for the second (beta).
// Rows are tiled by TR = 32 per CTA (lane = row); the 8 warps split the rp
// columns of d and the partial sums are reduced in shared memory.
template <typename T, typename S>
__global__ void __launch_bounds__(AP_THREADS)
    update_kernel(const S *__restrict__ Dm, int64_t ldn, int64_t coff, int rp,
                  const int64_t *__restrict__ bounds, int L, int c, int chunks, int64_t chunk_rows,
                  const T *__restrict__ y, int s, T *__restrict__ xt, int64_t ldt, const float *__restrict__ dscale) {
    const int child = blockIdx.x / chunks, ch = blockIdx.x % chunks;
    const int64_t n0 = bounds[(size_t)child << (L - c)];
    const int64_t n1 = bounds[(size_t)(child + 1) << (L - c)];
    const int64_t a = n0 + ch * chunk_rows;
    const int64_t e = (a + chunk_rows < n1) ? a + chunk_rows : n1;
    if (a >= e) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    extern __shared__ __align__(16) unsigned char smem[];
    T *ys = reinterpret_cast<T *>(smem);     // rp * s
    T *part = ys + (size_t)rp * s;           // 8 warps * TR * MAX_RHS_CHUNK
    const int node = child >> 1;
    const int half = (child & 1) ? 0 : rp;   // alpha uses y2 (second half)
    const T *yn = y + ((size_t)node * 2 * rp + half) * s;
    for (int q = threadIdx.x; q < rp * s; q += AP_THREADS)
        ys[q] = dscale ? yn[q] * (T)dscale[(size_t)child * rp + q / s] : yn[q];
    __syncthreads();
    const int kper = (rp + 7) / 8, kb = warp * kper, ke = min(rp, kb + kper);
    const int64_t i = a + lane;
    for (int r0 = 0; r0 < s; r0 += MAX_RHS_CHUNK) {
        const int rr = (s - r0) < MAX_RHS_CHUNK ? (s - r0) : MAX_RHS_CHUNK;
        T acc[MAX_RHS_CHUNK];
#pragma unroll
        for (int q = 0; q < MAX_RHS_CHUNK; ++q) acc[q] = T(0);
        if (i < e) {
#pragma unroll 4
            for (int k = kb; k < ke; ++k) {
                const T dv = to_t<T>(Dm[i + (coff + k) * ldn]);
#pragma unroll
                for (int q = 0; q < MAX_RHS_CHUNK; ++q)
                    if (q < rr) acc[q] = fma(dv, ys[k * s + r0 + q], acc[q]);
            }
        }
#pragma unroll
        for (int q = 0; q < MAX_RHS_CHUNK; ++q) part[(warp * TR + lane) * MAX_RHS_CHUNK + q] = acc[q];
        __syncthreads();
        for (int t = threadIdx.x; t < TR * rr; t += AP_THREADS) {
            const int li = t % TR, q = t / TR;
            const int64_t ii = a + li;
            if (ii >= e) continue;
            T v = T(0);
            for (int wv = 0; wv < AP_THREADS / 32; ++wv) v += part[(wv * TR + li) * MAX_RHS_CHUNK + q];
            xt[ii + (r0 + q) * ldt] -= v;
        }
        __syncthreads();
    }
}

template <typename T>
__global__ void store_kernel(const T *__restrict__ xt, int64_t ldt, int64_t n, int s, double *__restrict__ X,
                             int64_t ldx) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * s;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e % n, r = e / n;
        X[i + r * ldx] = (double)xt[i + r * ldt];
    }
}

template <typename T>
__global__ void zero_kernel2(T *p, int64_t count) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count;
         e += (int64_t)gridDim.x * blockDim.x)
        p[e] = T(0);
}

template <typename T, typename S>
hodlr_status solve_typed(const hodlr_t *h, int s, double *X, int64_t ldx, cudaStream_t st, const S *V,
                         const S *Dm, const float *const *vsc, const float *const *dsc) {
    const int L = h->L;
    const int64_t n = h->n, ldn = h->ldn;
    hodlr_t *hm = const_cast<hodlr_t *>(h);
    // scratch: x_T (ldn * s), w (n*... <= 2^L * rpmax * s), y (same)
    int rpmax = 0;
    for (int c = 1; c <= L; ++c) rpmax = std::max(rpmax, h->lv[c].rp);
    const size_t xt_bytes = (size_t)ldn * s * sizeof(T);
    const size_t w_elems = (size_t)(1 << L) * std::max(rpmax, 1) * s;
    const size_t need = xt_bytes + 2 * w_elems * sizeof(T) + 1024;
    if (hm->work_bytes < need) {
        HODLR_TRY(ensure_work(hm, need, st));
    }
    char *wp = reinterpret_cast<char *>(hm->work);
    T *xt = reinterpret_cast<T *>(wp);
    T *w = reinterpret_cast<T *>(wp + ((xt_bytes + 255) & ~size_t(255)));
    T *y = w + w_elems;
    const T *Kinv = reinterpret_cast<const T *>(h->leafinv);
    {
        dim3 grid(1 << L, s);
        size_t sm = (size_t)h->bmax * sizeof(T);
        leaf_apply_kernel<T><<<grid, AP_THREADS, sm, st>>>(Kinv, h->bmax, h->d_bounds, X, ldx, xt, ldn);
        HODLR_TRY_CUDA(cudaGetLastError());
    }
    for (int c = L; c >= 1; --c) {
        const int rp = h->lv[c].rp;
        if (rp == 0) continue;
        const int64_t coff = h->lv[c].coff;
        const int nch = 1 << c;
        int64_t node_rows = 0;
        for (int i = 0; i < nch; ++i)
            node_rows = std::max(node_rows, h->bounds[(size_t)(i + 1) << (L - c)] - h->bounds[(size_t)i << (L - c)]);
        const int64_t chunk_rows = 256;
        const int chunks = (int)((node_rows + chunk_rows - 1) / chunk_rows);
        {
            int64_t cnt = (int64_t)nch * rp * s;
            int blocks = (int)std::min<int64_t>((cnt + 255) / 256, 1024);
            zero_kernel2<T><<<blocks, 256, 0, st>>>(w, cnt);
            dim3 grid(nch * chunks, (rp + AP_THREADS / 32 - 1) / (AP_THREADS / 32));
            vtx_kernel<T, S><<<grid, AP_THREADS, 0, st>>>(V, ldn, coff, rp, h->d_bounds, L, c, chunks, chunk_rows,
                                                           xt, ldn, s, w, vsc ? vsc[c] : nullptr);
            HODLR_TRY_CUDA(cudaGetLastError());
        }
        const size_t part_bytes = (size_t)(AP_THREADS / 32) * TR * MAX_RHS_CHUNK * sizeof(T);
        {
            const T *Sinv = reinterpret_cast<const T *>(h->Sinv[c - 1]);
            const size_t sm = (size_t)2 * rp * s * sizeof(T) + part_bytes;
            if (sm > 48 * 1024)
                HODLR_TRY_CUDA(cudaFuncSetAttribute(core_apply_kernel<T>,
                                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
            dim3 grid(nch / 2, (2 * rp + TR - 1) / TR);
            core_apply_kernel<T><<<grid, AP_THREADS, sm, st>>>(Sinv, rp, w, s, y);
            HODLR_TRY_CUDA(cudaGetLastError());
        }
        {
            const int64_t urows = TR;
            const int uchunks = (int)((node_rows + urows - 1) / urows);
            const size_t sm = (size_t)rp * s * sizeof(T) + part_bytes;
            if (sm > 48 * 1024)
                HODLR_TRY_CUDA(cudaFuncSetAttribute(update_kernel<T, S>,
                                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
            update_kernel<T, S><<<nch * uchunks, AP_THREADS, sm, st>>>(Dm, ldn, coff, rp, h->d_bounds, L, c, uchunks,
                                                                        urows, y, s, xt, ldn, dsc ? dsc[c] : nullptr);
            HODLR_TRY_CUDA(cudaGetLastError());
        }
    }
    {
        int blocks = (int)std::min<int64_t>((n * s + 255) / 256, 4096);
        store_kernel<T><<<blocks, 256, 0, st>>>(xt, ldn, n, s, X, ldx);
        HODLR_TRY_CUDA(cudaGetLastError());
    }
    return HODLR_OK;
}

// ------------------------------------------------------------------ fused apply
// The whole apply in one cooperative launch.  Work is cut into 32-row tiles of
// the leaves (a tile lies inside one node of every level).  Phases, with a
// grid barrier after each:
//   A(L)   per tile: x = K_leaf^-1 x on its rows, then its partial V_L^T x
//   B(c)   per (node, 32 rows of S^-1): y(c) = S^-1 w(c); zero w(c-1)
//   A(c-1) per tile: x -= d(c) y_sib(c) on its rows, then its partial
//          V_(c-1)^T x (or, after level 1, the FP64 store of x)
// The barrier is a counter/generation pair in global memory; every wait gives
// up after a bounded number of polls and raises the timeout status bit.
constexpr int FA_RC = 8;   // right-hand sides per pass
constexpr unsigned long long FA_SPIN_LIMIT = 1ull << 26;

template <typename T, typename S>
struct FusedArgs {
    const T *Kinv;
    int bmax, L, s, rpmax;
    int64_t n, ldn, ldx;
    const S *V;
    const S *D;
    int rp[HODLR_MAX_LEVELS];
    int64_t coff[HODLR_MAX_LEVELS];
    const T *Sinv[HODLR_MAX_LEVELS];       // by parent level l = c - 1
    const float *vscale[HODLR_MAX_LEVELS];
    const float *dscale[HODLR_MAX_LEVELS];
    T *w[2];                               // w(c) in w[c & 1]
    T *y;
    T *xt;
    const int4 *tiles;                     // (leaf, first row, rows, 0)
    int ntiles;
    const int64_t *bounds;
    double *X;
    unsigned *bar;
    int *status;
};

__device__ void grid_sync(unsigned *bar, int *status) {
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
                if (++spins > FA_SPIN_LIMIT) {
                    atomicOr(status, ST_TIMEOUT);
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
    }
    __syncthreads();
}

// Lane-row / warp-split reduction helper: part[warp][lane][q] -> sum over warps.
template <typename T>
__device__ __forceinline__ T warp_parts_sum(const T *part, int lane_row, int q) {
    T v = T(0);
#pragma unroll
    for (int wv = 0; wv < AP_THREADS / 32; ++wv) v += part[(wv * TR + lane_row) * FA_RC + q];
    return v;
}

// Partial V_c^T x over one tile's rows into w(c): the tile's block of V (32
// rows x rp, coalesced column reads) and of x are staged in shared memory, then
// one thread per column forms its 32-term dot products (padded stride: no bank
// conflicts) and adds them to w with one atomic per (column, rhs).
template <typename T, typename S>
__device__ void fa_vtx(const FusedArgs<T, S> &a, int c, int child, int64_t row0, int nrows, int r0, int rr,
                       T *sv, T *xs) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int rp = a.rp[c];
    const S *Vc = a.V + a.coff[c] * a.ldn;
    T *w = a.w[c & 1];
    const float *vs = a.vscale[c];
    for (int col = warp; col < rp; col += AP_THREADS / 32)
        sv[col * (TR + 1) + lane] = (lane < nrows) ? to_t<T>(Vc[row0 + lane + (int64_t)col * a.ldn]) : T(0);
    for (int e = threadIdx.x; e < TR * FA_RC; e += AP_THREADS) {
        const int li = e % TR, q = e / TR;
        xs[q * TR + li] = (li < nrows && q < rr) ? a.xt[row0 + li + (r0 + q) * a.ldn] : T(0);
    }
    __syncthreads();
    for (int col = threadIdx.x; col < rp; col += AP_THREADS) {
        T acc[FA_RC];
#pragma unroll
        for (int q = 0; q < FA_RC; ++q) acc[q] = T(0);
#pragma unroll 8
        for (int li = 0; li < TR; ++li) {
            const T v = sv[col * (TR + 1) + li];
#pragma unroll
            for (int q = 0; q < FA_RC; ++q) acc[q] = fma(v, xs[q * TR + li], acc[q]);
        }
        const T sc = vs ? (T)vs[(size_t)child * rp + col] : T(1);
#pragma unroll
        for (int q = 0; q < FA_RC; ++q)
            if (q < rr) atomicAdd(&w[((size_t)child * rp + col) * a.s + r0 + q], acc[q] * sc);
    }
    __syncthreads();
}

template <typename T, typename S>
__global__ void __launch_bounds__(AP_THREADS) apply_fused_kernel(const FusedArgs<T, S> a) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    extern __shared__ __align__(16) unsigned char smem[];
    T *part = reinterpret_cast<T *>(smem);                          // 8 warps x 32 rows x FA_RC
    T *ys = part + (AP_THREADS / 32) * TR * FA_RC;                  // staged y: up to 2 rp x FA_RC
    T *sv = ys + 2 * (size_t)a.rpmax * FA_RC;                       // V tile: rp x (32 + 1)
    T *xs = sv + (size_t)a.rpmax * (TR + 1);                        // x tile: FA_RC x 32
    const int L = a.L;
    // ---- A(L): leaf solves and the leaf level's V^T x
    for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
        const int4 tl = a.tiles[t];
        const int leaf = tl.x, nrows = tl.z;
        const int64_t row0 = tl.y;
        const int64_t l0 = a.bounds[leaf];
        const int b = (int)(a.bounds[leaf + 1] - l0);
        const T *K = a.Kinv + (size_t)leaf * a.bmax * a.bmax;
        const int il = (int)(row0 - l0) + lane;
        const int kper = (b + 7) / 8, kb = warp * kper, ke = min(b, kb + kper);
        for (int r0 = 0; r0 < a.s; r0 += FA_RC) {
            const int rr = min(FA_RC, a.s - r0);
            T acc[FA_RC];
#pragma unroll
            for (int q = 0; q < FA_RC; ++q) acc[q] = T(0);
            if (lane < nrows) {
                for (int k = kb; k < ke; ++k) {
                    const T kv = K[il + (size_t)k * a.bmax];
#pragma unroll
                    for (int q = 0; q < FA_RC; ++q)
                        if (q < rr) acc[q] = fma(kv, dev::from_double<T>(a.X[l0 + k + (r0 + q) * a.ldx]), acc[q]);
                }
            }
#pragma unroll
            for (int q = 0; q < FA_RC; ++q) part[(warp * TR + lane) * FA_RC + q] = acc[q];
            __syncthreads();
            for (int e = threadIdx.x; e < TR * rr; e += AP_THREADS) {
                const int li = e % TR, q = e / TR;
                if (li < nrows) a.xt[row0 + li + (r0 + q) * a.ldn] = warp_parts_sum(part, li, q);
            }
            __syncthreads();
            if (L >= 1) fa_vtx(a, L, leaf, row0, nrows, r0, rr, sv, xs);
            __syncthreads();
        }
    }
    if (L == 0) {
        grid_sync(a.bar, a.status);
        for (int64_t e = blockIdx.x * (int64_t)AP_THREADS + threadIdx.x; e < a.n * a.s;
             e += (int64_t)gridDim.x * AP_THREADS) {
            const int64_t i = e % a.n, r = e / a.n;
            a.X[i + r * a.ldx] = (double)a.xt[i + r * a.ldn];
        }
        return;
    }
    grid_sync(a.bar, a.status);
    for (int c = L; c >= 1; --c) {
        const int rp = a.rp[c];
        const int s2 = 2 * rp;
        const int nn = 1 << (c - 1);
        // ---- B(c): y = S^-1 w per node; zero the other w buffer for level c - 1
        if (rp > 0) {
            const T *wc = a.w[c & 1];
            const int rtiles = (s2 + TR - 1) / TR;
            for (int item = blockIdx.x; item < nn * rtiles; item += gridDim.x) {
                const int node = item / rtiles, rt = item % rtiles;
                const T *Sn = a.Sinv[c - 1] + (size_t)node * s2 * s2;
                const T *wn = wc + (size_t)node * s2 * a.s;
                const int i = rt * TR + lane;
                const int kper = (s2 + 7) / 8, kb = warp * kper, ke = min(s2, kb + kper);
                for (int r0 = 0; r0 < a.s; r0 += FA_RC) {
                    const int rr = min(FA_RC, a.s - r0);
                    T acc[FA_RC];
#pragma unroll
                    for (int q = 0; q < FA_RC; ++q) acc[q] = T(0);
                    if (i < s2)
                        for (int k = kb; k < ke; ++k) {
                            const T sv = Sn[i + (size_t)k * s2];
#pragma unroll
                            for (int q = 0; q < FA_RC; ++q)
                                if (q < rr) acc[q] = fma(sv, wn[(size_t)k * a.s + r0 + q], acc[q]);
                        }
#pragma unroll
                    for (int q = 0; q < FA_RC; ++q) part[(warp * TR + lane) * FA_RC + q] = acc[q];
                    __syncthreads();
                    for (int e = threadIdx.x; e < TR * rr; e += AP_THREADS) {
                        const int li = e % TR, q = e / TR;
                        const int ii = rt * TR + li;
                        if (ii < s2) a.y[((size_t)node * s2 + ii) * a.s + r0 + q] = warp_parts_sum(part, li, q);
                    }
                    __syncthreads();
                }
            }
        }
        if (c > 1) {
            const int64_t cnt = (int64_t)(1 << (c - 1)) * a.rp[c - 1] * a.s;
            T *wz = a.w[(c - 1) & 1];
            for (int64_t e = blockIdx.x * (int64_t)AP_THREADS + threadIdx.x; e < cnt; e += (int64_t)gridDim.x * AP_THREADS)
                wz[e] = T(0);
        }
        grid_sync(a.bar, a.status);
        // ---- A(c-1): x -= d(c) y_sib on every tile, then V_(c-1)^T x or the store
        for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
            const int4 tl = a.tiles[t];
            const int leaf = tl.x, nrows = tl.z;
            const int64_t row0 = tl.y;
            const int child = leaf >> (L - c);
            const int node = child >> 1;
            const int half = (child & 1) ? 0 : rp;   // the first child takes y2
            const S *Dc = a.D + a.coff[c] * a.ldn;
            const float *ds = a.dscale[c];
            const int64_t row = row0 + lane;
            const int kper = (rp + 7) / 8, kb = warp * kper, ke = min(rp, kb + kper);
            for (int r0 = 0; r0 < a.s; r0 += FA_RC) {
                const int rr = min(FA_RC, a.s - r0);
                if (rp > 0) {
                    for (int e = threadIdx.x; e < rp * rr; e += AP_THREADS) {
                        const int k = e / rr, q = e % rr;
                        const T yv = a.y[((size_t)node * s2 + half + k) * a.s + r0 + q];
                        ys[k * FA_RC + q] = ds ? yv * (T)ds[(size_t)child * rp + k] : yv;
                    }
                    __syncthreads();
                    T acc[FA_RC];
#pragma unroll
                    for (int q = 0; q < FA_RC; ++q) acc[q] = T(0);
                    if (lane < nrows)
                        for (int k = kb; k < ke; ++k) {
                            const T dv = to_t<T>(Dc[row + (int64_t)k * a.ldn]);
#pragma unroll
                            for (int q = 0; q < FA_RC; ++q)
                                if (q < rr) acc[q] = fma(dv, ys[k * FA_RC + q], acc[q]);
                        }
#pragma unroll
                    for (int q = 0; q < FA_RC; ++q) part[(warp * TR + lane) * FA_RC + q] = acc[q];
                    __syncthreads();
                    for (int e = threadIdx.x; e < TR * rr; e += AP_THREADS) {
                        const int li = e % TR, q = e / TR;
                        if (li < nrows) a.xt[row0 + li + (r0 + q) * a.ldn] -= warp_parts_sum(part, li, q);
                    }
                    __syncthreads();
                }
                if (c > 1) {
                    fa_vtx(a, c - 1, leaf >> (L - c + 1), row0, nrows, r0, rr, sv, xs);
                } else {
                    for (int e = threadIdx.x; e < TR * rr; e += AP_THREADS) {
                        const int li = e % TR, q = e / TR;
                        if (li < nrows)
                            a.X[row0 + li + (r0 + q) * a.ldx] = (double)a.xt[row0 + li + (r0 + q) * a.ldn];
                    }
                }
                __syncthreads();
            }
        }
        if (c > 1) grid_sync(a.bar, a.status);
    }
}

template <typename T, typename S>
hodlr_status solve_fused(const hodlr_t *h, int s, double *X, int64_t ldx, cudaStream_t st, const S *V, const S *Dm,
                         const float *const *vsc, const float *const *dsc) {
    hodlr_t *hm = const_cast<hodlr_t *>(h);
    HODLR_TRY(solve_prepare(h, s, st));
    const int L = h->L;
    int rpmax = 0;
    for (int c = 1; c <= L; ++c) rpmax = std::max(rpmax, h->lv[c].rp);
    const size_t xt_bytes = (size_t)h->ldn * s * sizeof(T);
    const size_t w_elems = (size_t)(1 << L) * std::max(rpmax, 1) * s;
    char *wp = reinterpret_cast<char *>(hm->work);
    FusedArgs<T, S> a{};
    a.Kinv = reinterpret_cast<const T *>(h->leafinv);
    a.bmax = h->bmax;
    a.L = L;
    a.s = s;
    a.n = h->n;
    a.ldn = h->ldn;
    a.ldx = ldx;
    a.V = V;
    a.D = Dm;
    for (int c = 1; c <= L; ++c) {
        a.rp[c] = h->lv[c].rp;
        a.coff[c] = h->lv[c].coff;
        a.Sinv[c - 1] = reinterpret_cast<const T *>(h->Sinv[c - 1]);
        a.vscale[c] = vsc ? vsc[c] : nullptr;
        a.dscale[c] = dsc ? dsc[c] : nullptr;
    }
    a.xt = reinterpret_cast<T *>(wp);
    a.w[0] = reinterpret_cast<T *>(wp + ((xt_bytes + 255) & ~size_t(255)));
    a.w[1] = a.w[0] + w_elems;
    a.y = a.w[1] + w_elems;
    a.tiles = h->d_tiles;
    a.ntiles = h->ntiles;
    a.bounds = h->d_bounds;
    a.X = X;
    a.bar = h->d_bar;
    a.status = h->ctx->d_status;
    if (L >= 1) HODLR_TRY_CUDA(cudaMemsetAsync(a.w[L & 1], 0, (size_t)(1 << L) * h->lv[L].rp * s * sizeof(T), st));
    a.rpmax = std::max(rpmax, 1);
    const size_t sm = ((size_t)(AP_THREADS / 32) * TR * FA_RC + 2 * (size_t)a.rpmax * FA_RC +
                       (size_t)a.rpmax * (TR + 1) + (size_t)TR * FA_RC) * sizeof(T);
    HODLR_TRY_CUDA(cudaFuncSetAttribute(apply_fused_kernel<T, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    int per_sm = 0;
    HODLR_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, apply_fused_kernel<T, S>, AP_THREADS, sm));
    if (per_sm <= 0) {
        set_error("fused apply: no resident CTA possible (%zu bytes of shared memory)", sm);
        return HODLR_RANGE;
    }
    const int grid = std::max(1, std::min(h->ctx->num_sms * std::min(per_sm, 2), std::max(h->ntiles, 1)));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(AP_THREADS);
    cfg.dynamicSmemBytes = sm;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    HODLR_TRY_CUDA(cudaLaunchKernelEx(&cfg, apply_fused_kernel<T, S>, a));
    return HODLR_OK;
}

}  // namespace

hodlr_status solve_impl(const hodlr_t *h, int s, double *X, int64_t ldx, cudaStream_t st) {
    if (h->prec == HODLR_FP64)
        return solve_fused<double, double>(h, s, X, ldx, st, reinterpret_cast<const double *>(h->V),
                                           reinterpret_cast<const double *>(h->D), nullptr, nullptr);
    if (h->store == HODLR_BF16)
        return solve_fused<float, __nv_bfloat16>(h, s, X, ldx, st, reinterpret_cast<const __nv_bfloat16 *>(h->Vq),
                                                 reinterpret_cast<const __nv_bfloat16 *>(h->Dq), nullptr, nullptr);
    if (h->store == HODLR_FP16)
        return solve_fused<float, __half>(h, s, X, ldx, st, reinterpret_cast<const __half *>(h->Vq),
                                          reinterpret_cast<const __half *>(h->Dq), h->vscale.data(),
                                          h->dscale.data());
    return solve_fused<float, float>(h, s, X, ldx, st, reinterpret_cast<const float *>(h->V),
                                     reinterpret_cast<const float *>(h->D), nullptr, nullptr);
}

}  // namespace hodlr

namespace hodlr {

// Allocate the apply's workspace for s right-hand sides ahead of time (the
// same sizing as solve_typed), so that later solves allocate nothing -- e.g.
// while they are being recorded into a graph.
hodlr_status solve_prepare(const hodlr_t *h, int s, cudaStream_t st) {
    const size_t es = elem_size(h->prec);
    int rpmax = 0;
    for (int c = 1; c <= h->L; ++c) rpmax = std::max(rpmax, h->lv[c].rp);
    const size_t xt_bytes = (size_t)h->ldn * s * es;
    const size_t w_elems = (size_t)(1 << h->L) * std::max(rpmax, 1) * s;
    const size_t need = xt_bytes + 3 * w_elems * es + 1024;   // x, w(c) double-buffered, y
    if (h->work_bytes < need) return ensure_work(const_cast<hodlr_t *>(h), need, st);
    return HODLR_OK;
}

}  // namespace hodlr
