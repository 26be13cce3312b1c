// Applying the factored HODLR inverse, X <- K~^-1 X (Sec. 4.3, Solve):
//   leaves:  x_leaf <- K_leaf^-1 x_leaf
//   for c = L .. 1 (children level), every parent node (alpha, beta):
//       w = [V_ba^T x_alpha ; V_ab^T x_beta]         (segmented reductions)
//       y = S^-1 w,  x_alpha -= d_alpha y2,  x_beta -= d_beta y1
// The last line is applied as x_alpha -= E_alpha w, x_beta -= E_beta w with
// E_alpha = d_alpha S^-1(rows rp..2rp-1, :) and E_beta = d_beta S^-1(rows
// 0..rp-1, :), formed once by the factorisation: the same product, associated
// differently, so no tile has to form y from the node's core.
// X is FP64 in and out; the arithmetic runs in the factor's precision T on a
// private copy of X.
//
// One persistent cooperative kernel over 32-row tiles of the leaves.  A tile's
// rows only ever change in that tile's CTA, so the only cross-tile dependency
// is the reduction w of each node: every tile adds its partial V^T x to w of
// its node and then bumps the node's arrival counter; a tile of that node
// waits for the counter to reach the node's tile count (a bounded spin: all
// CTAs are co-resident), updates its rows with E w and immediately adds its
// partial of the next level's w.  There is no grid-wide barrier: deep levels
// wait only for the few tiles of their own node.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <type_traits>
#include <vector>

#include "internal.cuh"

namespace hodlr {
namespace {

constexpr int AP_THREADS = 256;
constexpr int TR = 32;      // rows per tile
constexpr unsigned long long FA_SPIN_LIMIT = 1ull << 26;

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

template <typename T, typename S>
struct FusedArgs {
    const T *Kinv;
    int bmax, L, s, rpmax;
    int64_t n, ldn, ldx, ldxin;
    // per level c: V (ldn x rp(c)) and E (ldn x 2 rp(c)) at Vb + voff[c],
    // Eb + eoff[c]; one base and element offsets (a dynamically indexed array
    // of pointers in the kernel arguments measured ~15% slower here)
    const S *Vb, *Eb;
    int64_t voff[HODLR_MAX_LEVELS], eoff[HODLR_MAX_LEVELS];
    int rp[HODLR_MAX_LEVELS];
    const float *vscale[HODLR_MAX_LEVELS];
    const float *escale[HODLR_MAX_LEVELS];
    T *w[HODLR_MAX_LEVELS];                // w(c): [parent node][2 rp(c)][s], zeroed before the launch
    unsigned *cnt[HODLR_MAX_LEVELS];       // arrivals per parent node of level c, zeroed before the launch
    T *xt;
    const int4 *tiles;                     // (leaf, first row, rows, 0)
    const int *tile_first;                 // first tile of each leaf, 2^L + 1 entries
    int ntiles;
    // stage = 1: one tile per CTA, whose leaf-inverse rows and E, V rows of every
    // level are copied into shared memory at the start (byte offsets of each
    // level's block in the staging area; columns of 32 rows each)
    int stage, stage_at;
    int sofE[HODLR_MAX_LEVELS], sofV[HODLR_MAX_LEVELS];
    const int64_t *bounds;
    const double *Xin;
    double *X;
    float2 *Xs;        // optional: X also as FP32 (hi, lo) pairs, ld ldx (the product's split input)
    int *status;
    // bound of every wait (polls) and an addition to every wait's target (0;
    // a test sets 1, a tile that never arrives, to make the waits run out)
    unsigned long long spin_limit;
    unsigned target_extra;
};

// Lane-row / warp-split reduction helper: part[warp][lane][q] -> sum over warps.
template <typename T, int RC>
__device__ __forceinline__ T warp_parts_sum(const T *part, int lane_row, int q) {
    T v = T(0);
#pragma unroll
    for (int wv = 0; wv < AP_THREADS / 32; ++wv) v += part[(wv * TR + lane_row) * RC + q];
    return v;
}

// This tile's contribution to w(c) is complete: every thread orders its adds
// before the barrier, then one thread counts the tile.
__device__ __forceinline__ void arrive(unsigned *cnt) {
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) atomicAdd(cnt, 1u);
}

// Wait until all `target` tiles of the node have arrived (bounded: on timeout
// the status word gets ST_TIMEOUT and the kernel carries on).
__device__ __forceinline__ void wait_node(const unsigned *cnt, unsigned target, int *status,
                                          unsigned long long limit) {
    if (threadIdx.x == 0) {
        const volatile unsigned *vc = cnt;
        unsigned long long spins = 0;
        while (*vc < target) {
            if (++spins > limit) {
                atomicOr(status, ST_TIMEOUT);
                break;
            }
            __nanosleep(32);
        }
        __threadfence();
    }
    __syncthreads();
}

// Partial V_c^T x over one tile's rows into w(c): the tile's block of V (32
// rows x rp, coalesced column reads, four columns in flight per warp) and of x
// are staged in shared memory, then one thread per column forms its 32-term dot
// products (padded stride: no bank conflicts) and adds them to w with one
// atomic per (column, rhs).
template <typename T, typename S, int RC>
__device__ void fa_vtx(const FusedArgs<T, S> &a, int c, int child, int64_t row0, int nrows, int r0, int rr,
                       T *sv, T *xs, const unsigned char *stg) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int NW = AP_THREADS / 32;
    const int rp = a.rp[c];
    const S *Vc = a.Vb + a.voff[c];
    T *w = a.w[c];
    const float *vs = a.vscale[c];
    if (stg) {
        // the tile's V rows are staged (column-major, 32 rows per column)
        const S *Vs = reinterpret_cast<const S *>(stg + a.sofV[c]);
        for (int col = warp; col < rp; col += NW)
            sv[col * (TR + 1) + lane] = (lane < nrows) ? to_t<T>(Vs[col * TR + lane]) : T(0);
    } else {
        const int64_t row = row0 + lane;
        int col = warp;
        for (; col + 3 * NW < rp; col += 4 * NW) {
            T v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u)
                v[u] = (lane < nrows) ? to_t<T>(Vc[row + (int64_t)(col + u * NW) * a.ldn]) : T(0);
#pragma unroll
            for (int u = 0; u < 4; ++u) sv[(col + u * NW) * (TR + 1) + lane] = v[u];
        }
        for (; col < rp; col += NW)
            sv[col * (TR + 1) + lane] = (lane < nrows) ? to_t<T>(Vc[row + (int64_t)col * a.ldn]) : T(0);
    }
    {
        // all of a thread's loads in flight before its stores (a store through
        // a generic pointer between loads would serialise them)
        constexpr int U = (TR * RC + AP_THREADS - 1) / AP_THREADS;
        T v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int e = threadIdx.x + u * AP_THREADS, li = e % TR, q = e / TR;
            v[u] = (e < TR * RC && li < nrows && q < rr) ? a.xt[row0 + li + (r0 + q) * a.ldn] : T(0);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int e = threadIdx.x + u * AP_THREADS;
            if (e < TR * RC) xs[e] = v[u];
        }
    }
    __syncthreads();
    for (int cc = threadIdx.x; cc < rp; cc += AP_THREADS) {
        T acc[RC];
#pragma unroll
        for (int q = 0; q < RC; ++q) acc[q] = T(0);
#pragma unroll 8
        for (int li = 0; li < TR; ++li) {
            const T v = sv[cc * (TR + 1) + li];
#pragma unroll
            for (int q = 0; q < RC; ++q) acc[q] = fma(v, xs[q * TR + li], acc[q]);
        }
        const T sc = vs ? (T)vs[(size_t)child * rp + cc] : T(1);
#pragma unroll
        for (int q = 0; q < RC; ++q)
            if (q < rr) atomicAdd(&w[((size_t)child * rp + cc) * a.s + r0 + q], acc[q] * sc);
    }
    __syncthreads();
}

// acc[q] += sum_{k in [kb, ke)} M(k) y[k * RC + q] with M(k) = col[k * ldm] streamed
// from global memory eight columns at a time (loads in flight before the FMAs).
template <typename T, typename E, int RC>
__device__ __forceinline__ void stream_dot(const E *col, int64_t ldm, const T *y, int kb, int ke, T (&acc)[RC]) {
    int k = kb;
    for (; k + 8 <= ke; k += 8) {
        T m[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) m[u] = to_t<T>(col[(int64_t)(k + u) * ldm]);
#pragma unroll
        for (int u = 0; u < 8; ++u)
#pragma unroll
            for (int q = 0; q < RC; ++q) acc[q] = fma(m[u], y[(k + u) * RC + q], acc[q]);
    }
    for (; k < ke; ++k) {
        const T m = to_t<T>(col[(int64_t)k * ldm]);
#pragma unroll
        for (int q = 0; q < RC; ++q) acc[q] = fma(m, y[k * RC + q], acc[q]);
    }
}

__device__ __forceinline__ void prefetch_l2(const void *p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

// Pull everything this CTA's tiles will read into L2 up front (the leaf inverse
// rows, every level's E and V rows of the tiles), so that the dependent phases
// later hit L2 instead of HBM.
template <typename T, typename S>
__device__ void prefetch_tiles(const FusedArgs<T, S> &a) {
    constexpr int LINE = 128;
    constexpr int per_line = LINE / sizeof(S);
    for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
        const int4 tl = a.tiles[t];
        const int leaf = tl.x, nrows = tl.z;
        const int64_t row0 = tl.y;
        const int64_t l0 = a.bounds[leaf];
        const int b = (int)(a.bounds[leaf + 1] - l0);
        const T *K = a.Kinv + (size_t)leaf * a.bmax * a.bmax + (row0 - l0);
        for (int k = threadIdx.x; k < b; k += AP_THREADS) prefetch_l2(K + (size_t)k * a.bmax);
        const int lines = (nrows + per_line - 1) / per_line;   // every line starts inside the tile
        for (int c = 1; c <= a.L; ++c) {
            const int rp = a.rp[c];
            // columns 0 .. 2 rp - 1: E, 2 rp .. 3 rp - 1: V
            for (int e = threadIdx.x; e < 3 * rp * lines; e += AP_THREADS) {
                const int col = e / lines, r = e % lines;
                const S *base = col < 2 * rp ? a.Eb + a.eoff[c] + (int64_t)col * a.ldn
                                             : a.Vb + a.voff[c] + (int64_t)(col - 2 * rp) * a.ldn;
                prefetch_l2(base + row0 + (int64_t)r * per_line);
            }
        }
    }
}

__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}

// Copy `cols` columns of the tile's `nrows` (<= 32) rows, column j at src + j ld,
// to dst + 32 j: 16-byte asynchronous copies when the tile is full and every
// column starts on a 16-byte boundary, element copies otherwise.
template <typename X>
__device__ void stage_cols(X *dst, const X *src, int64_t ld, int cols, int nrows) {
    const bool vec = nrows == TR && (reinterpret_cast<uintptr_t>(src) & 15) == 0 && ((ld * sizeof(X)) & 15) == 0;
    if (vec) {
        constexpr int P = TR * (int)sizeof(X) / 16;   // 16-byte pieces per column
        for (int e = threadIdx.x; e < cols * P; e += AP_THREADS) {
            const int j = e / P, p = e % P;
            cp_async16(reinterpret_cast<char *>(dst + (size_t)j * TR) + 16 * p,
                       reinterpret_cast<const char *>(src + j * ld) + 16 * p);
        }
    } else {
        for (int e = threadIdx.x; e < cols * TR; e += AP_THREADS) {
            const int j = e / TR, r = e % TR;
            if (r < nrows) dst[(size_t)j * TR + r] = src[j * ld + r];
        }
    }
}

// X(o) = v in FP64, and (if requested) its FP32 (hi, lo) split for the product
// that follows: exact for an FP32 v (lo = 0), round-to-nearest parts for FP64.
template <typename T, typename S>
__device__ __forceinline__ void store_x(const FusedArgs<T, S> &a, int64_t o, T v) {
    a.X[o] = (double)v;
    if (a.Xs) {
        const float hi = (float)v;
        a.Xs[o] = make_float2(hi, (float)((double)v - (double)hi));
    }
}

// One tile's share of the leaf phase: x = K_leaf^-1 x on the tile's rows,
// then the leaf level's V^T x (partial sums added to w(L)).  Returns the leaf.
template <typename T, typename S, int RC>
__device__ __forceinline__ int leaf_tile(const FusedArgs<T, S> &a, int t, T *part, T *ws, T *sv, T *xs,
                                         const unsigned char *stg) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int L = a.L;
    const int4 tl = a.tiles[t];
    const int leaf = tl.x, nrows = tl.z;
    const int64_t row0 = tl.y;
    const int64_t l0 = a.bounds[leaf];
    const int b = (int)(a.bounds[leaf + 1] - l0);
    const T *K = a.Kinv + (size_t)leaf * a.bmax * a.bmax;
    const int il = (int)(row0 - l0) + lane;
    const int kper = (b + 7) / 8, kb = warp * kper, ke = min(b, kb + kper);
    for (int r0 = 0; r0 < a.s; r0 += RC) {
        const int rr = min(RC, a.s - r0);
        // the leaf's rows of X, converted once
        // eight loads in flight per thread before their stores
        for (int e0 = threadIdx.x; e0 < b * RC; e0 += 8 * AP_THREADS) {
            T v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int e = e0 + u * AP_THREADS, k = e / RC, q = e % RC;
                v[u] = (e < b * RC && q < rr) ? dev::from_double<T>(a.Xin[l0 + k + (int64_t)(r0 + q) * a.ldxin]) : T(0);
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int e = e0 + u * AP_THREADS;
                if (e < b * RC) ws[e] = v[u];
            }
        }
        __syncthreads();
        T acc[RC];
#pragma unroll
        for (int q = 0; q < RC; ++q) acc[q] = T(0);
        if (lane < nrows) {
            if (stg)
                stream_dot<T, T, RC>(reinterpret_cast<const T *>(stg) + lane, TR, ws, kb, ke, acc);
            else
                stream_dot<T, T, RC>(K + il, a.bmax, ws, kb, ke, acc);
        }
#pragma unroll
        for (int q = 0; q < RC; ++q) part[(warp * TR + lane) * RC + q] = acc[q];
        __syncthreads();
        for (int e = threadIdx.x; e < TR * rr; e += AP_THREADS) {
            const int li = e % TR, q = e / TR;
            if (li < nrows) {
                const T v = warp_parts_sum<T, RC>(part, li, q);
                a.xt[row0 + li + (r0 + q) * a.ldn] = v;
                if (L == 0) store_x(a, row0 + li + (r0 + q) * a.ldx, v);
            }
        }
        __syncthreads();
        if (L >= 1) fa_vtx<T, S, RC>(a, L, leaf, row0, nrows, r0, rr, sv, xs, stg);
    }
    return leaf;
}

// One tile's share of level c: (FUSED: once every tile of its node has added
// its part of w(c)) x -= E w(node) on the tile's rows, then the next level's
// V^T x, or (c = 1) the store of x.  Returns the leaf.
template <typename T, typename S, int RC, bool FUSED>
__device__ __forceinline__ int level_tile(const FusedArgs<T, S> &a, int c, int t, T *part, T *ws, T *sv, T *xs,
                                          const unsigned char *stg) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int L = a.L;
    const int rp = a.rp[c];
    const int s2 = 2 * rp;
    const int shift = L - c + 1;   // leaf -> parent node of level c
    const int4 tl = a.tiles[t];
    const int leaf = tl.x, nrows = tl.z;
    const int64_t row0 = tl.y;
    const int node = leaf >> shift;
    const int child = leaf >> (L - c);
    if constexpr (FUSED) {
        const unsigned target = (unsigned)(a.tile_first[(node + 1) << shift] - a.tile_first[node << shift]);
        wait_node(a.cnt[c] + node, target + a.target_extra, a.status, a.spin_limit);
    }
    const T *wn = a.w[c] + (size_t)node * s2 * a.s;
    const S *Ec = a.Eb + a.eoff[c];
    const float *es = a.escale[c];
    for (int r0 = 0; r0 < a.s; r0 += RC) {
        const int rr = min(RC, a.s - r0);
        if (rp > 0) {
            // w of the node (complete: read past L1), times E's FP16 column factors
            // (eight loads in flight per thread before their stores)
            for (int e0 = threadIdx.x; e0 < s2 * RC; e0 += 8 * AP_THREADS) {
                T v[8];
                float f[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int e = e0 + u * AP_THREADS, k = e / RC, q = e % RC;
                    v[u] = (e < s2 * RC && q < rr) ? __ldcg(wn + (size_t)k * a.s + r0 + q) : T(0);
                    f[u] = (es && e < s2 * RC) ? es[(size_t)child * s2 + k] : 1.0f;
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int e = e0 + u * AP_THREADS;
                    if (e < s2 * RC) ws[e] = v[u] * (T)f[u];
                }
            }
            __syncthreads();
            // x -= E w on the tile's rows: lanes over rows, warps split the 2 rp columns
            const int uper = (s2 + 7) / 8, ub = warp * uper, ue = min(s2, ub + uper);
            T acc[RC];
#pragma unroll
            for (int q = 0; q < RC; ++q) acc[q] = T(0);
            if (lane < nrows) {
                if (stg)
                    stream_dot<T, S, RC>(reinterpret_cast<const S *>(stg + a.sofE[c]) + lane, TR, ws, ub, ue,
                                         acc);
                else
                    stream_dot<T, S, RC>(Ec + row0 + lane, a.ldn, ws, ub, ue, acc);
            }
#pragma unroll
            for (int q = 0; q < RC; ++q) part[(warp * TR + lane) * RC + q] = acc[q];
            __syncthreads();
            for (int e = threadIdx.x; e < TR * rr; e += AP_THREADS) {
                const int li = e % TR, q = e / TR;
                if (li < nrows) {
                    const int64_t o = row0 + li + (int64_t)(r0 + q) * a.ldn;
                    const T v = a.xt[o] - warp_parts_sum<T, RC>(part, li, q);
                    a.xt[o] = v;
                    if (c == 1) store_x(a, row0 + li + (int64_t)(r0 + q) * a.ldx, v);
                }
            }
            __syncthreads();
        } else if (c == 1) {
            for (int e = threadIdx.x; e < TR * rr; e += AP_THREADS) {
                const int li = e % TR, q = e / TR;
                if (li < nrows)
                    store_x(a, row0 + li + (int64_t)(r0 + q) * a.ldx,
                            a.xt[row0 + li + (int64_t)(r0 + q) * a.ldn]);
            }
        }
        if (c > 1) fa_vtx<T, S, RC>(a, c - 1, leaf >> (L - c + 1), row0, nrows, r0, rr, sv, xs, stg);
    }
    return leaf;
}

template <typename T, typename S, int RC>
__global__ void __launch_bounds__(AP_THREADS) apply_fused_kernel(const FusedArgs<T, S> a) {
    extern __shared__ __align__(16) unsigned char smem[];
    T *part = reinterpret_cast<T *>(smem);                          // 8 warps x 32 rows x RC
    T *ws = part + (AP_THREADS / 32) * TR * RC;                     // w of the node: 2 rp x RC; the leaf's x
    T *sv = ws + (size_t)std::max(2 * a.rpmax, a.bmax) * RC;        // V tile: rp x (32 + 1)
    T *xs = sv + (size_t)a.rpmax * (TR + 1);                        // x tile: RC x 32
    const int L = a.L;
    // The tile's leaf-inverse rows, then E and V rows of every level, in shared
    // memory (one CTA per tile), or pulled into L2 for the phases below.
    const unsigned char *stg = nullptr;
    if (a.stage) {
        unsigned char *st = smem + a.stage_at;
        if ((int)blockIdx.x < a.ntiles) {
            const int4 tl = a.tiles[blockIdx.x];
            const int leaf = tl.x, nrows = tl.z;
            const int64_t row0 = tl.y;
            const int64_t l0 = a.bounds[leaf];
            const int b = (int)(a.bounds[leaf + 1] - l0);
            stage_cols<T>(reinterpret_cast<T *>(st), a.Kinv + (size_t)leaf * a.bmax * a.bmax + (row0 - l0), a.bmax, b,
                          nrows);
            for (int c = 1; c <= L; ++c) {
                stage_cols<S>(reinterpret_cast<S *>(st + a.sofE[c]), a.Eb + a.eoff[c] + row0, a.ldn, 2 * a.rp[c],
                              nrows);
                stage_cols<S>(reinterpret_cast<S *>(st + a.sofV[c]), a.Vb + a.voff[c] + row0, a.ldn, a.rp[c], nrows);
            }
            asm volatile("cp.async.commit_group;" ::: "memory");
            asm volatile("cp.async.wait_group 0;" ::: "memory");
        }
        __syncthreads();
        stg = st;
    } else {
        prefetch_tiles(a);
    }
    // ---- leaves: x = K_leaf^-1 x on the tile's rows, then the leaf level's V^T x
    for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
        const int leaf = leaf_tile<T, S, RC>(a, t, part, ws, sv, xs, stg);
        if (L >= 1) arrive(a.cnt[L] + (leaf >> 1));
    }
    // ---- levels c = L .. 1: x -= E w(node) on the tile's rows (E = d S^-1(half)
    // formed by the factorisation), then the next level's V^T x (or the store)
    for (int c = L; c >= 1; --c) {
        for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
            const int leaf = level_tile<T, S, RC, true>(a, c, t, part, ws, sv, xs, stg);
            if (c > 1) arrive(a.cnt[c - 1] + (leaf >> (L - c + 2)));
        }
    }
}

// The apply phase by phase, one launch per phase (the leaves with level L's
// V^T x, then each level c = L .. 1) and one CTA per tile: the kernel boundary
// orders the phases, so no tile waits for another inside a launch.  Taken when
// the tree has several tiles per resident CTA, where the single cooperative
// launch would walk each CTA's tiles in series with a wait per node and level.
template <typename T, typename S, int RC>
__global__ void __launch_bounds__(AP_THREADS, 2) apply_phase_kernel(const FusedArgs<T, S> a, int c) {
    extern __shared__ __align__(16) unsigned char smem[];
    T *part = reinterpret_cast<T *>(smem);                          // 8 warps x 32 rows x RC
    T *ws = part + (AP_THREADS / 32) * TR * RC;                     // w of the node: 2 rp x RC; the leaf's x
    T *sv = ws + (size_t)std::max(2 * a.rpmax, a.bmax) * RC;        // V tile: rp x (32 + 1)
    T *xs = sv + (size_t)a.rpmax * (TR + 1);                        // x tile: RC x 32
    if (c > a.L)
        leaf_tile<T, S, RC>(a, blockIdx.x, part, ws, sv, xs, nullptr);
    else
        level_tile<T, S, RC, false>(a, c, blockIdx.x, part, ws, sv, xs, nullptr);
}

// The per-phase apply for FP32 arithmetic, one CTA per 32-row tile and up to
// 32 right-hand sides per pass.  Everything a tile reads in a phase is requested
// before any of it is used -- E's (or the leaf inverse's) and the next level's V
// rows by asynchronous copies into shared memory, the node's w and the tile's x
// by batched loads -- so that a phase costs a few memory round trips per tile.
// Then
//   x -= E w          thread = 2 rows x 8 right-hand sides over a quarter of
//                     the k range (per k: one E pair, two broadcast w vectors,
//                     16 FMAs); the four quarter sums added in shared memory,
//   w(next) += V^T x  V transposed in shared memory, lane = 2 columns of V,
//                     warp = 4 right-hand sides, x broadcast (per row: one V
//                     pair, one x vector, 8 FMAs); atomics into w,
// or, at the top level, the store of x.  The leaf phase forms x = K_leaf^-1 x
// from the tile's rows of the leaf inverse the same way.

struct TileSmem {
    size_t xs, vs, ws, es, total;
};

// w (or the leaf's x) in shared memory: k rows of 32 right-hand sides, the
// eight 4-wide groups of row k permuted by k mod 8, so that a warp storing one
// right-hand side of 32 consecutive rows spreads over eight bank groups, and a
// warp storing 32 right-hand sides of one row over all 32 banks.
__device__ __forceinline__ int ws_at(int k, int q) { return k * 32 + ((((q >> 2) ^ k) & 7) << 2) + (q & 3); }
__device__ __forceinline__ int ws_group(int k, int g) { return k * 32 + (((g ^ k) & 7) << 2); }

// Row pitch (elements) of V transposed in shared memory: even, and an odd
// number of 32-bit words for 16-bit V (a column's 32 rows over 32 banks).
__host__ __device__ __forceinline__ int vt_pitch(int rv) { return (rv + 63) / 64 * 64 + 2; }

constexpr int TP_KPARTS = 4;                                 // k-range quarters of x -= E w
constexpr int TP_PART = 32 * 33;                             // one quarter's sums: x(row r, rhs q) at q 33 + r

template <typename S>
__device__ __forceinline__ float2 ld2f(const S *p) {
    if constexpr (std::is_same<S, __half>::value)
        return __half22float2(*reinterpret_cast<const __half2 *>(p));
    else if constexpr (std::is_same<S, __nv_bfloat16>::value)
        return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(p));
    else
        return *reinterpret_cast<const float2 *>(p);
}

__device__ __forceinline__ void fma8(float *acc, float e, const float4 &y0, const float4 &y1) {
    acc[0] = fmaf(e, y0.x, acc[0]);
    acc[1] = fmaf(e, y0.y, acc[1]);
    acc[2] = fmaf(e, y0.z, acc[2]);
    acc[3] = fmaf(e, y0.w, acc[3]);
    acc[4] = fmaf(e, y1.x, acc[4]);
    acc[5] = fmaf(e, y1.y, acc[5]);
    acc[6] = fmaf(e, y1.z, acc[6]);
    acc[7] = fmaf(e, y1.w, acc[7]);
}

// Shared-memory layout of one phase of apply_tile_kernel (offsets in bytes):
// x (32 rows x 32 rhs, row pitch 36), rv columns of the next level's V as
// staged (32 rows each), the w region (kw rows of w -- 2 r_c of a level, the
// leaf size b of the leaf phase -- later the quarter sums, then V transposed),
// and E's (or the leaf inverse's) rows.
template <typename S>
TileSmem tile_smem(int kw, int rv, bool leafp) {
    auto al = [](size_t b) { return (b + 15) & ~size_t(15); };
    TileSmem m{};
    const size_t wbytes = std::max({(size_t)kw * 32 * sizeof(float), (size_t)TP_KPARTS * TP_PART * sizeof(float),
                                    rv > 0 ? (size_t)32 * vt_pitch(rv) * sizeof(S) : size_t(0)});
    m.xs = 0;
    m.vs = m.xs + al(32 * 36 * sizeof(float));
    m.ws = m.vs + al((size_t)32 * rv * sizeof(S));
    m.es = m.ws + al(wbytes);
    m.total = m.es + al((size_t)kw * 32 * (leafp ? sizeof(float) : sizeof(S)));
    return m;
}

template <typename S>
__device__ __forceinline__ void tile_phase(const FusedArgs<float, S> &a, int c, const TileSmem &sm, int tile,
                                           unsigned char *smem) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, q0 = 4 * warp;
    const int L = a.L;
    const int4 tl = a.tiles[tile];
    const int leaf = tl.x, nrows = tl.z;
    const int64_t row0 = tl.y;
    const bool leafp = c > L;
    const int cv = leafp ? L : c - 1;              // the level whose V^T x this phase adds (0: none)
    const int rpv = cv >= 1 ? a.rp[cv] : 0;
    const int childv = cv >= 1 ? leaf >> (L - cv) : 0;
    float *xT = reinterpret_cast<float *>(smem + sm.xs);    // x(row r, rhs q) at r * 36 + q
    S *Vs = reinterpret_cast<S *>(smem + sm.vs);            // V(row r, column j) at j * 32 + r, as staged
    float *ws = reinterpret_cast<float *>(smem + sm.ws);
    unsigned char *es_raw = smem + sm.es;
    // ---- E's (or the leaf inverse's) rows of the tile: asynchronous copies
    int64_t l0 = 0;
    int b = 0, rp = 0, s2 = 0, node = 0, child = 0;
    if (leafp) {
        l0 = a.bounds[leaf];
        b = (int)(a.bounds[leaf + 1] - l0);
        stage_cols<float>(reinterpret_cast<float *>(es_raw),
                          a.Kinv + (size_t)leaf * a.bmax * a.bmax + (row0 - l0), a.bmax, b, nrows);
    } else {
        rp = a.rp[c];
        s2 = 2 * rp;
        node = leaf >> (L - c + 1);
        child = leaf >> (L - c);
        if (rp > 0) stage_cols<S>(reinterpret_cast<S *>(es_raw), a.Eb + a.eoff[c] + row0, a.ldn, s2, nrows);
    }
    // ---- the next level's V rows of the tile
    if (rpv > 0) stage_cols<S>(Vs, a.Vb + a.voff[cv] + row0, a.ldn, rpv, nrows);
    asm volatile("cp.async.commit_group;" ::: "memory");
    const float *vsc = cv >= 1 ? a.vscale[cv] : nullptr;
    // x -= E w: this thread's rows 2 rh, 2 rh + 1, right-hand sides 8 qb .. 8 qb + 7, k quarter kp
    const int kp = warp >> 1, qb = ((warp & 1) << 1) | (lane >> 4), rh = lane & 15;
    const int K = leafp ? b : s2;
    const int kc = (K + TP_KPARTS - 1) / TP_KPARTS;
    const int ka = min(K, kp * kc), kb = min(K, ka + kc);
    for (int r0 = 0; r0 < a.s; r0 += 32) {
        const int rr = min(32, a.s - r0);
        float xo[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        if (leafp) {
            // the leaf's rows of X (FP64 -> FP32): a warp reads 32 consecutive
            // rows of one right-hand side, sixteen loads in flight per thread
            for (int k0 = 0; k0 < b; k0 += 256) {
#pragma unroll 1
                for (int qq = warp; qq < 32; qq += 16) {
                    float v[16];
#pragma unroll
                    for (int u = 0; u < 16; ++u) {
                        const int q = qq + 8 * (u >> 3), k = k0 + lane + 32 * (u & 7);
                        v[u] = (k < b && q < rr) ? (float)a.Xin[l0 + k + (int64_t)(r0 + q) * a.ldxin] : 0.0f;
                    }
#pragma unroll
                    for (int u = 0; u < 16; ++u) {
                        const int q = qq + 8 * (u >> 3), k = k0 + lane + 32 * (u & 7);
                        if (k < b) ws[ws_at(k, q)] = v[u];
                    }
                }
            }
        } else {
            // the tile's x and the node's w (times E's column factors), eight loads in flight
#pragma unroll
            for (int j = 0; j < 4; ++j)
                xo[j] = (lane < nrows && q0 + j < rr) ? a.xt[row0 + lane + (int64_t)(r0 + q0 + j) * a.ldn] : 0.0f;
            const float *wn = a.w[c] + (size_t)node * s2 * a.s;
            const float *esc = a.escale[c];
            for (int e0 = threadIdx.x; e0 < s2 * 32; e0 += 8 * AP_THREADS) {
                float v[8], f[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int e = e0 + u * AP_THREADS, k = e >> 5, q = e & 31;
                    v[u] = (e < s2 * 32 && q < rr) ? __ldcg(wn + (size_t)k * a.s + r0 + q) : 0.0f;
                    f[u] = (esc && e < s2 * 32) ? esc[(size_t)child * s2 + k] : 1.0f;
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int e = e0 + u * AP_THREADS;
                    if (e < s2 * 32) ws[ws_at(e >> 5, e & 31)] = v[u] * f[u];
                }
            }
        }
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        __syncthreads();
        float acc[2][8];
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[i][j] = 0.0f;
        if (leafp) {
            const float *Ks = reinterpret_cast<const float *>(es_raw);
#pragma unroll 4
            for (int k = ka; k < kb; ++k) {
                const float2 e = *reinterpret_cast<const float2 *>(Ks + k * 32 + 2 * rh);
                const float4 y0 = *reinterpret_cast<const float4 *>(ws + ws_group(k, 2 * qb));
                const float4 y1 = *reinterpret_cast<const float4 *>(ws + ws_group(k, 2 * qb + 1));
                fma8(acc[0], e.x, y0, y1);
                fma8(acc[1], e.y, y0, y1);
            }
        } else {
            const S *Es = reinterpret_cast<const S *>(es_raw);
#pragma unroll 4
            for (int k = ka; k < kb; ++k) {
                const float2 e = ld2f<S>(Es + k * 32 + 2 * rh);
                const float4 y0 = *reinterpret_cast<const float4 *>(ws + ws_group(k, 2 * qb));
                const float4 y1 = *reinterpret_cast<const float4 *>(ws + ws_group(k, 2 * qb + 1));
                fma8(acc[0], e.x, y0, y1);
                fma8(acc[1], e.y, y0, y1);
            }
        }
        __syncthreads();   // every warp is done with w: its region takes the quarter sums
        float *part = ws + kp * TP_PART;
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) part[(8 * qb + j) * 33 + 2 * rh + i] = acc[i][j];
        __syncthreads();
        float x[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int o = (q0 + j) * 33 + lane;
            const float sum = ((ws[o] + ws[TP_PART + o]) + ws[2 * TP_PART + o]) + ws[3 * TP_PART + o];
            x[j] = leafp ? sum : xo[j] - sum;
        }
        if (lane >= nrows) x[0] = x[1] = x[2] = x[3] = 0.0f;   // rows past a ragged tile
        // ---- x: kept for the later phases, or (top level / single leaf) stored
        if (lane < nrows) {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (q0 + j < rr) {
                    if (cv == 0)
                        store_x(a, row0 + lane + (int64_t)(r0 + q0 + j) * a.ldx, x[j]);
                    else
                        a.xt[row0 + lane + (int64_t)(r0 + q0 + j) * a.ldn] = x[j];
                }
            }
        }
        if (cv >= 1) {
            // ---- w(cv) += V^T x over the tile's rows
            __syncthreads();   // the quarter sums are read: the w region takes V transposed
            *reinterpret_cast<float4 *>(xT + lane * 36 + q0) = make_float4(x[0], x[1], x[2], x[3]);
            const int vp = vt_pitch(rpv);
            S *Vt = reinterpret_cast<S *>(ws);   // V(row r, column j) at r * vp + j
            for (int e = threadIdx.x; e < rpv * 32; e += AP_THREADS) {
                const int col = e >> 5, r = e & 31;
                if (r < nrows) Vt[r * vp + col] = Vs[col * 32 + r];
            }
            __syncthreads();
            for (int j0 = 2 * lane; j0 < rpv; j0 += 64) {
                float a0[4] = {0.0f, 0.0f, 0.0f, 0.0f}, a1[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll 4
                for (int r = 0; r < nrows; ++r) {
                    const float2 v = ld2f<S>(Vt + r * vp + j0);
                    const float4 y = *reinterpret_cast<const float4 *>(xT + r * 36 + q0);
                    a0[0] = fmaf(v.x, y.x, a0[0]);
                    a0[1] = fmaf(v.x, y.y, a0[1]);
                    a0[2] = fmaf(v.x, y.z, a0[2]);
                    a0[3] = fmaf(v.x, y.w, a0[3]);
                    a1[0] = fmaf(v.y, y.x, a1[0]);
                    a1[1] = fmaf(v.y, y.y, a1[1]);
                    a1[2] = fmaf(v.y, y.z, a1[2]);
                    a1[3] = fmaf(v.y, y.w, a1[3]);
                }
                const bool two = j0 + 1 < rpv;
                const float sc0 = vsc ? vsc[(size_t)childv * rpv + j0] : 1.0f;
                const float sc1 = (vsc && two) ? vsc[(size_t)childv * rpv + j0 + 1] : 1.0f;
                float *wd = a.w[cv] + ((size_t)childv * rpv + j0) * a.s + r0 + q0;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    if (q0 + j < rr) {
                        atomicAdd(wd + j, a0[j] * sc0);
                        if (two) atomicAdd(wd + a.s + j, a1[j] * sc1);
                    }
                }
            }
        }
        __syncthreads();   // the shared buffers are refilled by the next pass (or tile)
    }
}

// One phase over all tiles: CTAs resident together walk the tiles, so that no
// partly filled last wave is left.
template <typename S>
__global__ void __launch_bounds__(AP_THREADS, 3) apply_tile_kernel(const FusedArgs<float, S> a, int c, TileSmem sm) {
    extern __shared__ __align__(16) unsigned char smem[];
    for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x) tile_phase<S>(a, c, sm, t, smem);
}

template <typename T, typename S, int RC>
hodlr_status launch_fused(const hodlr_t *h, const FusedArgs<T, S> &a, cudaStream_t st);

template <typename T, typename S>
hodlr_status solve_fused(const hodlr_t *h, int s, double *X, int64_t ldx, cudaStream_t st,
                         const std::vector<void *> &V, const std::vector<void *> &E, const float *const *vsc,
                         const float *const *esc, float2 *Xs) {
    hodlr_t *hm = const_cast<hodlr_t *>(h);
    HODLR_TRY(solve_prepare(h, s, st));
    const int L = h->L;
    int rpmax = 0;
    for (int c = 1; c <= L; ++c) rpmax = std::max(rpmax, h->lv[c].rp);
    FusedArgs<T, S> a{};
    a.Kinv = reinterpret_cast<const T *>(h->leafinv);
    a.bmax = h->bmax;
    a.L = L;
    a.s = s;
    a.n = h->n;
    a.ldn = h->ldn;
    a.ldx = ldx;
    a.spin_limit = h->ctx->wait_limit ? h->ctx->wait_limit : FA_SPIN_LIMIT;
    a.target_extra = h->ctx->wait_extra;
    // workspace: x (T), then the zeroed region: w(c) for c = 1..L, the counters
    char *wp = reinterpret_cast<char *>(hm->work);
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    a.xt = reinterpret_cast<T *>(wp);
    char *z0 = wp + al((size_t)h->ldn * s * sizeof(T));
    char *zp = z0;
    a.Vb = L >= 1 ? reinterpret_cast<const S *>(V[1]) : nullptr;
    a.Eb = L >= 1 ? reinterpret_cast<const S *>(E[1]) : nullptr;
    for (int c = 1; c <= L; ++c) {
        a.rp[c] = h->lv[c].rp;
        a.voff[c] = reinterpret_cast<const S *>(V[c]) - a.Vb;
        a.eoff[c] = reinterpret_cast<const S *>(E[c]) - a.Eb;
        a.vscale[c] = vsc ? vsc[c] : nullptr;
        a.escale[c] = esc ? esc[c] : nullptr;
        a.w[c] = reinterpret_cast<T *>(zp);
        zp += al((size_t)(1 << c) * h->lv[c].rp * s * sizeof(T));
    }
    for (int c = 1; c <= L; ++c) {
        a.cnt[c] = reinterpret_cast<unsigned *>(zp);
        zp += al((size_t)(1 << (c - 1)) * sizeof(unsigned));
    }
    a.tiles = h->d_tiles;
    a.tile_first = h->d_tile_first;
    a.ntiles = h->ntiles;
    a.bounds = h->d_bounds;
    a.X = X;
    a.status = h->ctx->d_status;
    a.rpmax = std::max(rpmax, 1);
    // X is read by the leaf solves and written by the last level; the last level
    // of a tree with L >= 1 waits for every tile, so it is safe in place.  A
    // single leaf (L = 0) reads its input from a copy.
    a.Xin = X;
    a.ldxin = ldx;
    a.Xs = Xs;
    if (L == 0) {
        double *cp = reinterpret_cast<double *>(zp);
        HODLR_TRY_CUDA(cudaMemcpy2DAsync(cp, h->ldn * sizeof(double), X, ldx * sizeof(double), h->n * sizeof(double),
                                         s, cudaMemcpyDeviceToDevice, st));
        a.Xin = cp;
        a.ldxin = h->ldn;
    }
    if (zp > z0) HODLR_TRY_CUDA(cudaMemsetAsync(z0, 0, (size_t)(zp - z0), st));
    if (s <= 1) return launch_fused<T, S, 1>(h, a, st);
    if (s <= 2) return launch_fused<T, S, 2>(h, a, st);
    if (s <= 4) return launch_fused<T, S, 4>(h, a, st);
    if (s <= 8) return launch_fused<T, S, 8>(h, a, st);
    // many right-hand sides: one pass over the factors' rows for 16 or 32 of them
    if constexpr (sizeof(T) == 4) {
        if (s > 16) return launch_fused<T, S, 32>(h, a, st);
    }
    return launch_fused<T, S, 16>(h, a, st);
}

template <typename T, typename S, int RC>
hodlr_status launch_fused(const hodlr_t *h, const FusedArgs<T, S> &a0, cudaStream_t st) {
    FusedArgs<T, S> a = a0;
    const size_t sm0 = (((size_t)(AP_THREADS / 32) * TR * RC + (size_t)std::max(2 * a.rpmax, a.bmax) * RC +
                         (size_t)a.rpmax * (TR + 1) + (size_t)TR * RC) *
                            sizeof(T) +
                        15) & ~size_t(15);
    // staging area of one tile: the leaf inverse's rows, then per level E (2 rp
    // columns) and V (rp columns), 32 rows per column
    auto al16 = [](size_t b) { return (b + 15) & ~size_t(15); };
    size_t sbytes = al16((size_t)a.bmax * TR * sizeof(T));
    for (int c = 1; c <= a.L; ++c) {
        a.sofE[c] = (int)sbytes;
        sbytes += al16((size_t)2 * a.rp[c] * TR * sizeof(S));
        a.sofV[c] = (int)sbytes;
        sbytes += al16((size_t)a.rp[c] * TR * sizeof(S));
    }
    int optin = 0;
    HODLR_TRY_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->ctx->device));
    size_t sm = sm0;
    a.stage = 0;
    a.stage_at = (int)sm0;
    if (h->ntiles <= h->ctx->num_sms && sm0 + sbytes <= (size_t)optin) {
        HODLR_TRY_CUDA(cudaFuncSetAttribute(apply_fused_kernel<T, S, RC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)(sm0 + sbytes)));
        int per = 0;
        HODLR_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, apply_fused_kernel<T, S, RC>, AP_THREADS,
                                                                     sm0 + sbytes));
        if (per >= 1) {
            a.stage = 1;
            sm = sm0 + sbytes;
        }
    }
    HODLR_TRY_CUDA(cudaFuncSetAttribute(apply_fused_kernel<T, S, RC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)sm));
    int per_sm = 0;
    HODLR_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, apply_fused_kernel<T, S, RC>, AP_THREADS, sm));
    if (per_sm <= 0) {
        set_error("fused apply: no resident CTA possible (%zu bytes of shared memory)", sm);
        return HODLR_RANGE;
    }
    // staging needs one CTA per tile (ntiles <= SMs <= resident CTAs)
    const int grid = a.stage ? std::max(h->ntiles, 1)
                             : std::max(1, std::min(h->ctx->num_sms * std::min(per_sm, 2), std::max(h->ntiles, 1)));
    const int path = h->ctx->apply_path ? h->ctx->apply_path : (!a.stage && h->ntiles >= 2 * grid ? 2 : 1);
    if (path == 2 && a.L >= 1) {
        // several tiles per CTA: one launch per phase, one CTA per tile
        if constexpr (std::is_same<T, float>::value) {
            // per phase: its own shared-memory layout (at most three CTAs' worth
            // per SM on the largest)
            std::vector<TileSmem> tsm(a.L + 2);
            size_t most = 0;
            for (int c = a.L + 1; c >= 1; --c) {
                const bool leafp = c > a.L;
                const int cv = leafp ? a.L : c - 1;
                tsm[c] = tile_smem<S>(leafp ? a.bmax : 2 * a.rp[c], cv >= 1 ? a.rp[cv] : 0, leafp);
                most = std::max(most, tsm[c].total);
            }
            if (most <= (size_t)optin / 2) {   // at least two CTAs per SM on every phase
                HODLR_TRY_CUDA(cudaFuncSetAttribute(apply_tile_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                    (int)most));
                ProfScope ps("apply_phase_kernel", st);
                for (int c = a.L + 1; c >= 1; --c) {
                    int per = 0;
                    HODLR_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, apply_tile_kernel<S>, AP_THREADS,
                                                                                 tsm[c].total));
                    const int g = std::max(1, std::min(h->ntiles, std::max(per, 1) * h->ctx->num_sms));
                    apply_tile_kernel<S><<<g, AP_THREADS, tsm[c].total, st>>>(a, c, tsm[c]);
                    note_launch();
                    HODLR_TRY_CUDA(cudaGetLastError());
                }
                return HODLR_OK;
            }
        }
        HODLR_TRY_CUDA(cudaFuncSetAttribute(apply_phase_kernel<T, S, RC>,
                                            cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm0));
        ProfScope ps("apply_phase_kernel", st);
        for (int c = a.L + 1; c >= 1; --c) {
            apply_phase_kernel<T, S, RC><<<h->ntiles, AP_THREADS, sm0, st>>>(a, c);
            note_launch();
            HODLR_TRY_CUDA(cudaGetLastError());
        }
        return HODLR_OK;
    }
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
    {
        ProfScope ps("apply_fused_kernel", st);
        HODLR_TRY_CUDA(cudaLaunchKernelEx(&cfg, apply_fused_kernel<T, S, RC>, a));
    }
    note_launch();
    return HODLR_OK;
}

}  // namespace

hodlr_status solve_impl(const hodlr_t *h, int s, double *X, int64_t ldx, cudaStream_t st, float2 *Xs) {
    if (h->diag) return diag_solve(h, s, X, ldx, st, Xs);
    if (h->prec == HODLR_FP64) return solve_fused<double, double>(h, s, X, ldx, st, h->Vl, h->El, nullptr, nullptr, Xs);
    if (h->store == HODLR_BF16)
        return solve_fused<float, __nv_bfloat16>(h, s, X, ldx, st, h->Vql, h->Eql, nullptr, nullptr, Xs);
    if (h->store == HODLR_FP16)
        return solve_fused<float, __half>(h, s, X, ldx, st, h->Vql, h->Eql, h->vscale.data(), h->escale.data(), Xs);
    return solve_fused<float, float>(h, s, X, ldx, st, h->Vl, h->El, nullptr, nullptr, Xs);
}

// Allocate the apply's workspace for s right-hand sides ahead of time (the
// sizing of solve_fused), so that later solves allocate nothing -- e.g. while
// they are being recorded into a graph.
hodlr_status solve_prepare(const hodlr_t *h, int s, cudaStream_t st) {
    const size_t es = elem_size(h->prec);
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    size_t need = al((size_t)h->ldn * s * es);
    for (int c = 1; c <= h->L; ++c) need += al((size_t)(1 << c) * h->lv[c].rp * s * es);
    for (int c = 1; c <= h->L; ++c) need += al((size_t)(1 << (c - 1)) * sizeof(unsigned));
    if (h->L == 0) need += al((size_t)h->ldn * s * sizeof(double));
    need += 1024;
    if (h->work_bytes < need) return ensure_work(const_cast<hodlr_t *>(h), need, st);
    return HODLR_OK;
}

}  // namespace hodlr
