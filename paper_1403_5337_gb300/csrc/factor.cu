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
#include <algorithm>
#include <climits>

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

template <typename T>
hodlr_status run_gj(hodlr_ctx *c, const std::vector<GJDesc<T>> &hd, cudaStream_t s, void *scratch) {
    if (hd.empty()) return HODLR_OK;
    int bmax = 0;
    for (auto &g : hd) bmax = std::max(bmax, g.b);
    GJDesc<T> *dd = reinterpret_cast<GJDesc<T> *>(scratch);
    HODLR_TRY_CUDA(cudaMemcpyAsync(dd, hd.data(), hd.size() * sizeof(GJDesc<T>),
                                   cudaMemcpyHostToDevice, s));
    size_t sm = 3 * (size_t)bmax * sizeof(T);
    HODLR_TRY_CUDA(cudaFuncSetAttribute(gj_inverse_kernel<T>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    gj_inverse_kernel<T><<<(int)hd.size(), GJ_THREADS, sm, s>>>(dd, c->d_status);
    HODLR_TRY_CUDA(cudaGetLastError());
    return HODLR_OK;
}

// Upload a vector of GEMM descriptors into `scratch` and launch.
template <typename T>
hodlr_status run_gemm(hodlr_ctx *c, const std::vector<GemmDesc<T>> &hd, int transA, T alpha,
                      cudaStream_t s, void *scratch) {
    if (hd.empty()) return HODLR_OK;
    int maxM = 0, maxN = 0, maxK = 0;
    for (auto &g : hd) {
        maxM = std::max(maxM, g.M);
        maxN = std::max(maxN, g.N);
        maxK = std::max(maxK, g.K);
    }
    if (maxM == 0 || maxN == 0 || maxK == 0) return HODLR_OK;
    GemmDesc<T> *dd = reinterpret_cast<GemmDesc<T> *>(scratch);
    HODLR_TRY_CUDA(cudaMemcpyAsync(dd, hd.data(), hd.size() * sizeof(GemmDesc<T>),
                                   cudaMemcpyHostToDevice, s));
    return gemm_batched<T>(c, dd, (int)hd.size(), maxM, maxN, maxK, transA, alpha, s);
}

// A descriptor upload area per step; several steps are enqueued before any sync,
// so each uses its own slice of the scratch.
struct Scratch {
    char *base = nullptr;
    size_t used = 0, cap = 0;
    void *take(size_t bytes) {
        size_t off = (used + 255) & ~size_t(255);
        if (off + bytes > cap) return nullptr;
        used = off + bytes;
        return base + off;
    }
};

template <typename T>
hodlr_status factor_typed(hodlr_t *h, cudaStream_t s) {
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
    need += (size_t)nleaf * 2 * bmax * bmax * sizeof(T);      // GJ work (leaves)
    need += (size_t)ldn * W * sizeof(T);                         // leaf stack output
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
    need += lvl_max;
    const size_t desc_bytes = (size_t)64 << 20;
    need += desc_bytes;
    HODLR_TRY(ensure_work(h, need, s));
    char *wp = reinterpret_cast<char *>(h->work);
    auto carve = [&](size_t bytes) {
        char *p = wp;
        wp += (bytes + 255) & ~size_t(255);
        return p;
    };
    T *gjw = reinterpret_cast<T *>(carve((size_t)nleaf * 2 * bmax * bmax * sizeof(T)));
    T *D2 = reinterpret_cast<T *>(carve((size_t)ldn * W * sizeof(T)));
    char *lvl = carve(lvl_max);
    Scratch sc;
    sc.base = carve(desc_bytes);
    sc.cap = desc_bytes;

    // ---- 1. leaf inverses
    T *Kinv = reinterpret_cast<T *>(h->leafinv);
    {
        std::vector<GJDesc<T>> gd(nleaf);
        for (int i = 0; i < nleaf; ++i) {
            int64_t r0, m;
            node_range(L, i, r0, m);
            gd[i] = GJDesc<T>{h->A + r0 * h->lda + r0, h->lda, nullptr, 0,
                              gjw + (size_t)i * 2 * bmax * bmax, Kinv + (size_t)i * bmax * bmax,
                              bmax, (int)m};
        }
        void *dd = sc.take(gd.size() * sizeof(GJDesc<T>));
        if (!dd) return HODLR_OUT_OF_MEMORY;
        HODLR_TRY(run_gj<T>(c, gd, s, dd));
    }
    // ---- 2. leaf stack: D2 = Kinv_leaf * D (all columns), then swap
    if (W > 0) {
        HODLR_TRY(zero<T>(D2, ldn * W, s));
        std::vector<GemmDesc<T>> gd(nleaf);
        for (int i = 0; i < nleaf; ++i) {
            int64_t r0, m;
            node_range(L, i, r0, m);
            gd[i] = GemmDesc<T>{Kinv + (size_t)i * bmax * bmax, D + r0, D2 + r0, bmax, ldn, ldn,
                                (int)m, (int)W, (int)m};
        }
        void *dd = sc.take(gd.size() * sizeof(GemmDesc<T>));
        if (!dd) return HODLR_OUT_OF_MEMORY;
        HODLR_TRY(run_gemm<T>(c, gd, 0, T(1), s, dd));
        HODLR_TRY_CUDA(cudaMemcpyAsync(D, D2, (size_t)ldn * W * sizeof(T), cudaMemcpyDeviceToDevice, s));
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
        HODLR_TRY(zero<T>(Y, (int64_t)nch * rp * Wc, s));
        {
            std::vector<GemmDesc<T>> gd(nch);
            for (int i = 0; i < nch; ++i) {
                int64_t r0, m;
                node_range(cch, i, r0, m);
                gd[i] = GemmDesc<T>{V + coffc * ldn + r0, D + r0, Y + (size_t)i * rp * Wc, ldn, ldn,
                                    rp, rp, (int)Wc, (int)m};
            }
            void *dd = sc.take(gd.size() * sizeof(GemmDesc<T>));
            if (!dd) return HODLR_OUT_OF_MEMORY;
            HODLR_TRY(run_gemm<T>(c, gd, 1, T(1), s, dd));
        }
        // (b) M = I - P Q per node
        {
            dim3 grid(std::max(1, std::min(64, (rp * rp + 255) / 256)), nn);
            set_identity_kernel<T><<<grid, 256, 0, s>>>(M, rp, rp, nn, (int64_t)rp * rp);
            HODLR_TRY_CUDA(cudaGetLastError());
            std::vector<GemmDesc<T>> gd(nn);
            for (int i = 0; i < nn; ++i) {
                const T *P = Y + (size_t)(2 * i) * rp * Wc + coffc * rp;
                const T *Q = Y + (size_t)(2 * i + 1) * rp * Wc + coffc * rp;
                gd[i] = GemmDesc<T>{P, Q, M + (size_t)i * rp * rp, rp, rp, rp, rp, rp, rp};
            }
            void *dd = sc.take(gd.size() * sizeof(GemmDesc<T>));
            if (!dd) return HODLR_OUT_OF_MEMORY;
            HODLR_TRY(run_gemm<T>(c, gd, 0, T(-1), s, dd));
        }
        // (c) M^-1 into the top-left block of S^-1
        {
            std::vector<GJDesc<T>> gd(nn);
            for (int i = 0; i < nn; ++i)
                gd[i] = GJDesc<T>{nullptr, 0, M + (size_t)i * rp * rp, rp, gw + (size_t)i * 2 * rp * rp,
                                  Sinv + (size_t)i * s2 * s2, s2, rp};
            void *dd = sc.take(gd.size() * sizeof(GJDesc<T>));
            if (!dd) return HODLR_OUT_OF_MEMORY;
            HODLR_TRY(run_gj<T>(c, gd, s, dd));
        }
        // (d) the other three blocks of S^-1
        {
            // TR = -M^-1 P ; BL = -Q M^-1 (zeroed first), BR = I - Q TR
            for (int i = 0; i < nn; ++i) {
                T *S = Sinv + (size_t)i * s2 * s2;
                // zero TR and BL, identity BR: handled by kernels below via cudaMemset2D
                HODLR_TRY_CUDA(cudaMemset2DAsync(S + rp * s2, s2 * sizeof(T), 0, rp * sizeof(T), rp, s));
                HODLR_TRY_CUDA(cudaMemset2DAsync(S + rp, s2 * sizeof(T), 0, rp * sizeof(T), rp, s));
            }
            {
                dim3 grid(std::max(1, std::min(64, (rp * rp + 255) / 256)), nn);
                set_identity_kernel<T><<<grid, 256, 0, s>>>(Sinv + rp + rp * s2, s2, rp, nn, s2 * s2);
                HODLR_TRY_CUDA(cudaGetLastError());
            }
            std::vector<GemmDesc<T>> g1(nn), g2(nn), g3(nn);
            for (int i = 0; i < nn; ++i) {
                T *S = Sinv + (size_t)i * s2 * s2;
                const T *P = Y + (size_t)(2 * i) * rp * Wc + coffc * rp;
                const T *Q = Y + (size_t)(2 * i + 1) * rp * Wc + coffc * rp;
                g1[i] = GemmDesc<T>{S, P, S + rp * s2, s2, rp, s2, rp, rp, rp};        // TR -= Minv P
                g2[i] = GemmDesc<T>{Q, S, S + rp, rp, s2, s2, rp, rp, rp};              // BL -= Q Minv
                g3[i] = GemmDesc<T>{Q, S + rp * s2, S + rp + rp * s2, rp, s2, s2, rp, rp, rp};  // BR -= Q TR
            }
            void *d1 = sc.take(nn * sizeof(GemmDesc<T>));
            void *d2 = sc.take(nn * sizeof(GemmDesc<T>));
            void *d3 = sc.take(nn * sizeof(GemmDesc<T>));
            if (!d1 || !d2 || !d3) return HODLR_OUT_OF_MEMORY;
            HODLR_TRY(run_gemm<T>(c, g1, 0, T(-1), s, d1));
            HODLR_TRY(run_gemm<T>(c, g2, 0, T(-1), s, d2));
            HODLR_TRY(run_gemm<T>(c, g3, 0, T(-1), s, d3));
        }
        // (e) update the ancestor columns (levels 1..l) for l >= 1
        if (l >= 1 && coffc > 0) {
            HODLR_TRY(zero<T>(Yv, (int64_t)nn * s2 * coffc, s));
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
            void *da = sc.take(nn * sizeof(GemmDesc<T>));
            void *db = sc.take(nn * sizeof(GemmDesc<T>));
            if (!da || !db) return HODLR_OUT_OF_MEMORY;
            HODLR_TRY(run_gemm<T>(c, gA, 0, T(1), s, da));
            HODLR_TRY(run_gemm<T>(c, gB, 0, T(1), s, db));
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
            void *du = sc.take(gu.size() * sizeof(GemmDesc<T>));
            if (!du) return HODLR_OUT_OF_MEMORY;
            HODLR_TRY(run_gemm<T>(c, gu, 0, T(-1), s, du));
        }
    }
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

hodlr_status factor_impl(hodlr_t *h, cudaStream_t s) {
    if (h->prec == HODLR_FP64) return factor_typed<double>(h, s);
    return factor_typed<float>(h, s);
}

}  // namespace hodlr
