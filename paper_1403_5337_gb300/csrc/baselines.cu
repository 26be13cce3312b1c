// The paper's comparison points on the same GPU (Sec. 7): GMRES with the
// diagonal (Jacobi) preconditioner, the "Diag" curve of Fig. 8, and the
// conventional dense LU solve of the front, the "LU" column of Table 3.
//
// The diagonal preconditioner is a hodlr_t without levels whose apply is
// x_i <- x_i / A(i,i); gmres_solve, hodlr_solve and hodlr_precond_error take
// it like any HODLR preconditioner.
#include <algorithm>
#include <climits>
#include <cmath>
#include <vector>

#include "internal.cuh"

namespace hodlr {
namespace {

// dinv(i) = 1 / A(i, i); a zero diagonal entry is reported as singular, a
// non-finite one as non-finite input
__global__ void diag_inverse_kernel(const double *__restrict__ A, int64_t n, int64_t lda, double *__restrict__ dinv,
                                    int *status) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double a = A[i * lda + i];
        if (!isfinite(a))
            atomicOr(status, ST_NONFINITE);
        else if (a == 0.0)
            atomicOr(status, ST_SINGULAR);
        dinv[i] = (a != 0.0 && isfinite(a)) ? 1.0 / a : 0.0;
    }
}

// X(:, r) <- dinv .* X(:, r); Xs (optional) the result as FP32 (hi, lo) pairs
// for the product, in the layout of the HODLR apply (ld ldx)
__global__ void diag_apply_kernel(const double *__restrict__ dinv, int64_t n, int s, double *__restrict__ X,
                                  int64_t ldx, float2 *__restrict__ Xs) {
    const int r = blockIdx.y;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t o = i + (int64_t)r * ldx;
        const double v = X[o] * dinv[i];
        X[o] = v;
        if (Xs) {
            const float hi = (float)v;
            Xs[o] = make_float2(hi, (float)(v - (double)hi));
        }
    }
}

// ------------------------------------------------------------------ dense LU
// Right-looking blocked LU with row partial pivoting of the column-major copy
// W (n x n, ld n), panels of LU_NB columns: the panel is factored by one CTA
// (pivot = the largest |W(i, j)| over i >= j, lowest row on ties; swap; scale;
// rank-1 update of the panel's remaining columns), the panel's swaps are
// applied to the other columns, U12 = L11^-1 A12 by forward substitution, and
// the trailing block is updated with the batched GEMM.
constexpr int LU_NB = 64;
constexpr int LU_THREADS = 1024;

// W(:, c) = A(c, :) (column-major copy of the row-major A)
__global__ void lu_copy_kernel(const double *__restrict__ A, int64_t n, int64_t lda, double *__restrict__ W) {
    __shared__ double t[32][33];
    const int64_t r0 = (int64_t)blockIdx.y * 32, c0 = (int64_t)blockIdx.x * 32;
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int64_t r = r0 + k, c = c0 + threadIdx.x;
        t[k][threadIdx.x] = (r < n && c < n) ? A[r * lda + c] : 0.0;
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int64_t c = c0 + k, r = r0 + threadIdx.x;   // W(r, c) = A(r, c): column c contiguous in W
        if (r < n && c < n) W[r + c * n] = t[threadIdx.x][k];
    }
}

__global__ void __launch_bounds__(LU_THREADS) lu_panel_kernel(double *__restrict__ W, int64_t n, int64_t k0, int jb,
                                                              int *__restrict__ ipiv, int *status) {
    __shared__ double red_v[LU_THREADS / 32];
    __shared__ int64_t red_i[LU_THREADS / 32];
    __shared__ double prow[LU_NB];
    __shared__ int64_t s_p;
    __shared__ int s_bad;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_bad = 0;
    for (int j = 0; j < jb; ++j) {
        const int64_t col = k0 + j;
        const double *cj = W + col * n;
        double bv = -1.0;
        int64_t bi = INT64_MAX;
        for (int64_t i = col + tid; i < n; i += LU_THREADS) {
            const double a = fabs(cj[i]);
            if (a > bv) {
                bv = a;
                bi = i;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double ov = __shfl_down_sync(0xffffffffu, bv, o);
            const int64_t oi = __shfl_down_sync(0xffffffffu, bi, o);
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
            for (int w = 1; w < LU_THREADS / 32; ++w)
                if (red_v[w] > red_v[0] || (red_v[w] == red_v[0] && red_i[w] < red_i[0])) {
                    red_v[0] = red_v[w];
                    red_i[0] = red_i[w];
                }
            // no usable pivot (a zero or NaN column): record no exchange and stop
            const bool bad = !(red_v[0] > 0.0) || red_i[0] < col || red_i[0] >= n;
            if (bad) s_bad = 1;
            s_p = bad ? col : red_i[0];
            ipiv[col] = (int)(bad ? col : red_i[0]);
        }
        __syncthreads();
        if (s_bad) break;
        const int64_t p = s_p;
        // swap rows col and p over the panel's columns, and keep the pivot row
        for (int c = tid; c < jb; c += LU_THREADS) {
            double *wc = W + (k0 + c) * n;
            const double t = wc[col];
            wc[col] = wc[p];
            wc[p] = t;
            prow[c] = wc[col];
        }
        __syncthreads();
        const double d = 1.0 / prow[j];
        for (int64_t i = col + 1 + tid; i < n; i += LU_THREADS) {
            const double l = W[i + col * n] * d;
            W[i + col * n] = l;
            for (int c = j + 1; c < jb; ++c) W[i + (k0 + c) * n] -= l * prow[c];
        }
        __syncthreads();
    }
    if (tid == 0 && s_bad) atomicOr(status, ST_SINGULAR);
}

__global__ void lu_iota_kernel(int *__restrict__ ipiv, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        ipiv[i] = (int)i;
}

// the swaps of the panel k0 .. k0 + jb - 1 on every column outside it
__global__ void lu_laswp_kernel(double *__restrict__ W, int64_t n, int64_t k0, int jb, const int *__restrict__ ipiv) {
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x) {
        if (c >= k0 && c < k0 + jb) continue;
        double *wc = W + c * n;
        for (int j = 0; j < jb; ++j) {
            const int64_t r = k0 + j, p = ipiv[r];
            if (p != r && p >= 0 && p < n) {
                const double t = wc[r];
                wc[r] = wc[p];
                wc[p] = t;
            }
        }
    }
}

// Triangular solves with an nb x nb diagonal block T of W (rows/columns t0 ..
// t0 + nb - 1): unit lower (forward) or upper (backward), on the rows t0 ..
// t0 + nb - 1 of `cols` columns of M (ld ldm), one thread per column.
__global__ void lu_trsm_kernel(const double *__restrict__ W, int64_t n, int64_t t0, int nb, double *__restrict__ M,
                               int64_t ldm, int64_t cols, int upper) {
    __shared__ double T[LU_NB][LU_NB + 1];
    for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
        const int i = e % nb, j = e / nb;
        T[i][j] = W[(t0 + i) + (t0 + j) * n];
    }
    __syncthreads();
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= cols) return;
    double *m = M + c * ldm + t0;
    double x[LU_NB];
#pragma unroll
    for (int i = 0; i < LU_NB; ++i) x[i] = (i < nb) ? m[i] : 0.0;
    if (!upper) {
#pragma unroll
        for (int i = 0; i < LU_NB; ++i) {
            if (i >= nb) break;
            double v = x[i];
#pragma unroll
            for (int t = 0; t < LU_NB; ++t)
                if (t < i) v -= T[i][t] * x[t];
            x[i] = v;
        }
    } else {
#pragma unroll
        for (int i = LU_NB - 1; i >= 0; --i) {
            if (i >= nb) continue;
            double v = x[i];
#pragma unroll
            for (int t = 0; t < LU_NB; ++t)
                if (t > i && t < nb) v -= T[i][t] * x[t];
            x[i] = v / T[i][i];
        }
    }
#pragma unroll
    for (int i = 0; i < LU_NB; ++i)
        if (i < nb) m[i] = x[i];
}

// X(:, r) = P B(:, r): the recorded row swaps of the whole factorisation in order
__global__ void lu_permute_kernel(const double *__restrict__ B, int64_t ldb, double *__restrict__ X, int64_t ldx,
                                  int64_t n, int s, const int *__restrict__ ipiv) {
    const int r = blockIdx.x;
    if (r >= s) return;
    double *x = X + (int64_t)r * ldx;
    const double *b = B + (int64_t)r * ldb;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) x[i] = b[i];
    __syncthreads();
    if (threadIdx.x == 0)
        for (int64_t i = 0; i < n; ++i) {
            const int64_t p = ipiv[i];
            if (p != i && p >= 0 && p < n) {
                const double t = x[i];
                x[i] = x[p];
                x[p] = t;
            }
        }
}

}  // namespace

hodlr_status diag_solve(const hodlr_t *h, int s, double *X, int64_t ldx, cudaStream_t st, float2 *Xs) {
    const unsigned gx = (unsigned)std::max<int64_t>(1, std::min<int64_t>((h->n + 255) / 256, 1024));
    diag_apply_kernel<<<dim3(gx, (unsigned)s), 256, 0, st>>>(h->dinv, h->n, s, X, ldx, Xs);
    note_launch();
    HODLR_TRY_CUDA(cudaGetLastError());
    return HODLR_OK;
}

}  // namespace hodlr

using namespace hodlr;

extern "C" {

hodlr_status hodlr_build_diag(hodlr_ctx *c, const hodlr_matrix *A, hodlr_stream stream, hodlr_t **out) {
    if (!c || !A || !A->data || A->n <= 0 || A->ld < A->n || !out) {
        set_error("hodlr_build_diag: invalid argument");
        return HODLR_INVALID_ARG;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    HODLR_TRY_CUDA(cudaSetDevice(c->device));
    hodlr_t *h = new hodlr_t();
    h->ctx = c;
    h->A = A->data;
    h->n = A->n;
    h->lda = A->ld;
    h->sym = A->symmetric ? 1 : 0;
    h->L = 0;
    h->prec = HODLR_FP64;
    h->store = HODLR_FP64;
    h->diag = true;
    h->dinv = reinterpret_cast<double *>(own(h, (size_t)A->n * sizeof(double), st));
    if (!h->dinv) {
        hodlr_destroy(h);
        set_error("hodlr_build_diag: out of device memory");
        return HODLR_OUT_OF_MEMORY;
    }
    const unsigned gx = (unsigned)std::max<int64_t>(1, std::min<int64_t>((A->n + 255) / 256, 1024));
    diag_inverse_kernel<<<gx, 256, 0, st>>>(A->data, A->n, A->ld, h->dinv, c->d_status);
    note_launch();
    const hodlr_status r = take_status(c, st);
    if (r != HODLR_OK) {
        hodlr_destroy(h);
        return r;
    }
    h->factored = true;
    *out = h;
    return HODLR_OK;
}

hodlr_status hodlr_dense_lu_solve(hodlr_ctx *c, const hodlr_matrix *A, int s, const double *B, int64_t ldb,
                                  double *X, int64_t ldx, hodlr_stream stream) {
    if (!c || !A || !A->data || A->n <= 0 || A->ld < A->n || s <= 0 || !B || !X || ldb < A->n || ldx < A->n) {
        set_error("hodlr_dense_lu_solve: invalid argument");
        return HODLR_INVALID_ARG;
    }
    if (A->n > (int64_t)INT32_MAX) {
        set_error("hodlr_dense_lu_solve: n too large");
        return HODLR_RANGE;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    HODLR_TRY_CUDA(cudaSetDevice(c->device));
    const int64_t n = A->n;
    const int np = (int)((n + LU_NB - 1) / LU_NB);
    // descriptors of every trailing update and solve update, uploaded at once
    std::vector<GemmDesc<double>> gd;
    Arena ar;
    const size_t oW = ar.take((size_t)n * n * sizeof(double));
    const size_t oP = ar.take((size_t)n * sizeof(int));
    const size_t oD = ar.take((size_t)3 * np * sizeof(GemmDesc<double>));
    char *base = reinterpret_cast<char *>(dalloc(c, ar.bytes, st));
    if (!base) {
        set_error("hodlr_dense_lu_solve: out of device memory (%zu bytes)", ar.bytes);
        return HODLR_OUT_OF_MEMORY;
    }
    double *W = reinterpret_cast<double *>(base + oW);
    int *ipiv = reinterpret_cast<int *>(base + oP);
    GemmDesc<double> *dd = reinterpret_cast<GemmDesc<double> *>(base + oD);
    std::vector<int> upd(np, -1), fwd(np, -1), bwd(np, -1);
    for (int b = 0; b < np; ++b) {
        const int64_t k0 = (int64_t)b * LU_NB, jb = std::min<int64_t>(LU_NB, n - k0), r = n - k0 - jb;
        if (r > 0) {
            upd[b] = (int)gd.size();   // W22 -= L21 U12
            gd.push_back(GemmDesc<double>{W + (k0 + jb) + k0 * n, W + k0 + (k0 + jb) * n, W + (k0 + jb) + (k0 + jb) * n,
                                          n, n, n, (int)r, (int)r, (int)jb});
            fwd[b] = (int)gd.size();   // X(k0 + jb:, :) -= L21 X(k0:k0 + jb, :)
            gd.push_back(GemmDesc<double>{W + (k0 + jb) + k0 * n, X + k0, X + k0 + jb, n, ldx, ldx, (int)r, s,
                                          (int)jb});
        }
        if (k0 > 0) {
            bwd[b] = (int)gd.size();   // X(0:k0, :) -= U(0:k0, k0:k0 + jb) X(k0:k0 + jb, :)
            gd.push_back(GemmDesc<double>{W + k0 * n, X + k0, X, n, ldx, ldx, (int)k0, s, (int)jb});
        }
    }
    hodlr_status rs = HODLR_OK;
    auto fail = [&](hodlr_status r) {
        dfree(c, base, ar.bytes, st);
        return r;
    };
    if (!gd.empty() && cudaMemcpyAsync(dd, gd.data(), gd.size() * sizeof(GemmDesc<double>), cudaMemcpyHostToDevice,
                                       st) != cudaSuccess)
        return fail(HODLR_CUDA_ERROR);
    const unsigned nt = (unsigned)((n + 31) / 32);
    lu_copy_kernel<<<dim3(nt, nt), dim3(32, 8), 0, st>>>(A->data, n, A->ld, W);
    // every pivot index defined before anything reads one (a panel that meets a
    // zero column stops without writing the rest of its indices)
    lu_iota_kernel<<<(unsigned)std::min<int64_t>((n + 255) / 256, 1024), 256, 0, st>>>(ipiv, n);
    note_launch(2);
    const unsigned gsw = (unsigned)std::min<int64_t>((n + 255) / 256, 1024);
    for (int b = 0; b < np && rs == HODLR_OK; ++b) {
        const int64_t k0 = (int64_t)b * LU_NB;
        const int jb = (int)std::min<int64_t>(LU_NB, n - k0);
        const int64_t r = n - k0 - jb;
        lu_panel_kernel<<<1, LU_THREADS, 0, st>>>(W, n, k0, jb, ipiv, c->d_status);
        lu_laswp_kernel<<<gsw, 256, 0, st>>>(W, n, k0, jb, ipiv);
        note_launch(2);
        if (r > 0) {
            lu_trsm_kernel<<<(unsigned)((r + 127) / 128), 128, 0, st>>>(W, n, k0, jb, W + (k0 + jb) * n, n, r, 0);
            note_launch();
            rs = gemm_batched<double>(c, dd + upd[b], 1, (int)r, (int)r, jb, 0, -1.0, st);
        }
    }
    // X = P B, then L y = X (unit lower, forward) and U x = y (backward)
    if (rs == HODLR_OK) {
        lu_permute_kernel<<<(unsigned)s, 256, 0, st>>>(B, ldb, X, ldx, n, s, ipiv);
        note_launch();
        const unsigned gs = (unsigned)((s + 127) / 128);
        for (int b = 0; b < np && rs == HODLR_OK; ++b) {
            const int64_t k0 = (int64_t)b * LU_NB;
            const int jb = (int)std::min<int64_t>(LU_NB, n - k0);
            lu_trsm_kernel<<<gs, 128, 0, st>>>(W, n, k0, jb, X, ldx, s, 0);
            note_launch();
            if (fwd[b] >= 0) rs = gemm_batched<double>(c, dd + fwd[b], 1, (int)(n - k0 - jb), s, jb, 0, -1.0, st);
        }
        for (int b = np - 1; b >= 0 && rs == HODLR_OK; --b) {
            const int64_t k0 = (int64_t)b * LU_NB;
            const int jb = (int)std::min<int64_t>(LU_NB, n - k0);
            lu_trsm_kernel<<<gs, 128, 0, st>>>(W, n, k0, jb, X, ldx, s, 1);
            note_launch();
            if (bwd[b] >= 0) rs = gemm_batched<double>(c, dd + bwd[b], 1, (int)k0, s, jb, 0, -1.0, st);
        }
    }
    if (rs == HODLR_OK && cudaGetLastError() != cudaSuccess) rs = HODLR_CUDA_ERROR;
    if (rs != HODLR_OK) {
        cudaStreamSynchronize(st);
        return fail(rs);
    }
    const hodlr_status r2 = take_status(c, st);
    dfree(c, base, ar.bytes, st);
    return r2;
}

}  // extern "C"
