// Partial-pivoting adaptive cross approximation of every off-diagonal block of
// every HODLR level at once (Sec. 5.1; the compression step of Sec. 4.3,
// Factorize step 1).
//
// One CTA owns one block A(rows, cols) and runs the greedy cross sequence:
//   step k: r = A(i_k, :) - sum_l U(i_k, l) V(:, l)   -> j_k = argmax |r|
//           v_k = r / r(j_k)
//           u_k = A(:, j_k) - sum_l V(j_k, l) U(:, l)  -> i_{k+1} = argmax_unused |u_k|
//           ||S_k||_F^2 += 2 sum_{l<k} (u_k.u_l)(v_k.v_l) + ||u_k||^2 ||v_k||^2
//   stop after term k when ||u_k|| ||v_k|| <= tol ||S_k||_F, at min(m, n) or the cap.
// The residual entries are formed term by term (l = 0..k-1) with a separate
// round-to-nearest multiply and subtract, in the compression precision T, so the
// pivot decisions are reproducible.  Ties in every argmax go to the lowest index.
// An exactly zero residual row marks the row used and retries the lowest unused row.
// Rows/columns are written straight into the column-major U/V staging (the
// residual row becomes v_k in place), so shared memory only holds the k scalars
// of the pivot row/column, the dot products and the used-row flags.
#include <climits>

#include "internal.cuh"

namespace hodlr {
namespace {

constexpr int ACA_THREADS = 1024;
constexpr int ACA_WARPS = ACA_THREADS / 32;

template <typename T>
__device__ __forceinline__ void warp_argmax(T &v, int &i) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        T ov = __shfl_down_sync(0xffffffffu, v, o);
        int oi = __shfl_down_sync(0xffffffffu, i, o);
        if (ov > v || (ov == v && oi < i)) {
            v = ov;
            i = oi;
        }
    }
}

// Block-wide argmax (value, index; ties -> lowest index).  Result valid in all
// threads on return.
template <typename T>
__device__ void block_argmax(T &v, int &i, T *red_v, int *red_i) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    warp_argmax(v, i);
    if (lane == 0) {
        red_v[warp] = v;
        red_i[warp] = i;
    }
    __syncthreads();
    if (warp == 0) {
        v = lane < ACA_WARPS ? red_v[lane] : T(-1);
        i = lane < ACA_WARPS ? red_i[lane] : INT_MAX;
        warp_argmax(v, i);
        if (lane == 0) {
            red_v[0] = v;
            red_i[0] = i;
        }
    }
    __syncthreads();
    v = red_v[0];
    i = red_i[0];
    __syncthreads();
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <typename T>
__global__ void __launch_bounds__(ACA_THREADS, 1)
    aca_kernel(const double *__restrict__ A, int64_t lda, int sym,
               const AcaBlockDesc *__restrict__ blocks, double tol, int *status) {
    const AcaBlockDesc B = blocks[blockIdx.x];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    extern __shared__ __align__(16) unsigned char smem[];
    T *s_ui = reinterpret_cast<T *>(smem);   // U(i_k, 0..k-1)
    T *s_vj = s_ui + B.cap;                  // V(j_k, 0..k-1)
    T *s_du = s_vj + B.cap;                  // u_k . u_l, l = 0..k
    T *s_dv = s_du + B.cap + 1;              // v_k . v_l
    unsigned char *used = reinterpret_cast<unsigned char *>(s_dv + B.cap + 1);
    __shared__ T red_v[ACA_WARPS];
    __shared__ int red_i[ACA_WARPS];
    __shared__ int s_i, s_stop;
    __shared__ double s_norm2;

    T *U = reinterpret_cast<T *>(B.U);
    T *V = reinterpret_cast<T *>(B.V);
    const int64_t ld = B.ld, m = B.m, nc = B.nc;
    const int64_t mn = m < nc ? m : nc;
    const int kmax = (int)(B.cap < mn ? B.cap : mn);
    for (int64_t i = tid; i < m; i += ACA_THREADS) used[i] = 0;
    if (tid == 0) {
        s_i = 0;
        s_stop = 0;
        s_norm2 = 0.0;
    }
    __syncthreads();

    int k = 0;
    while (k < kmax) {
        const int i = s_i;
        for (int l = tid; l < k; l += ACA_THREADS) s_ui[l] = U[(int64_t)l * ld + B.r0 + i];
        __syncthreads();
        // ---- residual row -> V(:, k)
        const double *arow = A + (B.r0 + i) * lda + B.c0;
        T *vk = V + (int64_t)k * ld + B.c0;
        T bv = T(-1);
        int bj = INT_MAX;
        for (int64_t j = tid; j < nc; j += ACA_THREADS) {
            T r = dev::from_double<T>(arow[j]);
            const T *vcol = V + B.c0 + j;
            for (int l = 0; l < k; ++l) r = dev::sub_rn(r, dev::mul_rn(s_ui[l], vcol[(int64_t)l * ld]));
            vk[j] = r;
            T a = fabs(r);
            if (a != a) atomicOr(status, ST_NONFINITE);
            if (a > bv) {
                bv = a;
                bj = (int)j;
            }
        }
        block_argmax(bv, bj, red_v, red_i);
        if (tid == 0) used[i] = 1;
        const T piv = (bj < nc) ? vk[bj] : T(0);
        __syncthreads();
        if (piv == T(0)) {
            // exhausted row: retry the lowest unused row, if any
            T fv = T(-1);
            int fi = INT_MAX;
            for (int64_t i2 = tid; i2 < m; i2 += ACA_THREADS)
                if (!used[i2] && fv < T(0)) {
                    fv = T(0);
                    fi = (int)i2;
                }
            block_argmax(fv, fi, red_v, red_i);
            if (fv < T(0)) break;
            if (tid == 0) s_i = fi;
            __syncthreads();
            continue;
        }
        for (int64_t j = tid; j < nc; j += ACA_THREADS) vk[j] = dev::div_rn(vk[j], piv);
        for (int l = tid; l < k; l += ACA_THREADS) s_vj[l] = V[(int64_t)l * ld + B.c0 + bj];
        __syncthreads();
        // ---- residual column -> U(:, k)
        T *uk = U + (int64_t)k * ld + B.r0;
        const double *acol;
        int64_t astride;
        if (sym) {
            acol = A + (B.c0 + bj) * lda + B.r0;
            astride = 1;
        } else {
            acol = A + B.r0 * lda + B.c0 + bj;
            astride = lda;
        }
        T bu = T(-1);
        int bi = INT_MAX;
        for (int64_t i2 = tid; i2 < m; i2 += ACA_THREADS) {
            T u = dev::from_double<T>(acol[i2 * astride]);
            const T *ucol = U + B.r0 + i2;
            for (int l = 0; l < k; ++l) u = dev::sub_rn(u, dev::mul_rn(s_vj[l], ucol[(int64_t)l * ld]));
            uk[i2] = u;
            if (u != u) atomicOr(status, ST_NONFINITE);
            if (!used[i2]) {
                T a = fabs(u);
                if (a > bu) {
                    bu = a;
                    bi = (int)i2;
                }
            }
        }
        block_argmax(bu, bi, red_v, red_i);
        // ---- dot products u_k.u_l and v_k.v_l (l = 0..k), one warp per l
        for (int l = warp; l <= k; l += ACA_WARPS) {
            const T *ul = U + (int64_t)l * ld + B.r0;
            const T *vl = V + (int64_t)l * ld + B.c0;
            T su = T(0), sv = T(0);
            for (int64_t i2 = lane; i2 < m; i2 += 32) su = fma(ul[i2], uk[i2], su);
            for (int64_t j = lane; j < nc; j += 32) sv = fma(vl[j], vk[j], sv);
            su = warp_sum(su);
            sv = warp_sum(sv);
            if (lane == 0) {
                s_du[l] = su;
                s_dv[l] = sv;
            }
        }
        __syncthreads();
        if (tid == 0) {
            double cross = 0.0;
            for (int l = 0; l < k; ++l) cross += (double)s_du[l] * (double)s_dv[l];
            const double uu = (double)s_du[k], vv = (double)s_dv[k];
            s_norm2 = s_norm2 + 2.0 * cross + uu * vv;
            B.prow[k] = i;
            B.pcol[k] = bj;
            const double nrm = s_norm2 > 0.0 ? s_norm2 : 0.0;
            int stop = (sqrt(uu) * sqrt(vv) <= tol * sqrt(nrm));
            if ((int64_t)(k + 1) >= mn) stop = 1;
            if (bu < T(0)) stop = 1;   // every row used
            s_stop = stop;
            s_i = bi;
        }
        __syncthreads();
        ++k;
        if (s_stop) break;
    }
    if (tid == 0) {
        *B.rank = k;
        *B.cap_hit = (k == B.cap && (int64_t)k < mn) ? 1 : 0;
    }
}

}  // namespace

hodlr_status launch_aca(hodlr_ctx *c, const double *A, int64_t lda, int sym, int cprec,
                        const AcaBlockDesc *d_blocks, int nblocks, int64_t max_m, double tol,
                        cudaStream_t s) {
    if (nblocks == 0) return HODLR_OK;
    // the cap is uniform per call (all blocks share the same staging width bound)
    // shared memory: 4 cap + 2 scalars of T plus max_m flags; cap <= 1024.
    const int cap = 1024;
    if (cprec == HODLR_FP64) {
        size_t sm = (4 * (size_t)cap + 2) * sizeof(double) + (size_t)max_m + 16;
        HODLR_TRY_CUDA(cudaFuncSetAttribute(aca_kernel<double>,
                                            cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        aca_kernel<double><<<nblocks, ACA_THREADS, sm, s>>>(A, lda, sym, d_blocks, tol, c->d_status);
    } else {
        size_t sm = (4 * (size_t)cap + 2) * sizeof(float) + (size_t)max_m + 16;
        HODLR_TRY_CUDA(cudaFuncSetAttribute(aca_kernel<float>,
                                            cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        aca_kernel<float><<<nblocks, ACA_THREADS, sm, s>>>(A, lda, sym, d_blocks, tol, c->d_status);
    }
    HODLR_TRY_CUDA(cudaGetLastError());
    return HODLR_OK;
}

}  // namespace hodlr
