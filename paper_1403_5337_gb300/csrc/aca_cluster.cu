// Partial-pivoting ACA (Sec. 5.1) with one thread-block cluster per
// off-diagonal block.
//
// The cluster's CL CTAs split the block's rows and columns into contiguous
// slices.  Every CTA keeps its slice of the u_l and v_l columns resident in
// shared memory (as many columns as fit; later ones stay in global memory), so
// the k-term residual of a row or column entry is read at shared-memory latency
// instead of being streamed from L2 by one SM.  Per step:
//   row pass     r_j = A(i_k, j) - sum_l U(i_k, l) V(j, l) on the CTA's columns,
//                local argmax -> candidate in shared memory
//   cluster barrier; every CTA reduces the CL candidates over DSMEM (same order,
//                so the same pivot everywhere)
//   v_k = r / r(j_k) on the CTA's columns
//   column pass  u_i = A(i, j_k) - sum_l V(j_k, l) U(i, l) on the CTA's rows,
//                local argmax over unused rows, partial dot products u_k.u_l and
//                v_k.v_l over the CTA's slices
//   cluster barrier; every CTA sums the partials over DSMEM in rank order and
//                takes the same stop decision
// Candidate and partial-sum slots are double-buffered by step parity, so two
// cluster barriers per step suffice.  The arithmetic of each residual entry
// (terms l = 0..k-1, separate round-to-nearest multiply and subtract), the
// tie-breaking (lowest index) and the zero-row rule are those of the
// single-block formulation.
#include <cooperative_groups.h>

#include <algorithm>
#include <climits>
#include <vector>

#include "internal.cuh"

namespace cg = cooperative_groups;

namespace hodlr {
namespace {

constexpr int CT = 256;            // threads per CTA
constexpr int CW = CT / 32;
constexpr int ACA_CAP = 1024;      // maximum rank (staging width)

struct Cand {
    double a;     // |value|, -1 = none
    double v;     // signed value
    int idx;      // block-local index, INT_MAX = none
    int pad;
};

__device__ __forceinline__ bool better(double a, int i, double ba, int bi) {
    return a > ba || (a == ba && i < bi);
}

// CTA-wide argmax of (a, idx, v); the result is returned in every thread.
__device__ Cand cta_argmax(double a, int idx, double v, Cand *red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double oa = __shfl_down_sync(0xffffffffu, a, o);
        const int oi = __shfl_down_sync(0xffffffffu, idx, o);
        const double ov = __shfl_down_sync(0xffffffffu, v, o);
        if (better(oa, oi, a, idx)) {
            a = oa;
            idx = oi;
            v = ov;
        }
    }
    if (lane == 0) red[warp] = Cand{a, v, idx, 0};
    __syncthreads();
    Cand best = red[0];
    for (int w = 1; w < CW; ++w)
        if (better(red[w].a, red[w].idx, best.a, best.idx)) best = red[w];
    __syncthreads();
    return best;
}

// Best of the CL cluster candidates slot[which]: lane q of every warp loads rank
// q's candidate over DSMEM, then an xor-shuffle argmax (ties -> lowest index)
// leaves the same result in every thread.
__device__ __forceinline__ Cand cluster_best(cg::cluster_group &cl, Cand *slot, int which, int CL) {
    const int lane = threadIdx.x & 31;
    double a = -1.0, v = 0.0;
    int idx = INT_MAX;
    if (lane < CL) {
        const Cand o = cl.map_shared_rank(slot, lane)[which];
        a = o.a;
        v = o.v;
        idx = o.idx;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double oa = __shfl_xor_sync(0xffffffffu, a, o);
        const double ov = __shfl_xor_sync(0xffffffffu, v, o);
        const int oi = __shfl_xor_sync(0xffffffffu, idx, o);
        if (better(oa, oi, a, idx)) {
            a = oa;
            v = ov;
            idx = oi;
        }
    }
    return Cand{a, v, idx, 0};
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <typename T>
__global__ void __launch_bounds__(CT, 1)
    aca_cluster_kernel(const double *__restrict__ A, int64_t lda, int sym, const AcaBlockDesc *__restrict__ blocks,
                       double tol, int kcs, int *status) {
    cg::cluster_group cl = cg::this_cluster();
    const int CL = (int)cl.num_blocks();
    const int c = (int)cl.block_rank();
    const AcaBlockDesc B = blocks[blockIdx.x / CL];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t m = B.m, nc = B.nc, ld = B.ld;
    const int64_t mr = (m + CL - 1) / CL, nr = (nc + CL - 1) / CL;
    const int64_t smr = mr + 1, snr = nr + 1;   // padded shared-memory strides (no bank conflicts)
    const int64_t i0 = std::min<int64_t>(m, c * mr), i1 = std::min<int64_t>(m, i0 + mr);
    const int64_t j0 = std::min<int64_t>(nc, c * nr), j1 = std::min<int64_t>(nc, j0 + nr);
    const int64_t mn = m < nc ? m : nc;
    const int kmax = (int)(B.cap < mn ? B.cap : mn);
    T *Ug = reinterpret_cast<T *>(B.U) + B.r0;   // Ug[l * ld + i], i block-local row
    T *Vg = reinterpret_cast<T *>(B.V) + B.c0;   // Vg[l * ld + j]

    // shared memory: 8-byte-aligned parts first, then the T arrays, then flags
    extern __shared__ __align__(16) unsigned char smem[];
    double *tot = reinterpret_cast<double *>(smem);                  // [2 (ACA_CAP + 1)] summed dots
    Cand *slot = reinterpret_cast<Cand *>(tot + 2 * (ACA_CAP + 1));  // [2 parities][row, col, free]
    T *dots = reinterpret_cast<T *>(slot + 6);                       // [2][2 (ACA_CAP + 1)] partial dots
    T *pu = dots + 4 * (ACA_CAP + 1);                                // U(i_k, 0..k-1)
    T *pv = pu + ACA_CAP;                                            // V(j_k, 0..k-1)
    T *Us = pv + ACA_CAP;                                            // [kcs][smr]
    T *Vs = Us + (size_t)kcs * smr;                                  // [kcs][snr]
    unsigned char *used = reinterpret_cast<unsigned char *>(Vs + (size_t)kcs * snr);  // [mr]
    __shared__ Cand red[CW];
    __shared__ double s_norm2;
    __shared__ int s_i, s_stop;

    for (int64_t i = tid; i < mr; i += CT) used[i] = 0;
    if (tid == 0) {
        s_norm2 = 0.0;
        s_i = 0;
        s_stop = 0;
    }
    __syncthreads();
    cl.sync();

    int k = 0;
    while (k < kmax) {
        const int par = k & 1;
        const int i = s_i;
        {
            // U(i_k, l): from the shared-memory slice of the CTA that owns row i_k
            const int co = (int)(i / mr);
            const int64_t li = i - (int64_t)co * mr;
            const T *Uo = cl.map_shared_rank(Us, co);
            for (int l = tid; l < k; l += CT) pu[l] = (l < kcs) ? Uo[(size_t)l * smr + li] : Ug[(int64_t)l * ld + i];
        }
        __syncthreads();
        // ---- row pass on own columns -> v_k (unscaled)
        const int kin = k < kcs ? k : kcs;
        double ba = -1.0, bv = 0.0;
        int bi = INT_MAX;
        const double *arow = A + (B.r0 + i) * lda + B.c0;
        for (int64_t j = j0 + tid; j < j1; j += CT) {
            const int64_t jl = j - j0;
            T r = dev::from_double<T>(arow[j]);
            int l = 0;
#pragma unroll 8
            for (; l < kin; ++l) r = dev::sub_rn(r, dev::mul_rn(pu[l], Vs[(size_t)l * snr + jl]));
            for (; l < k; ++l) r = dev::sub_rn(r, dev::mul_rn(pu[l], Vg[(int64_t)l * ld + j]));
            if (k < kcs) Vs[(size_t)k * snr + jl] = r;
            Vg[(int64_t)k * ld + j] = r;
            const double a = fabs((double)r);
            if (a != a) atomicOr(status, ST_NONFINITE);
            if (a > ba) {
                ba = a;
                bi = (int)j;
                bv = (double)r;
            }
        }
        Cand cr = cta_argmax(ba, bi, bv, red);
        if (tid == 0) slot[par * 3 + 0] = cr;
        cl.sync();
        const Cand best = cluster_best(cl, slot, par * 3 + 0, CL);
        const int jk = best.idx;
        const T piv = (T)best.v;
        // the owner of row i marks it used
        if (i >= i0 && i < i1 && tid == 0) used[i - i0] = 1;
        __syncthreads();
        if (jk == INT_MAX || piv == T(0)) {
            // exhausted row: the lowest unused row of the whole block, if any
            double fa = -1.0;
            int fi = INT_MAX;
            for (int64_t q = i0 + tid; q < i1; q += CT)
                if (!used[q - i0] && fa < 0.0) {
                    fa = 0.0;
                    fi = (int)q;
                }
            Cand cf = cta_argmax(fa, fi, 0.0, red);
            if (tid == 0) slot[par * 3 + 2] = cf;
            cl.sync();
            const Cand bf = cluster_best(cl, slot, par * 3 + 2, CL);
            if (bf.a < 0.0) break;
            if (tid == 0) s_i = bf.idx;
            __syncthreads();
            continue;
        }
        // ---- scale own columns of v_k
        for (int64_t j = j0 + tid; j < j1; j += CT) {
            const int64_t jl = j - j0;
            const T v = dev::div_rn(Vg[(int64_t)k * ld + j], piv);
            if (k < kcs) Vs[(size_t)k * snr + jl] = v;
            Vg[(int64_t)k * ld + j] = v;
        }
        // V(j_k, l) for l < k: written in earlier steps by the owner of column j_k
        {
            const int cv = (int)(jk / nr);
            const int64_t lj = jk - (int64_t)cv * nr;
            const T *Vo = cl.map_shared_rank(Vs, cv);
            for (int l = tid; l < k; l += CT) pv[l] = (l < kcs) ? Vo[(size_t)l * snr + lj] : Vg[(int64_t)l * ld + jk];
        }
        __syncthreads();
        // ---- column pass on own rows -> u_k
        const double *acol;
        int64_t astr;
        if (sym) {
            acol = A + (B.c0 + jk) * lda + B.r0;
            astr = 1;
        } else {
            acol = A + B.r0 * lda + B.c0 + jk;
            astr = lda;
        }
        double ca = -1.0, cv = 0.0;
        int ci = INT_MAX;
        for (int64_t q = i0 + tid; q < i1; q += CT) {
            const int64_t ql = q - i0;
            T u = dev::from_double<T>(acol[q * astr]);
            int l = 0;
#pragma unroll 8
            for (; l < kin; ++l) u = dev::sub_rn(u, dev::mul_rn(pv[l], Us[(size_t)l * smr + ql]));
            for (; l < k; ++l) u = dev::sub_rn(u, dev::mul_rn(pv[l], Ug[(int64_t)l * ld + q]));
            if (k < kcs) Us[(size_t)k * smr + ql] = u;
            Ug[(int64_t)k * ld + q] = u;
            if (u != u) atomicOr(status, ST_NONFINITE);
            if (!used[ql]) {
                const double a = fabs((double)u);
                if (a > ca) {
                    ca = a;
                    ci = (int)q;
                    cv = (double)u;
                }
            }
        }
        Cand cc = cta_argmax(ca, ci, cv, red);
        // ---- partial dots over own slices, l = 0..k: one thread per l runs down the
        // slice (padded strides keep the lanes on distinct banks); columns beyond
        // the shared-memory capacity use one warp per l over global memory
        T *dp = dots + (size_t)par * 2 * (ACA_CAP + 1);
        if (k < kcs) {
            const int64_t nrow = i1 - i0, ncol = j1 - j0;
            const T *uk = Us + (size_t)k * smr;
            const T *vk = Vs + (size_t)k * snr;
            for (int l = tid; l <= k; l += CT) {
                const T *ul = Us + (size_t)l * smr;
                const T *vl = Vs + (size_t)l * snr;
                // four interleaved partial sums (fixed combination order)
                T su[4] = {T(0), T(0), T(0), T(0)}, sv[4] = {T(0), T(0), T(0), T(0)};
                int64_t q = 0;
                for (; q + 4 <= nrow; q += 4) {
#pragma unroll
                    for (int t = 0; t < 4; ++t) su[t] = fma(ul[q + t], uk[q + t], su[t]);
                }
                for (; q < nrow; ++q) su[0] = fma(ul[q], uk[q], su[0]);
                q = 0;
                for (; q + 4 <= ncol; q += 4) {
#pragma unroll
                    for (int t = 0; t < 4; ++t) sv[t] = fma(vl[q + t], vk[q + t], sv[t]);
                }
                for (; q < ncol; ++q) sv[0] = fma(vl[q], vk[q], sv[0]);
                dp[l] = (su[0] + su[1]) + (su[2] + su[3]);
                dp[ACA_CAP + 1 + l] = (sv[0] + sv[1]) + (sv[2] + sv[3]);
            }
        } else {
            for (int l = warp; l <= k; l += CW) {
                T su = T(0), sv = T(0);
                for (int64_t q = i0 + lane; q < i1; q += 32) su = fma(Ug[(int64_t)l * ld + q], Ug[(int64_t)k * ld + q], su);
                for (int64_t j = j0 + lane; j < j1; j += 32) sv = fma(Vg[(int64_t)l * ld + j], Vg[(int64_t)k * ld + j], sv);
                su = warp_sum(su);
                sv = warp_sum(sv);
                if (lane == 0) {
                    dp[l] = su;
                    dp[ACA_CAP + 1 + l] = sv;
                }
            }
        }
        if (tid == 0) slot[par * 3 + 1] = cc;
        __syncthreads();
        cl.sync();
        // ---- cluster-wide: next row, dot products (rank order), stop decision
        const Cand bc = cluster_best(cl, slot, par * 3 + 1, CL);
        for (int l = tid; l <= k; l += CT) {
            T su = T(0), sv = T(0);
#pragma unroll 4
            for (int q = 0; q < CL; ++q) {
                const T *rp = cl.map_shared_rank(dots, q) + (size_t)par * 2 * (ACA_CAP + 1);
                su += rp[l];
                sv += rp[ACA_CAP + 1 + l];
            }
            tot[l] = (double)su;
            tot[ACA_CAP + 1 + l] = (double)sv;
        }
        __syncthreads();
        // cross term sum_{l<k} (u_k.u_l)(v_k.v_l): lane-strided partial sums, then a
        // fixed xor-shuffle tree (the same order in every CTA of the cluster)
        double cross = 0.0;
        if (warp == 0) {
            for (int l = lane; l < k; l += 32) cross += tot[l] * tot[ACA_CAP + 1 + l];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) cross += __shfl_xor_sync(0xffffffffu, cross, o);
        }
        if (tid == 0) {
            const double uu = tot[k], vv = tot[ACA_CAP + 1 + k];
            s_norm2 = s_norm2 + 2.0 * cross + uu * vv;
            if (c == 0) {
                B.prow[k] = i;
                B.pcol[k] = jk;
            }
            const double nrm = s_norm2 > 0.0 ? s_norm2 : 0.0;
            int stop = (sqrt(uu) * sqrt(vv) <= tol * sqrt(nrm));
            if ((int64_t)(k + 1) >= mn) stop = 1;
            if (bc.a < 0.0) stop = 1;   // every row used
            s_stop = stop;
            s_i = bc.idx;
        }
        __syncthreads();
        ++k;
        if (s_stop) break;
    }
    if (c == 0 && tid == 0) {
        *B.rank = k;
        *B.cap_hit = (k == B.cap && (int64_t)k < mn) ? 1 : 0;
    }
    // no CTA may leave while another can still read its shared memory
    cl.sync();
}

constexpr size_t SMEM_BUDGET = 220 * 1024;

template <typename T>
size_t fixed_smem() {
    return sizeof(T) * (2 * ACA_CAP + 4 * (ACA_CAP + 1)) + sizeof(double) * 2 * (ACA_CAP + 1) + sizeof(Cand) * 6 + 16;
}

template <typename T>
hodlr_status launch_level(hodlr_ctx *c, const double *A, int64_t lda, int sym, const AcaBlockDesc *d_blocks,
                          int nblocks, int CL, int64_t mr, int64_t nr, double tol, cudaStream_t s) {
    const size_t fixed = fixed_smem<T>() + (size_t)mr + 16;
    int kcs = 0;
    if (fixed < SMEM_BUDGET)
        kcs = (int)std::min<size_t>(ACA_CAP, (SMEM_BUDGET - fixed) / ((mr + nr + 2) * sizeof(T)));
    const size_t sm = fixed + (size_t)kcs * (mr + nr + 2) * sizeof(T);
    HODLR_TRY_CUDA(cudaFuncSetAttribute(aca_cluster_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    if (CL > 8)
        HODLR_TRY_CUDA(cudaFuncSetAttribute(aca_cluster_kernel<T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(nblocks * CL));
    cfg.blockDim = dim3(CT);
    cfg.dynamicSmemBytes = sm;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    HODLR_TRY_CUDA(cudaLaunchKernelEx(&cfg, aca_cluster_kernel<T>, A, lda, sym, d_blocks, tol, kcs, c->d_status));
    return HODLR_OK;
}

}  // namespace

hodlr_status launch_aca_levels(hodlr_ctx *c, const double *A, int64_t lda, int sym, int cprec,
                               const AcaBlockDesc *d_blocks, const std::vector<int> &level_first,
                               const std::vector<int64_t> &level_maxdim, double tol, cudaStream_t s) {
    // level_first[l] .. level_first[l+1]: the blocks of level l (all of one size class)
    const int nlev = (int)level_first.size() - 1;
    cudaEvent_t fork;
    HODLR_TRY_CUDA(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
    HODLR_TRY_CUDA(cudaEventRecord(fork, s));
    std::vector<cudaEvent_t> joins;
    hodlr_status rs = HODLR_OK;
    for (int l = 0; l < nlev && rs == HODLR_OK; ++l) {
        const int nb = level_first[l + 1] - level_first[l];
        if (nb == 0) continue;
        const int64_t dim = level_maxdim[l];
        int CL = 1;
        while (CL < 16 && dim > (int64_t)CL * 128) CL *= 2;
        const int64_t mr = (dim + CL - 1) / CL;
        cudaStream_t ls = c->side[l % HODLR_SIDE_STREAMS];
        if (cudaStreamWaitEvent(ls, fork, 0) != cudaSuccess) {
            rs = HODLR_CUDA_ERROR;
            break;
        }
        const AcaBlockDesc *db = d_blocks + level_first[l];
        rs = (cprec == HODLR_FP64) ? launch_level<double>(c, A, lda, sym, db, nb, CL, mr, mr, tol, ls)
                                   : launch_level<float>(c, A, lda, sym, db, nb, CL, mr, mr, tol, ls);
        cudaEvent_t j;
        cudaEventCreateWithFlags(&j, cudaEventDisableTiming);
        cudaEventRecord(j, ls);
        joins.push_back(j);
    }
    for (auto j : joins) {
        cudaStreamWaitEvent(s, j, 0);
        cudaEventDestroy(j);
    }
    cudaEventDestroy(fork);
    return rs;
}

}  // namespace hodlr
