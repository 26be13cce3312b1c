// Partial-pivoting ACA (Sec. 5.1) with one thread-block cluster per
// off-diagonal block.
//
// The cluster's CL CTAs split the block's rows and columns into contiguous
// slices.  Every CTA keeps its slice of the u_l and v_l columns resident in
// shared memory (as many columns as fit; later ones stay in global memory), so
// the k-term residual of a row or column entry is read at shared-memory latency
// instead of being streamed from L2 by one SM.  Per step:
//   row pass     r_j = A(i_k, j) - sum_l U(i_k, l) V(j, l) on the CTA's columns
//                (kept in registers), local argmax -> candidate slot
//   cluster barrier; every CTA reduces the CL candidates over DSMEM (same order,
//                so the same pivot everywhere) and starts loading column j_k of A
//   v_k = r / r(j_k) on the CTA's columns
//   column pass  u_i = A(i, j_k) - sum_l V(j_k, l) U(i, l) on the CTA's rows,
//                local argmax over unused rows, partial dot products u_k.u_l and
//                v_k.v_l over the CTA's slices (16-byte shared-memory loads)
//   cluster barrier; every CTA picks the next row i_{k+1}, starts loading row
//                i_{k+1} of A and gathering U(i_{k+1}, :), sums the partials over
//                DSMEM in rank order and takes the same stop decision
// Candidate and partial-sum slots are double-buffered by step parity, so two
// cluster barriers per step suffice.  Pivot candidates are compared in the
// compression precision (the same argmax as after widening); the norm
// recurrence and the stopping test are FP64.  The arithmetic of each residual
// entry (terms l = 0..k-1, separate round-to-nearest multiply and subtract), the
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
constexpr int MAX_CL = 16;         // largest cluster

// A pivot candidate in the compression precision T: comparing |r| in T picks the
// same entry as comparing it after a widening conversion, and keeps the
// reductions off GB300's narrow FP64 pipe.
template <typename T>
struct Cand {
    T a;      // |value|, -1 = none
    T v;      // signed value
    int idx;  // block-local index, INT_MAX = none
    int pad;
};

template <typename T>
__device__ __forceinline__ bool better(T a, int i, T ba, int bi) {
    return a > ba || (a == ba && i < bi);
}

// xor-shuffle argmax inside groups of W lanes: every lane of a group ends with
// the group's best (largest |value|, lowest index on ties).
template <typename T, int W>
__device__ __forceinline__ void shfl_argmax(T &a, T &v, int &idx) {
#pragma unroll
    for (int o = W / 2; o > 0; o >>= 1) {
        const T oa = __shfl_xor_sync(0xffffffffu, a, o);
        const T ov = __shfl_xor_sync(0xffffffffu, v, o);
        const int oi = __shfl_xor_sync(0xffffffffu, idx, o);
        if (better(oa, oi, a, idx)) {
            a = oa;
            v = ov;
            idx = oi;
        }
    }
}

template <typename T>
__device__ __forceinline__ Cand<T> lane0(T a, T v, int idx) {
    return Cand<T>{__shfl_sync(0xffffffffu, a, 0), __shfl_sync(0xffffffffu, v, 0),
                   __shfl_sync(0xffffffffu, idx, 0), 0};
}

// CTA-wide argmax; the result is returned in every thread.  One barrier: the
// caller keeps consecutive uses of the same `red` apart by another barrier.
template <typename T>
__device__ Cand<T> cta_argmax(T a, int idx, T v, Cand<T> *red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    shfl_argmax<T, 32>(a, v, idx);
    if (lane == 0) red[warp] = Cand<T>{a, v, idx, 0};
    __syncthreads();
    T ra = T(-1), rv = T(0);
    int ri = INT_MAX;
    if (lane < CW) {
        const Cand<T> o = red[lane];
        ra = o.a;
        rv = o.v;
        ri = o.idx;
    }
    shfl_argmax<T, CW>(ra, rv, ri);
    return lane0(ra, rv, ri);
}

// Candidate exchange: every CTA posts its candidate into slot c of every CTA
// of the cluster (remote shared-memory stores, ordered by the cluster barrier
// that follows), so that after the barrier each CTA reduces the CL candidates
// from its own shared memory, in the same order everywhere.
template <typename T>
__device__ __forceinline__ void post_cand(cg::cluster_group &cl, Cand<T> *slots, int c, int CL, const Cand<T> &v) {
    const int t = threadIdx.x;
    if (t < CL) cl.map_shared_rank(slots, t)[c] = v;
}
template <typename T>
__device__ __forceinline__ Cand<T> best_of_slots(const Cand<T> *slots, int CL) {
    const int lane = threadIdx.x & 31;
    T a = T(-1), v = T(0);
    int idx = INT_MAX;
    if (lane < CL) {
        const Cand<T> o = slots[lane];
        a = o.a;
        v = o.v;
        idx = o.idx;
    }
    shfl_argmax<T, MAX_CL>(a, v, idx);
    return lane0(a, v, idx);
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Dot product of two shared-memory columns of nv 16-byte groups (zero-padded).
__device__ __forceinline__ float vdot(const float *x, const float *y, int nv) {
    const float4 *x4 = reinterpret_cast<const float4 *>(x), *y4 = reinterpret_cast<const float4 *>(y);
    float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
    for (int q = 0; q < nv; ++q) {
        const float4 a = x4[q], b = y4[q];
        s0 = fmaf(a.x, b.x, s0);
        s1 = fmaf(a.y, b.y, s1);
        s2 = fmaf(a.z, b.z, s2);
        s3 = fmaf(a.w, b.w, s3);
    }
    return (s0 + s1) + (s2 + s3);
}
__device__ __forceinline__ double vdot(const double *x, const double *y, int nv) {
    const double2 *x2 = reinterpret_cast<const double2 *>(x), *y2 = reinterpret_cast<const double2 *>(y);
    double s0 = 0.0, s1 = 0.0;
    for (int q = 0; q < nv; ++q) {
        const double2 a = x2[q], b = y2[q];
        s0 = fma(a.x, b.x, s0);
        s1 = fma(a.y, b.y, s1);
    }
    return s0 + s1;
}

// Sum of the exact products su sv over the cross terms.  FP32 dots: the products
// are formed exactly (TwoProduct) and summed as unevaluated float pairs
// (TwoSum), so the sum carries ~2^-48 relative error without FP64 arithmetic;
// FP64 dots: plain FP64.
template <typename T>
struct CrossAcc;
template <>
struct CrossAcc<float> {
    float hi = 0.f, lo = 0.f;
    __device__ __forceinline__ void add_pair(float p, float e) {
        const float s = hi + p;
        const float bp = s - hi;
        const float err = (hi - (s - bp)) + (p - bp);
        hi = s;
        lo += err + e;
    }
    __device__ __forceinline__ void add_prod(float a, float b) {
        const float p = a * b;
        add_pair(p, fmaf(a, b, -p));
    }
    __device__ __forceinline__ void warp_reduce() {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float oh = __shfl_xor_sync(0xffffffffu, hi, o);
            const float ol = __shfl_xor_sync(0xffffffffu, lo, o);
            add_pair(oh, ol);
        }
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};
template <>
struct CrossAcc<double> {
    double hi = 0.0;
    __device__ __forceinline__ void add_pair(double p, double e) { hi += p + e; }
    __device__ __forceinline__ void add_prod(double a, double b) { hi += a * b; }
    __device__ __forceinline__ void warp_reduce() { hi = warp_sum(hi); }
    __device__ __forceinline__ double value() const { return hi; }
};

// Padded stride of a shared-memory column slice of m entries: a whole number of
// 16-byte groups, and an odd number of them, so that eight threads reading
// eight consecutive columns with 16-byte loads hit distinct banks.
template <typename T>
__host__ __device__ __forceinline__ int64_t slice_stride(int64_t m) {
    constexpr int64_t VW = 16 / sizeof(T);
    int64_t q = (m + VW - 1) / VW;
    if ((q & 1) == 0) ++q;
    return q * VW;
}

template <typename T>
__host__ __device__ __forceinline__ size_t fixed_smem_bytes() {
    return sizeof(T) * (4 * (ACA_CAP + 1) + 2 * ACA_CAP) + 16;
}

template <typename T, int NPT>
__global__ void __launch_bounds__(CT, 1)
    aca_cluster_kernel(const double *__restrict__ A, int64_t lda, int sym, const AcaBlockDesc *__restrict__ blocks,
                       double tol2, int kcs, int *status) {
    cg::cluster_group cl = cg::this_cluster();
    const int CL = (int)cl.num_blocks();
    const int c = (int)cl.block_rank();
    const AcaBlockDesc B = blocks[blockIdx.x / CL];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int VW = 16 / sizeof(T);
    const int64_t m = B.m, nc = B.nc, ld = B.ld;
    const int64_t mr = (m + CL - 1) / CL, nr = (nc + CL - 1) / CL;
    const int64_t smr = slice_stride<T>(mr), snr = slice_stride<T>(nr);
    const int64_t i0 = std::min<int64_t>(m, c * mr), i1 = std::min<int64_t>(m, i0 + mr);
    const int64_t j0 = std::min<int64_t>(nc, c * nr), j1 = std::min<int64_t>(nc, j0 + nr);
    const int64_t mn = m < nc ? m : nc;
    const int kmax = (int)(B.cap < mn ? B.cap : mn);
    T *Ug = reinterpret_cast<T *>(B.U) + B.r0;   // Ug[l * ld + i], i block-local row
    T *Vg = reinterpret_cast<T *>(B.V) + B.c0;   // Vg[l * ld + j]

    // shared memory: candidate slots, partial dots, the pivot row/column of U/V,
    // the U and V slices, the used-row flags
    extern __shared__ __align__(16) unsigned char smem[];
    T *dots = reinterpret_cast<T *>(smem);                                         // [2][2 (ACA_CAP + 1)]
    T *pu = dots + 4 * (ACA_CAP + 1);                                              // U(i_k, 0..k-1)
    T *pv = pu + ACA_CAP;                                                          // V(j_k, 0..k-1)
    T *Us = pv + ACA_CAP;                                                          // [kcs][smr]
    T *Vs = Us + (size_t)kcs * smr;                                                // [kcs][snr]
    unsigned char *used = reinterpret_cast<unsigned char *>(Vs + (size_t)kcs * snr);   // [mr]
    __shared__ Cand<T> slots[2][3][MAX_CL];   // [parity][row, col, free row][posting CTA]
    __shared__ Cand<T> red[2][CW];
    __shared__ float xr_hi[CW], xr_lo[CW];
    __shared__ double xr_d[CW];
    __shared__ double s_norm2, s_uu, s_vv;
    __shared__ int s_stop;

    for (int64_t e = tid; e < (int64_t)kcs * (smr + snr); e += CT) Us[e] = T(0);
    for (int64_t q = tid; q < mr; q += CT) used[q] = 0;
    if (tid == 0) {
        s_norm2 = 0.0;
        s_stop = 0;
    }

    // A entries of the next row pass and of the current column pass, loaded into
    // registers as soon as the pivot index is known (thread tid owns the slice
    // entries tid + t CT, t < NPT)
    double arow_pf[NPT], acol_pf[NPT];
    auto load_row = [&](int ir) {
        const double *arow = A + (B.r0 + ir) * lda + B.c0;
#pragma unroll
        for (int t = 0; t < NPT; ++t) {
            const int64_t j = j0 + tid + (int64_t)t * CT;
            arow_pf[t] = (j < j1) ? __ldg(arow + j) : 0.0;
        }
    };
    auto load_col = [&](int jc) {
        const double *acol;
        int64_t astr;
        if (sym) {
            acol = A + (B.c0 + jc) * lda + B.r0;
            astr = 1;
        } else {
            acol = A + B.r0 * lda + B.c0 + jc;
            astr = lda;
        }
#pragma unroll
        for (int t = 0; t < NPT; ++t) {
            const int64_t q = i0 + tid + (int64_t)t * CT;
            acol_pf[t] = (q < i1) ? __ldg(acol + q * astr) : 0.0;
        }
    };
    // U(ir, l), l < kk: from the shared-memory slice of the CTA that owns row ir
    auto gather_pu = [&](int ir, int kk) {
        const int co = (int)(ir / mr);
        const int64_t li = ir - (int64_t)co * mr;
        const T *Uo = cl.map_shared_rank(Us, co);
        for (int l = tid; l < kk; l += CT) pu[l] = (l < kcs) ? Uo[(size_t)l * smr + li] : Ug[(int64_t)l * ld + ir];
    };
    // The same gathers split into a register-staged load, issued as soon as the
    // index is known, and the store to shared memory where the values are due,
    // so that the remote (DSMEM) latency overlaps other work.
    constexpr int GR = ACA_CAP / CT;
    T greg[GR];
    auto pu_load = [&](int ir, int kk) {
        const int co = (int)(ir / mr);
        const int64_t li = ir - (int64_t)co * mr;
        const T *Uo = cl.map_shared_rank(Us, co);
#pragma unroll
        for (int t = 0; t < GR; ++t) {
            const int l = tid + t * CT;
            greg[t] = (l < kk) ? ((l < kcs) ? Uo[(size_t)l * smr + li] : Ug[(int64_t)l * ld + ir]) : T(0);
        }
    };
    auto pv_load = [&](int jc, int kk) {
        const int cv = (int)(jc / nr);
        const int64_t lj = jc - (int64_t)cv * nr;
        const T *Vo = cl.map_shared_rank(Vs, cv);
#pragma unroll
        for (int t = 0; t < GR; ++t) {
            const int l = tid + t * CT;
            greg[t] = (l < kk) ? ((l < kcs) ? Vo[(size_t)l * snr + lj] : Vg[(int64_t)l * ld + jc]) : T(0);
        }
    };
    auto greg_store = [&](T *dst, int kk) {
#pragma unroll
        for (int t = 0; t < GR; ++t) {
            const int l = tid + t * CT;
            if (l < kk) dst[l] = greg[t];
        }
    };
    load_row(0);
    __syncthreads();
    cl.sync();

    // The stop test of a step is made by the upper half of the warps while the
    // lower half already runs the next step's row pass, when every column of
    // the CTA's slice is owned by the lower half (the row pass writes nothing
    // outside registers; the decision is read at its first barrier).
    const bool split = (NPT == 1) && (nr <= CT / 2);
    bool deferred = false;
    int i_next = 0;
    int k = 0;
    while (k < kmax) {
        const int par = k & 1;
        const int i = i_next;
        // ---- row pass on own columns -> v_k (unscaled, kept in registers); U(i_k, :)
        // was gathered into pu at the end of the previous step
        const int kin = k < kcs ? k : kcs;
        // the NPT entries of a thread advance together through l (independent
        // chains in flight; each entry's own terms still in the order l = 0..k-1)
        T rreg[NPT];
        int jl[NPT];   // slice-local (below NPT CT)
        bool jok[NPT];
#pragma unroll
        for (int t = 0; t < NPT; ++t) {
            const int64_t j = j0 + tid + (int64_t)t * CT;
            jok[t] = j < j1;
            jl[t] = jok[t] ? (int)(j - j0) : 0;   // a slice entry that exists, for the idle lanes
            rreg[t] = jok[t] ? dev::from_double<T>(arow_pf[t]) : T(0);
        }
        if (jok[0]) {   // (a thread that owns no column skips the pass)
            int l = 0;
            if constexpr (sizeof(T) == 4) {   // U(i_k, l..l+3) in one 16-byte broadcast load
#pragma unroll 2
                for (; l + 4 <= kin; l += 4) {
                    const float4 p4 = *reinterpret_cast<const float4 *>(pu + l);
#pragma unroll
                    for (int t = 0; t < NPT; ++t) {
                        const T *vs = Vs + (size_t)l * snr + jl[t];
                        rreg[t] = dev::sub_rn(rreg[t], dev::mul_rn(p4.x, vs[0]));
                        rreg[t] = dev::sub_rn(rreg[t], dev::mul_rn(p4.y, vs[snr]));
                        rreg[t] = dev::sub_rn(rreg[t], dev::mul_rn(p4.z, vs[2 * snr]));
                        rreg[t] = dev::sub_rn(rreg[t], dev::mul_rn(p4.w, vs[3 * snr]));
                    }
                }
            }
#pragma unroll(NPT == 1 ? 8 : (NPT >= 8 ? 2 : 4))
            for (; l < kin; ++l) {
                const T p = pu[l];
#pragma unroll
                for (int t = 0; t < NPT; ++t)
                    rreg[t] = dev::sub_rn(rreg[t], dev::mul_rn(p, Vs[(size_t)l * snr + jl[t]]));
            }
#pragma unroll(NPT >= 8 ? 2 : 4)
            for (; l < k; ++l) {
                const T p = pu[l];
                const T *vg = Vg + (int64_t)l * ld + j0;
#pragma unroll
                for (int t = 0; t < NPT; ++t)
                    if (jok[t]) rreg[t] = dev::sub_rn(rreg[t], dev::mul_rn(p, vg[jl[t]]));
            }
        }
        T ba = T(-1), bv = T(0);
        int bi = INT_MAX;
#pragma unroll
        for (int t = 0; t < NPT; ++t) {
            if (jok[t]) {
                const T r = rreg[t];
                const T a = fabs(r);
                if (a != a) atomicOr(status, ST_NONFINITE);
                if (a > ba) {
                    ba = a;
                    bi = (int)(j0 + jl[t]);
                    bv = r;
                }
            }
        }
        const Cand<T> cr = cta_argmax(ba, bi, bv, red[0]);
        if (deferred) {   // the previous step's stop test, made meanwhile by the upper warps
            deferred = false;
            if (s_stop) break;
        }
        post_cand(cl, &slots[par][0][0], c, CL, cr);
        cl.sync();
        const Cand<T> best = best_of_slots(&slots[par][0][0], CL);
        const int jk = best.idx;
        const T piv = best.v;
        const bool have = !(jk == INT_MAX || piv == T(0));
        if (have) {
            load_col(jk);
            pv_load(jk, k);   // V(j_k, l), l < k: written in earlier steps by the owner of column j_k
        }
        // the owner of row i marks it used
        if (i >= i0 && i < i1 && tid == 0) used[i - i0] = 1;
        if (!have) {
            // exhausted row: the lowest unused row of the whole block, if any
            __syncthreads();
            T fa = T(-1);
            int fi = INT_MAX;
            for (int64_t q = i0 + tid; q < i1; q += CT)
                if (!used[q - i0] && fa < T(0)) {
                    fa = T(0);
                    fi = (int)q;
                }
            const Cand<T> cf = cta_argmax(fa, fi, T(0), red[1]);
            post_cand(cl, &slots[par][2][0], c, CL, cf);
            cl.sync();
            const Cand<T> bf = best_of_slots(&slots[par][2][0], CL);
            if (bf.a < T(0)) break;
            load_row(bf.idx);
            gather_pu(bf.idx, k);
            i_next = bf.idx;
            __syncthreads();
            continue;
        }
        // ---- v_k = r / r(j_k) on own columns
#pragma unroll
        for (int t = 0; t < NPT; ++t) {
            const int64_t j = j0 + tid + (int64_t)t * CT;
            if (j < j1) {
                const T v = dev::div_rn(rreg[t], piv);
                if (k < kcs) Vs[(size_t)k * snr + (j - j0)] = v;
                Vg[(int64_t)k * ld + j] = v;
            }
        }
        greg_store(pv, k);
        __syncthreads();
        // ---- column pass on own rows -> u_k
        T ureg[NPT];
        int ql[NPT];
        bool qok[NPT];
#pragma unroll
        for (int t = 0; t < NPT; ++t) {
            const int64_t q = i0 + tid + (int64_t)t * CT;
            qok[t] = q < i1;
            ql[t] = qok[t] ? (int)(q - i0) : 0;
            ureg[t] = qok[t] ? dev::from_double<T>(acol_pf[t]) : T(0);
        }
        if (qok[0]) {
            int l = 0;
            if constexpr (sizeof(T) == 4) {   // V(j_k, l..l+3) in one 16-byte broadcast load
#pragma unroll 2
                for (; l + 4 <= kin; l += 4) {
                    const float4 p4 = *reinterpret_cast<const float4 *>(pv + l);
#pragma unroll
                    for (int t = 0; t < NPT; ++t) {
                        const T *us = Us + (size_t)l * smr + ql[t];
                        ureg[t] = dev::sub_rn(ureg[t], dev::mul_rn(p4.x, us[0]));
                        ureg[t] = dev::sub_rn(ureg[t], dev::mul_rn(p4.y, us[smr]));
                        ureg[t] = dev::sub_rn(ureg[t], dev::mul_rn(p4.z, us[2 * smr]));
                        ureg[t] = dev::sub_rn(ureg[t], dev::mul_rn(p4.w, us[3 * smr]));
                    }
                }
            }
#pragma unroll(NPT == 1 ? 8 : (NPT >= 8 ? 2 : 4))
            for (; l < kin; ++l) {
                const T p = pv[l];
#pragma unroll
                for (int t = 0; t < NPT; ++t)
                    ureg[t] = dev::sub_rn(ureg[t], dev::mul_rn(p, Us[(size_t)l * smr + ql[t]]));
            }
#pragma unroll(NPT >= 8 ? 2 : 4)
            for (; l < k; ++l) {
                const T p = pv[l];
                const T *ug = Ug + (int64_t)l * ld + i0;
#pragma unroll
                for (int t = 0; t < NPT; ++t)
                    if (qok[t]) ureg[t] = dev::sub_rn(ureg[t], dev::mul_rn(p, ug[ql[t]]));
            }
        }
        T ca = T(-1), cvv = T(0);
        int ci = INT_MAX;
#pragma unroll
        for (int t = 0; t < NPT; ++t) {
            if (qok[t]) {
                const int64_t q = i0 + ql[t];
                const T u = ureg[t];
                if (k < kcs) Us[(size_t)k * smr + ql[t]] = u;
                Ug[(int64_t)k * ld + q] = u;
                if (u != u) atomicOr(status, ST_NONFINITE);
                if (!used[ql[t]]) {
                    const T a = fabs(u);
                    if (a > ca) {
                        ca = a;
                        ci = (int)q;
                        cvv = u;
                    }
                }
            }
        }
        // (its barrier also publishes column k of the U slice to the dots below)
        const Cand<T> cc = cta_argmax(ca, ci, cvv, red[1]);
        // ---- partial dots u_k.u_l and v_k.v_l (l = 0..k) over own slices
        T *dp = dots + (size_t)par * 2 * (ACA_CAP + 1);
        if (k < kcs) {
            const int nvr = (int)((i1 - i0 + VW - 1) / VW), nvc = (int)((j1 - j0 + VW - 1) / VW);
            for (int it = tid; it < 2 * (k + 1); it += CT) {
                const bool isu = it <= k;
                const int l = isu ? it : it - (k + 1);
                const T d = isu ? vdot(Us + (size_t)l * smr, Us + (size_t)k * smr, nvr)
                                : vdot(Vs + (size_t)l * snr, Vs + (size_t)k * snr, nvc);
                dp[(isu ? 0 : ACA_CAP + 1) + l] = d;
            }
        } else {
            // LG columns l per warp at a time (independent chains; each dot
            // still lane-strided in ascending q, then summed over the warp)
            constexpr int LG = 4;
            for (int l0 = warp * LG; l0 <= k; l0 += CW * LG) {
                T su[LG], sv[LG];
                const T *ul[LG], *vl[LG];
#pragma unroll
                for (int g = 0; g < LG; ++g) {
                    su[g] = sv[g] = T(0);
                    const int l = l0 + g <= k ? l0 + g : k;   // a column that exists, for the idle chains
                    ul[g] = Ug + (int64_t)l * ld;
                    vl[g] = Vg + (int64_t)l * ld;
                }
                const T *uk = Ug + (int64_t)k * ld, *vk = Vg + (int64_t)k * ld;
                for (int64_t q = i0 + lane; q < i1; q += 32) {
                    const T b = uk[q];
#pragma unroll
                    for (int g = 0; g < LG; ++g) su[g] = fma(ul[g][q], b, su[g]);
                }
                for (int64_t j = j0 + lane; j < j1; j += 32) {
                    const T b = vk[j];
#pragma unroll
                    for (int g = 0; g < LG; ++g) sv[g] = fma(vl[g][j], b, sv[g]);
                }
#pragma unroll
                for (int g = 0; g < LG; ++g) {
                    const T tu = warp_sum(su[g]), tv = warp_sum(sv[g]);
                    if (lane == 0 && l0 + g <= k) {
                        dp[l0 + g] = tu;
                        dp[ACA_CAP + 1 + l0 + g] = tv;
                    }
                }
            }
        }
        post_cand(cl, &slots[par][1][0], c, CL, cc);
        cl.sync();
        // ---- cluster-wide: next row, dot products (rank order), stop decision
        const Cand<T> bc = best_of_slots(&slots[par][1][0], CL);
        if (bc.a >= T(0)) {
            load_row(bc.idx);          // the next pivot row and its U entries, while the stop test is made
            pu_load(bc.idx, k + 1);
        }
        // dot products summed over the cluster in rank order, the cross term, the
        // norm recurrence and the stop decision of step k, by warps [w0, w0 + nw)
        auto stop_test = [&](int w0, int nw) {
            const int t0 = 32 * w0, nt = 32 * nw;
            CrossAcc<T> xacc;
            for (int l = tid - t0; l <= k; l += nt) {
                T pu_[MAX_CL], pv_[MAX_CL];
#pragma unroll
                for (int q = 0; q < MAX_CL; ++q)
                    if (q < CL) {
                        const T *rp = cl.map_shared_rank(dots, q) + (size_t)par * 2 * (ACA_CAP + 1);
                        pu_[q] = rp[l];
                        pv_[q] = rp[ACA_CAP + 1 + l];
                    }
                T su = T(0), sv = T(0);
#pragma unroll
                for (int q = 0; q < MAX_CL; ++q)
                    if (q < CL) {
                        su += pu_[q];
                        sv += pv_[q];
                    }
                if (l < k) {
                    xacc.add_prod(su, sv);
                } else {
                    s_uu = (double)su;
                    s_vv = (double)sv;
                }
            }
            xacc.warp_reduce();
            if (lane == 0) {
                if constexpr (sizeof(T) == 4) {
                    xr_hi[warp - w0] = (float)xacc.hi;
                    xr_lo[warp - w0] = (float)xacc.lo;
                } else {
                    xr_d[warp - w0] = (double)xacc.hi;
                }
            }
            if (nw == CW)
                __syncthreads();
            else
                asm volatile("bar.sync 1, %0;" ::"r"(nt) : "memory");
            if (tid == t0) {
                CrossAcc<T> tot;
                for (int w = 0; w < nw; ++w) {
                    if constexpr (sizeof(T) == 4)
                        tot.add_pair(xr_hi[w], xr_lo[w]);
                    else
                        tot.add_pair(xr_d[w], 0.0);
                }
                const double cross = tot.value(), uu = s_uu, vv = s_vv;
                // ||S_k||^2 = ||S_{k-1}||^2 + 2 cross + ||u_k||^2 ||v_k||^2, evaluated left to right
                s_norm2 = __dadd_rn(__dadd_rn(s_norm2, __dmul_rn(2.0, cross)), __dmul_rn(uu, vv));
                if (c == 0) {
                    B.prow[k] = i;
                    B.pcol[k] = jk;
                }
                const double nrm = s_norm2 > 0.0 ? s_norm2 : 0.0;
                int stop = (__dmul_rn(uu, vv) <= __dmul_rn(tol2, nrm));   // ||u|| ||v|| <= tol ||S||, squared
                if ((int64_t)(k + 1) >= mn) stop = 1;
                if (bc.a < T(0)) stop = 1;   // every row used
                s_stop = stop;
            }
        };
        const bool more = bc.a >= T(0) && (int64_t)(k + 1) < mn && k + 1 < kmax;
        if (split && more) {
            greg_store(pu, k + 1);
            __syncthreads();   // U(i_{k+1}, :) in place for the next row pass
            if (warp >= CW / 2) stop_test(CW / 2, CW / 2);
            i_next = bc.idx;
            ++k;
            deferred = true;
            continue;
        }
        stop_test(0, CW);
        if (bc.a >= T(0)) greg_store(pu, k + 1);
        __syncthreads();
        i_next = bc.idx;
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

template <typename T, int NPT>
hodlr_status launch_level_npt(hodlr_ctx *c, const double *A, int64_t lda, int sym, const AcaBlockDesc *d_blocks,
                              int nblocks, int CL, int64_t mr, int64_t nr, double tol, cudaStream_t s) {
    const int64_t smr = slice_stride<T>(mr), snr = slice_stride<T>(nr);
    const size_t fixed = fixed_smem_bytes<T>() + (size_t)mr + 16;
    int kcs = 0;
    if (fixed < SMEM_BUDGET)
        kcs = (int)std::min<size_t>(ACA_CAP, (SMEM_BUDGET - fixed) / ((smr + snr) * sizeof(T)));
    const size_t sm = fixed + (size_t)kcs * (smr + snr) * sizeof(T);
    HODLR_TRY_CUDA(cudaFuncSetAttribute(aca_cluster_kernel<T, NPT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    if (CL > 8)
        HODLR_TRY_CUDA(cudaFuncSetAttribute(aca_cluster_kernel<T, NPT>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
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
    {
        ProfScope ps("aca_cluster_kernel", cfg.stream);
        HODLR_TRY_CUDA(
            cudaLaunchKernelEx(&cfg, aca_cluster_kernel<T, NPT>, A, lda, sym, d_blocks, tol * tol, kcs, c->d_status));
    }
    note_launch();
    return HODLR_OK;
}

// Slices of up to NPT * CT rows (columns) per CTA: every thread keeps NPT
// entries of the row and column passes in registers.
template <typename T>
hodlr_status launch_level(hodlr_ctx *c, const double *A, int64_t lda, int sym, const AcaBlockDesc *d_blocks,
                          int nblocks, int CL, int64_t mr, int64_t nr, double tol, cudaStream_t s) {
    const int64_t w = std::max(mr, nr);
    if (w <= CT) return launch_level_npt<T, 1>(c, A, lda, sym, d_blocks, nblocks, CL, mr, nr, tol, s);
    if (w <= 2 * CT) return launch_level_npt<T, 2>(c, A, lda, sym, d_blocks, nblocks, CL, mr, nr, tol, s);
    if (w <= 4 * CT) return launch_level_npt<T, 4>(c, A, lda, sym, d_blocks, nblocks, CL, mr, nr, tol, s);
    if (w <= 8 * CT) return launch_level_npt<T, 8>(c, A, lda, sym, d_blocks, nblocks, CL, mr, nr, tol, s);
    set_error("ACA: off-diagonal blocks of %lld rows exceed the %d-row limit of one cluster",
              (long long)w * CL, 8 * CT * CL);
    return HODLR_INVALID_ARG;
}

}  // namespace

hodlr_status launch_aca_levels(hodlr_ctx *c, const double *A, int64_t lda, int sym, int cprec,
                               const AcaBlockDesc *d_blocks, const std::vector<int> &level_first,
                               const std::vector<int64_t> &level_maxdim, double tol, cudaStream_t s,
                               std::vector<cudaEvent_t> &done, const std::function<hodlr_status()> &after_first) {
    // level_first[l] .. level_first[l+1]: the blocks of level l + 1 (all of one size class)
    const int nlev = (int)level_first.size() - 1;
    done.assign(nlev, nullptr);
    cudaEvent_t fork;
    HODLR_TRY_CUDA(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
    HODLR_TRY_CUDA(cudaEventRecord(fork, s));
    // Entries per CTA of a block's cluster: 128, unless that puts more than
    // four full-SM CTAs per SM in flight over all levels (the levels then wait
    // for one another in waves); 512 then (on the n = 32768 front: 1448 CTAs
    // become 480 and the build takes 9.0 ms instead of 11.5; on the n = 4096
    // front, 160 CTAs, 128 stays faster: 1.6 ms against 2.6)
    auto cluster_of = [](int64_t dim, int64_t per) {
        int CL = 1;
        while (CL < 16 && dim > (int64_t)CL * per) CL *= 2;
        return CL;
    };
    int64_t ctas = 0;
    for (int l = 0; l < nlev; ++l)
        ctas += (int64_t)(level_first[l + 1] - level_first[l]) * cluster_of(level_maxdim[l], 128);
    const int64_t per_cta = ctas > 4 * (int64_t)std::max(1, c->num_sms) ? 512 : 128;
    hodlr_status rs = HODLR_OK;
    for (int l = 0; l < nlev && rs == HODLR_OK; ++l) {
        const int nb = level_first[l + 1] - level_first[l];
        cudaStream_t ls = c->side[l % HODLR_SIDE_STREAMS];
        if (cudaStreamWaitEvent(ls, fork, 0) != cudaSuccess) {
            rs = HODLR_CUDA_ERROR;
            break;
        }
        if (nb > 0) {
            const int64_t dim = level_maxdim[l];
            const int CL = cluster_of(dim, per_cta);
            const int64_t mr = (dim + CL - 1) / CL;
            const AcaBlockDesc *db = d_blocks + level_first[l];
            rs = (cprec == HODLR_FP64) ? launch_level<double>(c, A, lda, sym, db, nb, CL, mr, mr, tol, ls)
                                       : launch_level<float>(c, A, lda, sym, db, nb, CL, mr, mr, tol, ls);
        }
        cudaEventCreate(&done[l]);   // timed: the build reports the compression time
        cudaEventRecord(done[l], ls);
        if (l == 0 && rs == HODLR_OK && after_first) rs = after_first();
    }
    cudaEventDestroy(fork);
    return rs;
}

}  // namespace hodlr
