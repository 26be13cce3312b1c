// Boundary-distance low-rank approximation, BDLR (Sec. 5.3, eq. Ahat):
//   rows R = the node, columns C = its sibling.  The boundary of R is the set
//   of its vertices with a graph edge into C; d = breadth-first distance from
//   that boundary inside the subgraph induced on R (likewise for C).
//   I = {v in R : d(v) <= depth}, J = {w in C : d(w) <= depth}, each sorted by
//   (d, index).  A^ = A(I, J) = P^-1 L U Q^-1 by full-pivoting LU, stopped
//   before the first pivot with |p_k| < eps |p_1| (or at the rank cap);
//   U_block = A(R, J_r) U11^-1,  V_block^T = L11^-1 A(I_r, C).
// The index lists are integer work done once on the host; the gather, the LU
// and the two triangular solves run on the device, one block per CTA (LU) or
// per row/column chunk (solves).  The LU forms every trailing update with a
// separate round-to-nearest multiply and subtract and takes the pivot with the
// lowest row (then column) among equal magnitudes, so its pivot sequence is
// reproducible.
#include <algorithm>
#include <climits>
#include <cmath>
#include <vector>

#include "internal.cuh"

namespace hodlr {
namespace {

struct BdlrDesc {
    const int32_t *I;   // global row indices, sorted by (d, index)
    const int32_t *J;   // global col indices
    int nI, nJ;
    void *Ahat;         // nI x nJ column-major, ld nI
    int32_t *lrow;      // nI: row order after pivoting (positions in I)
    int32_t *lcol;      // nJ
    int64_t r0, m, c0, nc;
    int64_t ld;
    void *U;
    void *V;
    int cap;
    int32_t *rank;
    int32_t *prow;
    int32_t *pcol;
    int32_t *cap_hit;
};

constexpr int LU_THREADS = 1024;

template <typename T>
__global__ void __launch_bounds__(LU_THREADS, 1)
    bdlr_lu_kernel(const double *__restrict__ A, int64_t lda, const BdlrDesc *__restrict__ descs, double eps,
                   int *status) {
    const BdlrDesc d = descs[blockIdx.x];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nI = d.nI, nJ = d.nJ;
    T *Ah = reinterpret_cast<T *>(d.Ahat);
    __shared__ T red_v[LU_THREADS / 32];
    __shared__ long long red_i[LU_THREADS / 32];
    __shared__ double s_p1;
    __shared__ int s_stop;
    for (int64_t e = tid; e < (int64_t)nI * nJ; e += LU_THREADS) {
        const int i = (int)(e % nI), j = (int)(e / nI);
        const T v = dev::from_double<T>(A[(int64_t)d.I[i] * lda + d.J[j]]);
        if (v != v) atomicOr(status, ST_NONFINITE);
        Ah[e] = v;
    }
    for (int i = tid; i < nI; i += LU_THREADS) d.lrow[i] = i;
    for (int j = tid; j < nJ; j += LU_THREADS) d.lcol[j] = j;
    if (tid == 0) {
        s_p1 = 0.0;
        s_stop = 0;
    }
    __syncthreads();
    const int kmax = min(min(nI, nJ), d.cap);
    int k = 0;
    for (; k < kmax; ++k) {
        // argmax |A^(i,j)| over the trailing block; ties -> lowest row, then column
        T bv = T(-1);
        long long bi = LLONG_MAX;
        const int rows = nI - k, cols = nJ - k;
        for (int64_t e = tid; e < (int64_t)rows * cols; e += LU_THREADS) {
            const int i = k + (int)(e % rows), j = k + (int)(e / rows);
            const T a = fabs(Ah[i + (int64_t)j * nI]);
            const long long key = (long long)i * nJ + j;   // row-major order
            if (a > bv || (a == bv && key < bi)) {
                bv = a;
                bi = key;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            T ov = __shfl_down_sync(0xffffffffu, bv, o);
            long long oi = __shfl_down_sync(0xffffffffu, bi, o);
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
            const double p = (double)red_v[0];
            if (k == 0) s_p1 = p;
            s_stop = (!(p > 0.0) || p < eps * s_p1) ? 1 : 0;
        }
        __syncthreads();
        if (s_stop) break;
        const int pi = (int)(red_i[0] / nJ), pj = (int)(red_i[0] % nJ);
        if (pi != k) {
            for (int j = tid; j < nJ; j += LU_THREADS) {
                T t = Ah[k + (int64_t)j * nI];
                Ah[k + (int64_t)j * nI] = Ah[pi + (int64_t)j * nI];
                Ah[pi + (int64_t)j * nI] = t;
            }
            if (tid == 0) {
                int t = d.lrow[k];
                d.lrow[k] = d.lrow[pi];
                d.lrow[pi] = t;
            }
        }
        __syncthreads();
        if (pj != k) {
            for (int i = tid; i < nI; i += LU_THREADS) {
                T t = Ah[i + (int64_t)k * nI];
                Ah[i + (int64_t)k * nI] = Ah[i + (int64_t)pj * nI];
                Ah[i + (int64_t)pj * nI] = t;
            }
            if (tid == 0) {
                int t = d.lcol[k];
                d.lcol[k] = d.lcol[pj];
                d.lcol[pj] = t;
            }
        }
        __syncthreads();
        const T piv = Ah[k + (int64_t)k * nI];
        for (int i = k + 1 + tid; i < nI; i += LU_THREADS)
            Ah[i + (int64_t)k * nI] = dev::div_rn(Ah[i + (int64_t)k * nI], piv);
        __syncthreads();
        const int r2 = nI - k - 1, c2 = nJ - k - 1;
        for (int64_t e = tid; e < (int64_t)r2 * c2; e += LU_THREADS) {
            const int i = k + 1 + (int)(e % r2), j = k + 1 + (int)(e / r2);
            Ah[i + (int64_t)j * nI] =
                dev::sub_rn(Ah[i + (int64_t)j * nI], dev::mul_rn(Ah[i + (int64_t)k * nI], Ah[k + (int64_t)j * nI]));
        }
        __syncthreads();
    }
    if (tid == 0) {
        *d.rank = k;
        *d.cap_hit = (k == d.cap && k < min(nI, nJ)) ? 1 : 0;
    }
    for (int t = tid; t < k; t += LU_THREADS) {
        d.prow[t] = d.I[d.lrow[t]] - (int)d.r0;
        d.pcol[t] = d.J[d.lcol[t]] - (int)d.c0;
    }
}

// U(R rows, 0:r) = A(R, J_r) U11^-1 : one thread per row, x U11 = c by columns.
template <typename T>
__global__ void bdlr_u_kernel(const double *__restrict__ A, int64_t lda, const BdlrDesc *__restrict__ descs) {
    const BdlrDesc d = descs[blockIdx.y];
    const int r = *d.rank;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= d.m || r == 0) return;
    const T *Ah = reinterpret_cast<const T *>(d.Ahat);
    T *U = reinterpret_cast<T *>(d.U) + d.r0 + i;
    const double *arow = A + (d.r0 + i) * lda;
    for (int j = 0; j < r; ++j) {
        T acc = dev::from_double<T>(arow[d.J[d.lcol[j]]]);
        for (int t = 0; t < j; ++t) acc -= U[(int64_t)t * d.ld] * Ah[t + (int64_t)j * d.nI];
        U[(int64_t)j * d.ld] = acc / Ah[j + (int64_t)j * d.nI];
    }
}

// V(C rows, 0:r) = (L11^-1 A(I_r, C))^T : one thread per column of the block.
template <typename T>
__global__ void bdlr_v_kernel(const double *__restrict__ A, int64_t lda, const BdlrDesc *__restrict__ descs) {
    const BdlrDesc d = descs[blockIdx.y];
    const int r = *d.rank;
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= d.nc || r == 0) return;
    const T *Ah = reinterpret_cast<const T *>(d.Ahat);
    T *V = reinterpret_cast<T *>(d.V) + d.c0 + j;
    for (int k = 0; k < r; ++k) {
        T acc = dev::from_double<T>(A[(int64_t)d.I[d.lrow[k]] * lda + d.c0 + j]);
        for (int t = 0; t < k; ++t) acc -= Ah[k + (int64_t)t * d.nI] * V[(int64_t)t * d.ld];
        V[(int64_t)k * d.ld] = acc;
    }
}

// Boundary-distance selection of one side: vertices of [o0,o1) with d <= depth,
// sorted by (d, index); boundary = vertices with an edge into [t0,t1).  ring
// (optional): the vertices at distance exactly depth + 1, by index.
void select_side(const hodlr_graph *g, int64_t o0, int64_t o1, int64_t t0, int64_t t1, int depth,
                 std::vector<int32_t> &out, std::vector<int32_t> *ring = nullptr) {
    const int64_t m = o1 - o0;
    std::vector<int> dist(m, -1);
    std::vector<int32_t> frontier, next;
    for (int64_t v = o0; v < o1; ++v) {
        for (int32_t e = g->rowptr[v]; e < g->rowptr[v + 1]; ++e) {
            const int32_t w = g->colind[e];
            if (w >= t0 && w < t1) {
                dist[v - o0] = 0;
                frontier.push_back((int32_t)v);
                break;
            }
        }
    }
    int dd = 0;
    const int reach = ring ? depth + 1 : depth;
    while (!frontier.empty() && dd < reach) {
        next.clear();
        for (int32_t v : frontier)
            for (int32_t e = g->rowptr[v]; e < g->rowptr[v + 1]; ++e) {
                const int32_t w = g->colind[e];
                if (w >= o0 && w < o1 && dist[w - o0] < 0) {
                    dist[w - o0] = dd + 1;
                    next.push_back(w);
                }
            }
        frontier.swap(next);
        ++dd;
    }
    out.clear();
    for (int q = 0; q <= depth; ++q)
        for (int64_t v = o0; v < o1; ++v)
            if (dist[v - o0] == q) out.push_back((int32_t)v);
    if (ring) {
        ring->clear();
        for (int64_t v = o0; v < o1; ++v)
            if (dist[v - o0] == depth + 1) ring->push_back((int32_t)v);
    }
}

// The held-out error of the adaptive scheme (Sec. 5.3), for one block per
// blockIdx.y: vector q of the sample list (rows: the held-out ring Hr, then the
// selected I; columns: the ring Hc, then J) -- a row h contributes its squared
// residual A(h, C) - U(h, :) V(C, :)^T to num when held out, and its squared
// entries to den always; likewise a column.  FP64 sums, one CTA per vector.
struct HeldDesc {
    const int32_t *vec;    // nHr + nI rows, then nHc + nJ columns (global indices)
    int nHr, nI, nHc, nJ;
    int64_t r0, m, c0, nc, ld;
    const void *U, *V;
    const int32_t *rank;
    double *num, *den;
};

template <typename T>
__global__ void bdlr_heldout_kernel(const double *__restrict__ A, int64_t lda, const HeldDesc *__restrict__ descs) {
    const HeldDesc d = descs[blockIdx.y];
    const int q = blockIdx.x;
    const int nrow = d.nHr + d.nI, ntot = nrow + d.nHc + d.nJ;
    if (q >= ntot) return;
    const bool is_row = q < nrow;
    const bool held = is_row ? q < d.nHr : (q - nrow) < d.nHc;
    const int64_t h = d.vec[q];
    const int r = *d.rank;
    const T *U = reinterpret_cast<const T *>(d.U);
    const T *V = reinterpret_cast<const T *>(d.V);
    double sr = 0.0, sa = 0.0;
    const int64_t len = is_row ? d.nc : d.m;
    for (int64_t t = threadIdx.x; t < len; t += blockDim.x) {
        const int64_t row = is_row ? h : d.r0 + t, col = is_row ? d.c0 + t : h;
        const double a = A[row * lda + col];
        sa += a * a;
        if (held) {
            double uv = 0.0;
            for (int k = 0; k < r; ++k) uv += (double)U[row + (int64_t)k * d.ld] * (double)V[col + (int64_t)k * d.ld];
            sr += (a - uv) * (a - uv);
        }
    }
    __shared__ double red[2][32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sr += __shfl_xor_sync(0xffffffffu, sr, o);
        sa += __shfl_xor_sync(0xffffffffu, sa, o);
    }
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = sr;
        red[1][threadIdx.x >> 5] = sa;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a0 = 0.0, a1 = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            a0 += red[0][w];
            a1 += red[1][w];
        }
        if (held) atomicAdd(d.num, a0);
        atomicAdd(d.den, a1);
    }
}

}  // namespace

namespace {

struct BdlrBlock {
    int l, i, depth;
};

// One pass of BDLR over `todo` (each block at its own depth): the index lists
// on the host, the gather, LU and triangular solves on the device; with
// `held` also the held-out error of every block (err[k], and whether it had
// any held-out row or column, ring[k]).
hodlr_status bdlr_pass(hodlr_t *h, const hodlr_graph *g, const std::vector<BdlrBlock> &todo, cudaStream_t s,
                       std::vector<void *> &Ust, std::vector<void *> &Vst, bool held, std::vector<double> &err,
                       std::vector<char> &ring) {
    hodlr_ctx *c = h->ctx;
    const int L = h->L;
    std::vector<BdlrDesc> descs;
    std::vector<int32_t> idx;                        // all I and J lists, concatenated
    std::vector<std::pair<size_t, size_t>> ij_off;   // offset of I, J per block
    std::vector<int32_t> hv;                         // held-out samples per block: Hr, I, Hc, J
    std::vector<HeldDesc> hd;
    std::vector<size_t> hv_off;
    size_t ah_elems = 0, perm_elems = 0;
    int max_vec = 0;
    std::vector<int32_t> side, sideJ, rr, rc;
    ring.assign(todo.size(), 0);
    for (const BdlrBlock &bk : todo) {
        const int l = bk.l, i = bk.i;
        const int64_t r0 = h->bounds[(size_t)i << (L - l)], r1 = h->bounds[(size_t)(i + 1) << (L - l)];
        const int sib = i ^ 1;
        const int64_t c0 = h->bounds[(size_t)sib << (L - l)], c1 = h->bounds[(size_t)(sib + 1) << (L - l)];
        BdlrDesc d{};
        const size_t oi = idx.size();
        select_side(g, r0, r1, c0, c1, bk.depth, side, held ? &rr : nullptr);
        idx.insert(idx.end(), side.begin(), side.end());
        d.nI = (int)side.size();
        const size_t oj = idx.size();
        select_side(g, c0, c1, r0, r1, bk.depth, sideJ, held ? &rc : nullptr);
        idx.insert(idx.end(), sideJ.begin(), sideJ.end());
        d.nJ = (int)sideJ.size();
        ij_off.push_back({oi, oj});
        d.r0 = r0;
        d.m = r1 - r0;
        d.c0 = c0;
        d.nc = c1 - c0;
        d.ld = h->ldn;
        d.U = Ust[l];
        d.V = Vst[l];
        d.cap = h->lv[l].cap;
        d.rank = h->d_ranks[l] + i;
        d.prow = h->piv_rows[l] + (size_t)i * h->lv[l].cap;
        d.pcol = h->piv_cols[l] + (size_t)i * h->lv[l].cap;
        ah_elems += (size_t)d.nI * d.nJ;
        perm_elems += (size_t)d.nI + d.nJ;
        descs.push_back(d);
        if (held) {
            ring[descs.size() - 1] = (!rr.empty() || !rc.empty()) ? 1 : 0;
            hv_off.push_back(hv.size());
            hv.insert(hv.end(), rr.begin(), rr.end());
            hv.insert(hv.end(), side.begin(), side.end());
            hv.insert(hv.end(), rc.begin(), rc.end());
            hv.insert(hv.end(), sideJ.begin(), sideJ.end());
            HeldDesc q{};
            q.nHr = (int)rr.size();
            q.nI = d.nI;
            q.nHc = (int)rc.size();
            q.nJ = d.nJ;
            q.r0 = r0;
            q.m = d.m;
            q.c0 = c0;
            q.nc = d.nc;
            q.ld = h->ldn;
            q.U = Ust[l];
            q.V = Vst[l];
            q.rank = d.rank;
            hd.push_back(q);
            max_vec = std::max(max_vec, q.nHr + q.nI + q.nHc + q.nJ);
        }
    }
    const size_t es = elem_size(h->cprec);
    const int nb = (int)descs.size();
    const size_t bytes = idx.size() * 4 + 256 + ah_elems * es + 256 + perm_elems * 4 + 256 + nb * sizeof(BdlrDesc) +
                         256 + nb * 4 + 256 + (held ? hv.size() * 4 + 256 + nb * sizeof(HeldDesc) + 256 +
                                                          2 * nb * sizeof(double) + 256
                                                    : 0);
    char *base = (char *)dalloc(c, bytes, s);
    if (!base) return HODLR_OUT_OF_MEMORY;
    char *p = base;
    auto carve = [&](size_t b) {
        char *q = p;
        p += (b + 255) & ~size_t(255);
        return q;
    };
    int32_t *d_idx = (int32_t *)carve(idx.size() * 4);
    char *d_ah = carve(ah_elems * es);
    int32_t *d_perm = (int32_t *)carve(perm_elems * 4);
    BdlrDesc *d_desc = (BdlrDesc *)carve(nb * sizeof(BdlrDesc));
    int32_t *d_caphit = (int32_t *)carve(nb * 4);
    int32_t *d_hv = held ? (int32_t *)carve(hv.size() * 4) : nullptr;
    HeldDesc *d_hd = held ? (HeldDesc *)carve(nb * sizeof(HeldDesc)) : nullptr;
    double *d_nd = held ? (double *)carve(2 * nb * sizeof(double)) : nullptr;
    size_t ao = 0, po = 0;
    int64_t max_rows = 0;
    for (int b = 0; b < nb; ++b) {
        BdlrDesc &d = descs[b];
        d.I = d_idx + ij_off[b].first;
        d.J = d_idx + ij_off[b].second;
        d.Ahat = d_ah + ao * es;
        ao += (size_t)d.nI * d.nJ;
        d.lrow = d_perm + po;
        po += d.nI;
        d.lcol = d_perm + po;
        po += d.nJ;
        d.cap_hit = d_caphit + b;
        max_rows = std::max(max_rows, std::max(d.m, d.nc));
        if (held) {
            hd[b].vec = d_hv + hv_off[b];
            hd[b].num = d_nd + 2 * b;
            hd[b].den = d_nd + 2 * b + 1;
        }
    }
    hodlr_status rs = HODLR_OK;
    if (cudaMemcpyAsync(d_idx, idx.data(), idx.size() * 4, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(d_desc, descs.data(), nb * sizeof(BdlrDesc), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        (held && (cudaMemcpyAsync(d_hv, hv.data(), hv.size() * 4, cudaMemcpyHostToDevice, s) != cudaSuccess ||
                  cudaMemcpyAsync(d_hd, hd.data(), nb * sizeof(HeldDesc), cudaMemcpyHostToDevice, s) != cudaSuccess ||
                  cudaMemsetAsync(d_nd, 0, 2 * nb * sizeof(double), s) != cudaSuccess))) {
        rs = HODLR_CUDA_ERROR;
    } else {
        const dim3 tgrid((unsigned)((max_rows + 127) / 128), nb);
        if (h->cprec == HODLR_FP64) {
            bdlr_lu_kernel<double><<<nb, LU_THREADS, 0, s>>>(h->A, h->lda, d_desc, h->tol, c->d_status);
            bdlr_u_kernel<double><<<tgrid, 128, 0, s>>>(h->A, h->lda, d_desc);
            bdlr_v_kernel<double><<<tgrid, 128, 0, s>>>(h->A, h->lda, d_desc);
            if (held) bdlr_heldout_kernel<double><<<dim3(max_vec, nb), 128, 0, s>>>(h->A, h->lda, d_hd);
        } else {
            bdlr_lu_kernel<float><<<nb, LU_THREADS, 0, s>>>(h->A, h->lda, d_desc, h->tol, c->d_status);
            bdlr_u_kernel<float><<<tgrid, 128, 0, s>>>(h->A, h->lda, d_desc);
            bdlr_v_kernel<float><<<tgrid, 128, 0, s>>>(h->A, h->lda, d_desc);
            if (held) bdlr_heldout_kernel<float><<<dim3(max_vec, nb), 128, 0, s>>>(h->A, h->lda, d_hd);
        }
        note_launch(held ? 4 : 3);
        if (cudaGetLastError() != cudaSuccess) rs = HODLR_CUDA_ERROR;
    }
    std::vector<int32_t> hc(nb);
    std::vector<double> nd(held ? 2 * nb : 0);
    cudaMemcpyAsync(hc.data(), d_caphit, nb * 4, cudaMemcpyDeviceToHost, s);
    if (held) cudaMemcpyAsync(nd.data(), d_nd, 2 * nb * sizeof(double), cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    for (int v : hc) h->cap_hit |= v;
    if (held) {
        err.assign(nb, 0.0);
        for (int b = 0; b < nb; ++b)
            err[b] = (ring[b] && nd[2 * b + 1] > 0.0) ? std::sqrt(nd[2 * b] / nd[2 * b + 1]) : 0.0;
    }
    dfree(c, base, bytes, s);
    if (rs != HODLR_OK) set_error("BDLR kernel launch failed");
    return rs;
}

}  // namespace

// depth >= 0: every block at that depth.  depth < 0: the adaptive scheme of
// Sec. 5.3 -- every block from depth 1; a block whose relative Frobenius error
// on the held-out rows and columns (those at distance depth + 1, relative to
// every row and column examined) exceeds tol, while such rows or columns
// exist, is computed again at depth + 1.
hodlr_status run_bdlr(hodlr_t *h, const hodlr_graph *g, int depth, cudaStream_t s, std::vector<void *> &Ust,
                      std::vector<void *> &Vst) {
    const int L = h->L;
    if (h->n > INT32_MAX) {
        set_error("BDLR: n beyond 2^31");
        return HODLR_RANGE;
    }
    for (int64_t v = 0; v < h->n; ++v)
        if (g->rowptr[v + 1] < g->rowptr[v]) {
            set_error("BDLR: graph rowptr not monotone at %lld", (long long)v);
            return HODLR_INVALID_ARG;
        }
    const bool adaptive = depth < 0;
    std::vector<BdlrBlock> todo;
    for (int l = 1; l <= L; ++l)
        for (int i = 0; i < (1 << l); ++i) todo.push_back(BdlrBlock{l, i, adaptive ? 1 : depth});
    std::vector<double> err;
    std::vector<char> ring;
    h->bdlr_depth_max = 0;
    while (!todo.empty()) {
        HODLR_TRY(bdlr_pass(h, g, todo, s, Ust, Vst, adaptive, err, ring));
        for (auto &b : todo) h->bdlr_depth_max = std::max(h->bdlr_depth_max, b.depth);
        if (!adaptive) break;
        std::vector<BdlrBlock> next;
        for (size_t k = 0; k < todo.size(); ++k)
            if (err[k] > h->tol && ring[k]) next.push_back(BdlrBlock{todo[k].l, todo[k].i, todo[k].depth + 1});
        todo.swap(next);
    }
    return HODLR_OK;
}

}  // namespace hodlr
