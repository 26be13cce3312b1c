// C ABI of libhodlr: contexts, HODLR construction (tree, compression staging,
// rank compaction), factor / solve entry points, statistics and export.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "internal.cuh"

namespace hodlr {

static thread_local char g_err[1024] = "";

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

static std::atomic<long long> g_launches{0};
static thread_local LaunchCapture *t_capture = nullptr;

void note_launch(long long k) {
    if (t_capture)
        t_capture->captured += k;
    else
        g_launches.fetch_add(k, std::memory_order_relaxed);
}
long long launch_total() { return g_launches.load(std::memory_order_relaxed); }
LaunchCapture::LaunchCapture() : prev(t_capture) { t_capture = this; }
LaunchCapture::~LaunchCapture() { t_capture = prev; }

// ------------------------------------------------------------------ profiling
namespace {
struct ProfRec {
    const char *name;
    cudaEvent_t e0, e1;
};
std::mutex g_prof_mu;
std::vector<ProfRec> g_prof;
std::atomic<int> g_prof_on{0};
}  // namespace

ProfScope::ProfScope(const char *kernel, cudaStream_t stream) {
    if (!g_prof_on.load(std::memory_order_relaxed)) return;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
        cudaGetLastError();
        return;
    }
    if (cudaEventCreate(&e0) != cudaSuccess) {
        cudaGetLastError();
        e0 = nullptr;
        return;
    }
    name = kernel;
    s = stream;
    cudaEventRecord(e0, s);
}

ProfScope::~ProfScope() {
    if (!e0) return;
    cudaEvent_t e1 = nullptr;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        cudaEventDestroy(e0);
        return;
    }
    cudaEventRecord(e1, s);
    std::lock_guard<std::mutex> lock(g_prof_mu);
    g_prof.push_back(ProfRec{name, e0, e1});
}

static void prof_clear() {
    std::lock_guard<std::mutex> lock(g_prof_mu);
    for (auto &r : g_prof) {
        cudaEventDestroy(r.e0);
        cudaEventDestroy(r.e1);
    }
    g_prof.clear();
}

hodlr_status status_from_word(int w) {
    if (w & ST_NONFINITE) return HODLR_NONFINITE_INPUT;
    if (w & ST_SINGULAR) return HODLR_SINGULAR;
    if (w & ST_TIMEOUT) return HODLR_TIMEOUT;
    if (w & ST_RANGE) return HODLR_RANGE;
    return HODLR_OK;
}

hodlr_status take_status(hodlr_ctx *c, cudaStream_t s) {
    HODLR_TRY_CUDA(cudaMemcpyAsync(c->h_status, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, s));
    HODLR_TRY_CUDA(cudaMemsetAsync(c->d_status, 0, sizeof(int), s));
    HODLR_TRY_CUDA(cudaStreamSynchronize(s));
    return status_word(*c->h_status);
}

hodlr_status status_word(int w) {
    if (w) {
        set_error("device status word 0x%x (%s%s%s%s)", w, (w & ST_NONFINITE) ? "non-finite value " : "",
                  (w & ST_SINGULAR) ? "zero pivot " : "", (w & ST_TIMEOUT) ? "wait budget exceeded " : "",
                  (w & ST_RANGE) ? "size limit " : "");
    }
    return status_from_word(w);
}

// Device memory of the library: the context's allocator (or the CUDA pool) for
// new blocks; released blocks are kept in the context's cache and handed out
// again for requests of the same rounded size, so repeated solves of one
// problem allocate nothing.  A cached block carries an event recorded on the
// stream that released it; a request on another stream waits for it.
namespace {
size_t round_block(size_t bytes) { return (std::max<size_t>(bytes, 1) + 255) & ~size_t(255); }

void *raw_alloc(hodlr_ctx *c, size_t bytes, cudaStream_t s) {
    if (c->alloc) return c->alloc(bytes, c->user, reinterpret_cast<hodlr_stream>(s));
    void *p = nullptr;
    if (cudaMallocAsync(&p, bytes, s) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void raw_free(hodlr_ctx *c, void *p, size_t bytes, cudaStream_t s) {
    if (c->free_fn)
        c->free_fn(p, bytes, c->user, reinterpret_cast<hodlr_stream>(s));
    else
        cudaFreeAsync(p, s);
}
}  // namespace

void *dalloc(hodlr_ctx *c, size_t bytes, cudaStream_t s) {
    const size_t sz = round_block(bytes);
    hodlr_cached_block b{nullptr, 0, nullptr, nullptr};
    {
        std::lock_guard<std::mutex> lock(c->cache_mu);
        auto it = c->cache.find(sz);
        if (it != c->cache.end() && !it->second.empty()) {
            auto &v = it->second;
            size_t k = v.size() - 1;
            for (size_t q = v.size(); q-- > 0;)
                if (v[q].stream == s) {   // prefer a block released on this stream
                    k = q;
                    break;
                }
            b = v[k];
            v[k] = v.back();
            v.pop_back();
            c->cache_bytes -= sz;
            --c->cache_count;
        }
    }
    if (b.p) {
        // wait first, then recycle the event (a later record of it does not
        // affect a wait already issued)
        if (b.stream != s) cudaStreamWaitEvent(s, b.ev, 0);
        std::lock_guard<std::mutex> lock(c->cache_mu);
        c->spare_events.push_back(b.ev);
        return b.p;
    }
    return raw_alloc(c, sz, s);
}

void dfree(hodlr_ctx *c, void *p, size_t bytes, cudaStream_t s) {
    if (!p) return;
    const size_t sz = round_block(bytes);
    cudaEvent_t ev = nullptr;
    {
        std::lock_guard<std::mutex> lock(c->cache_mu);
        if (!c->spare_events.empty()) {
            ev = c->spare_events.back();
            c->spare_events.pop_back();
        }
    }
    if (!ev && cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        raw_free(c, p, sz, s);
        return;
    }
    cudaEventRecord(ev, s);
    std::vector<hodlr_cached_block> evict;
    {
        std::lock_guard<std::mutex> lock(c->cache_mu);
        c->cache[sz].push_back(hodlr_cached_block{p, sz, s, ev});
        c->fifo.push_back({p, sz});
        c->cache_bytes += sz;
        ++c->cache_count;
        while (c->cache_bytes > HODLR_CACHE_LIMIT && !c->fifo.empty()) {
            const auto f = c->fifo.front();
            c->fifo.pop_front();
            auto &v = c->cache[f.second];
            for (size_t q = 0; q < v.size(); ++q)
                if (v[q].p == f.first) {
                    evict.push_back(v[q]);
                    v[q] = v.back();
                    v.pop_back();
                    c->cache_bytes -= f.second;
                    --c->cache_count;
                    break;
                }
        }
        if (c->fifo.size() > 2 * c->cache_count + 64) {
            // drop the entries of blocks handed out again
            std::deque<std::pair<void *, size_t>> keep;
            for (const auto &f : c->fifo) {
                const auto it = c->cache.find(f.second);
                if (it == c->cache.end()) continue;
                for (const auto &q : it->second)
                    if (q.p == f.first) {
                        keep.push_back(f);
                        break;
                    }
            }
            c->fifo.swap(keep);
        }
    }
    for (auto &b : evict) {
        // the block may have been used on streams its allocator does not know
        // about: hand it back only once that use is complete
        cudaEventSynchronize(b.ev);
        raw_free(c, b.p, b.bytes, b.stream);
        cudaEventDestroy(b.ev);
    }
}

size_t Arena::take(size_t b) {
    const size_t o = bytes;
    bytes += (std::max<size_t>(b, 1) + 255) & ~size_t(255);
    return o;
}

void *own(hodlr_t *h, size_t bytes, cudaStream_t s) {
    void *p = dalloc(h->ctx, bytes, s);
    if (p) h->owned.push_back(DevBuf{p, bytes == 0 ? 256 : bytes});
    return p;
}

hodlr_status ensure_work(hodlr_t *h, size_t bytes, cudaStream_t s) {
    if (h->work_bytes >= bytes) return HODLR_OK;
    if (h->work) dfree(h->ctx, h->work, h->work_bytes, s);
    h->work = dalloc(h->ctx, bytes, s);
    if (!h->work) {
        h->work_bytes = 0;
        set_error("out of device memory (%zu bytes of workspace)", bytes);
        return HODLR_OUT_OF_MEMORY;
    }
    h->work_bytes = bytes;
    return HODLR_OK;
}

namespace {

// dst(:, col) for the rows of every node of a level: src column if col < rank, else 0.
// U rows of a node carry the node's own block (rank(node)); V rows of a node
// carry the sibling's block A(sibling, node) (rank(sibling)): sib = 1.
template <typename S, typename D>
__global__ void compact_kernel(const S *__restrict__ src, int64_t lds, D *__restrict__ dst, int64_t ldd,
                               const int64_t *__restrict__ bounds, int L, int l, const int32_t *__restrict__ ranks,
                               int rp, int sib) {
    const int col = blockIdx.y;
    const int node = blockIdx.z;
    const int64_t r0 = bounds[(size_t)node << (L - l)];
    const int64_t r1 = bounds[(size_t)(node + 1) << (L - l)];
    const int rk = ranks[sib ? (node ^ 1) : node];
    for (int64_t i = r0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < r1; i += (int64_t)gridDim.x * blockDim.x)
        dst[i + col * ldd] = col < rk ? (D)src[i + col * lds] : (D)0;
}

template <typename S>
__global__ void to_double_kernel(const S *__restrict__ src, int64_t lds, double *__restrict__ dst, int64_t ldd,
                                 int64_t rows, int64_t cols) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < rows * cols;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e % rows, j = e / rows;
        dst[i + j * ldd] = (double)src[i + j * lds];
    }
}

template <typename S, typename D>
hodlr_status launch_compact(const void *src, int64_t lds, void *dst, int64_t ldd, const int64_t *bounds, int L, int l,
                            const int32_t *ranks, int rp, int64_t node_max, cudaStream_t s) {
    if (rp == 0) return HODLR_OK;
    dim3 grid((unsigned)std::max<int64_t>(1, std::min<int64_t>((node_max + 255) / 256, 64)), rp, 1u << l);
    // src/dst given as the U pair: U(node rows) uses rank(node)
    compact_kernel<S, D><<<grid, 256, 0, s>>>(reinterpret_cast<const S *>(src), lds, reinterpret_cast<D *>(dst), ldd,
                                              bounds, L, l, ranks, rp, 0);
    note_launch();
    HODLR_TRY_CUDA(cudaGetLastError());
    return HODLR_OK;
}

template <typename S, typename D>
hodlr_status launch_compact_v(const void *src, int64_t lds, void *dst, int64_t ldd, const int64_t *bounds, int L,
                              int l, const int32_t *ranks, int rp, int64_t node_max, cudaStream_t s) {
    if (rp == 0) return HODLR_OK;
    dim3 grid((unsigned)std::max<int64_t>(1, std::min<int64_t>((node_max + 255) / 256, 64)), rp, 1u << l);
    compact_kernel<S, D><<<grid, 256, 0, s>>>(reinterpret_cast<const S *>(src), lds, reinterpret_cast<D *>(dst), ldd,
                                              bounds, L, l, ranks, rp, 1);
    note_launch();
    HODLR_TRY_CUDA(cudaGetLastError());
    return HODLR_OK;
}

hodlr_status check_matrix(const hodlr_matrix *A) {
    if (!A || !A->data || A->n <= 0 || A->ld < A->n) {
        set_error("invalid matrix descriptor");
        return HODLR_INVALID_ARG;
    }
    return HODLR_OK;
}

}  // namespace
}  // namespace hodlr

using namespace hodlr;

extern "C" {

const char *hodlr_status_string(hodlr_status s) {
    switch (s) {
        case HODLR_OK: return "ok";
        case HODLR_INVALID_ARG: return "invalid argument";
        case HODLR_OUT_OF_MEMORY: return "out of device memory";
        case HODLR_CUDA_ERROR: return "CUDA error";
        case HODLR_SINGULAR: return "singular leaf block or Woodbury core";
        case HODLR_NOT_FACTORED: return "not factored";
        case HODLR_NOT_CONVERGED: return "GMRES did not converge";
        case HODLR_TIMEOUT: return "device wait exceeded its budget";
        case HODLR_NONFINITE_INPUT: return "non-finite or out-of-range input";
        case HODLR_RANGE: return "size beyond a fixed limit";
    }
    return "unknown status";
}

const char *hodlr_last_error(void) { return g_err; }

hodlr_status hodlr_ctx_set_wait_test(hodlr_ctx *c, unsigned long long spin_limit, int unreachable) {
    if (!c || spin_limit > (1ull << 40)) {
        set_error("hodlr_ctx_set_wait_test: invalid argument");
        return HODLR_INVALID_ARG;
    }
    c->wait_limit = spin_limit;
    c->wait_extra = unreachable ? 1u : 0u;
    return HODLR_OK;
}

hodlr_status hodlr_ctx_set_apply_path(hodlr_ctx *c, int path) {
    if (!c || path < 0 || path > 2) {
        set_error("hodlr_ctx_set_apply_path: invalid argument");
        return HODLR_INVALID_ARG;
    }
    c->apply_path = path;
    return HODLR_OK;
}

hodlr_status hodlr_profile_enable(int on) {
    hodlr::prof_clear();
    hodlr::g_prof_on.store(on ? 1 : 0);
    return HODLR_OK;
}

hodlr_status hodlr_profile_read(const char *kernel, double *ms_total, long long *launches) {
    if (!kernel || !ms_total || !launches) {
        set_error("hodlr_profile_read: NULL argument");
        return HODLR_INVALID_ARG;
    }
    double ms = 0.0;
    long long cnt = 0;
    std::lock_guard<std::mutex> lock(hodlr::g_prof_mu);
    for (auto &r : hodlr::g_prof) {
        if (std::strcmp(r.name, kernel) != 0) continue;
        float t = 0.f;
        HODLR_TRY_CUDA(cudaEventSynchronize(r.e1));
        HODLR_TRY_CUDA(cudaEventElapsedTime(&t, r.e0, r.e1));
        ms += t;
        ++cnt;
    }
    *ms_total = ms;
    *launches = cnt;
    return HODLR_OK;
}

hodlr_status hodlr_launch_count(long long *out) {
    if (!out) return HODLR_INVALID_ARG;
    *out = hodlr::launch_total();
    return HODLR_OK;
}

void hodlr_opts_default(hodlr_opts *o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->precision = HODLR_FP32;
    o->compress_precision = -1;
    o->rank_cap = 0;
    o->bdlr_depth = -1;
    o->core_cond_threshold = 0.0;
    o->leaf_bounds = nullptr;
    o->n_leaf_bounds = 0;
    o->seed = 2;
}

hodlr_status hodlr_ctx_create(int device, hodlr_alloc_fn alloc, hodlr_free_fn free_fn, void *user, hodlr_ctx **out) {
    if (!out || ((alloc == nullptr) != (free_fn == nullptr))) {
        set_error("hodlr_ctx_create: out is NULL or only one of alloc/free given");
        return HODLR_INVALID_ARG;
    }
    int ndev = 0;
    HODLR_TRY_CUDA(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) {
        set_error("hodlr_ctx_create: device %d of %d", device, ndev);
        return HODLR_INVALID_ARG;
    }
    HODLR_TRY_CUDA(cudaSetDevice(device));
    hodlr_ctx *c = new hodlr_ctx();
    c->device = device;
    c->alloc = alloc;
    c->free_fn = free_fn;
    c->user = user;
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (cudaMalloc(&c->d_status, sizeof(int)) != cudaSuccess ||
        cudaMallocHost(&c->h_status, 65 * sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        set_error("hodlr_ctx_create: cannot allocate the status word");
        return HODLR_OUT_OF_MEMORY;
    }
    if (cudaMallocHost(&c->h_report, HODLR_REPORT_BYTES) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(c->d_status);
        cudaFreeHost(c->h_status);
        delete c;
        set_error("hodlr_ctx_create: cannot allocate the pinned report buffer");
        return HODLR_OUT_OF_MEMORY;
    }
    cudaMemset(c->d_status, 0, sizeof(int));
    *c->h_status = 0;
    c->h_scratch = c->h_status + 1;
    for (int i = 0; i < HODLR_SIDE_STREAMS; ++i)
        if (cudaStreamCreateWithFlags(&c->side[i], cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            for (int q = 0; q < i; ++q) cudaStreamDestroy(c->side[q]);
            cudaFree(c->d_status);
            cudaFreeHost(c->h_status);
            cudaFreeHost(c->h_report);
            delete c;
            set_error("hodlr_ctx_create: cannot create streams");
            return HODLR_CUDA_ERROR;
        }
    *out = c;
    return HODLR_OK;
}

hodlr_status hodlr_ctx_destroy(hodlr_ctx *c) {
    if (!c) return HODLR_OK;
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    for (auto &g : c->graph_trash) {
        if (g.first) cudaGraphExecDestroy(g.first);
        if (g.second) cudaGraphDestroy(g.second);
    }
    c->graph_trash.clear();
    for (auto &kv : c->cache)
        for (auto &b : kv.second) {
            raw_free(c, b.p, b.bytes, nullptr);
            cudaEventDestroy(b.ev);
        }
    c->cache.clear();
    c->fifo.clear();
    for (auto e : c->spare_events) cudaEventDestroy(e);
    c->spare_events.clear();
    cudaDeviceSynchronize();
    for (int i = 0; i < HODLR_SIDE_STREAMS; ++i)
        if (c->side[i]) cudaStreamDestroy(c->side[i]);
    cudaFree(c->d_status);
    cudaFreeHost(c->h_status);
    if (c->h_report) cudaFreeHost(c->h_report);
    delete c;
    return HODLR_OK;
}

hodlr_status hodlr_destroy(hodlr_t *h) {
    if (!h) return HODLR_OK;
    cudaSetDevice(h->ctx->device);
    cudaDeviceSynchronize();
    free_plan(h, nullptr);
    for (auto &e : h->fev)
        if (e) cudaEventDestroy(e);
    for (auto &b : h->owned) dfree(h->ctx, b.p, b.bytes, nullptr);
    if (h->work) dfree(h->ctx, h->work, h->work_bytes, nullptr);
    delete h;
    return HODLR_OK;
}

// One front.  With sync_leaf_status false a single-leaf front returns without
// reading the status word (its compression is empty); the caller reads it once
// for a whole batch.
static hodlr_status build_one(hodlr_ctx *c, const hodlr_matrix *A, int leaf, double tol, int method,
                              const hodlr_graph *g, const hodlr_opts *o_in, hodlr_stream stream, hodlr_t **out,
                              bool sync_leaf_status) {
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (!c || !out) {
        set_error("hodlr_build: NULL context or output");
        return HODLR_INVALID_ARG;
    }
    HODLR_TRY(check_matrix(A));
    hodlr_opts o;
    hodlr_opts_default(&o);
    if (o_in) o = *o_in;
    if (!(tol > 0.0) || !(tol < 1.0)) {
        set_error("hodlr_build: tol must be in (0, 1)");
        return HODLR_INVALID_ARG;
    }
    if (method != HODLR_ACA && method != HODLR_BDLR) {
        set_error("hodlr_build: unknown method %d", method);
        return HODLR_INVALID_ARG;
    }
    if (method == HODLR_BDLR && (!g || !g->rowptr || !g->colind || g->n != A->n)) {
        set_error("hodlr_build: BDLR needs the graph of the matrix");
        return HODLR_INVALID_ARG;
    }
    if (o.precision < HODLR_FP64 || o.precision > HODLR_FP16) {
        set_error("hodlr_build: unknown precision %d", o.precision);
        return HODLR_INVALID_ARG;
    }
    int cprec = o.compress_precision;
    if (cprec < 0) cprec = (o.precision == HODLR_FP64) ? HODLR_FP64 : HODLR_FP32;
    if (cprec != HODLR_FP64 && cprec != HODLR_FP32) {
        set_error("hodlr_build: compress_precision must be FP64 or FP32");
        return HODLR_INVALID_ARG;
    }
    const int rank_cap = o.rank_cap <= 0 ? 1024 : o.rank_cap;
    if (rank_cap > 1024) {
        set_error("hodlr_build: rank_cap %d > 1024", rank_cap);
        return HODLR_RANGE;
    }
    HODLR_TRY_CUDA(cudaSetDevice(c->device));
    const int64_t n = A->n;
    // ---- tree
    std::vector<int64_t> bounds;
    if (o.leaf_bounds && o.n_leaf_bounds > 0) {
        const int nb = o.n_leaf_bounds;
        const int nl = nb - 1;
        if (nl < 1 || (nl & (nl - 1)) != 0 || o.leaf_bounds[0] != 0 || o.leaf_bounds[nl] != n) {
            set_error("hodlr_build: leaf_bounds must hold 2^L + 1 increasing offsets from 0 to n");
            return HODLR_INVALID_ARG;
        }
        for (int i = 0; i < nl; ++i)
            if (o.leaf_bounds[i + 1] <= o.leaf_bounds[i]) {
                set_error("hodlr_build: leaf_bounds not strictly increasing");
                return HODLR_INVALID_ARG;
            }
        bounds.assign(o.leaf_bounds, o.leaf_bounds + nb);
    } else {
        if (leaf < 1) {
            set_error("hodlr_build: leaf must be >= 1");
            return HODLR_INVALID_ARG;
        }
        std::vector<std::pair<int64_t, int64_t>> r{{0, n}};
        auto widest = [&]() {
            int64_t w = 0;
            for (auto &q : r) w = std::max(w, q.second - q.first);
            return w;
        };
        while (widest() > leaf) {
            std::vector<std::pair<int64_t, int64_t>> nx;
            for (auto &q : r) {
                const int64_t mid = q.first + (q.second - q.first) / 2;
                nx.push_back({q.first, mid});
                nx.push_back({mid, q.second});
            }
            r.swap(nx);
            if (r.size() > (1u << 15)) break;
        }
        for (auto &q : r) bounds.push_back(q.first);
        bounds.push_back(n);
    }
    const int nleaf = (int)bounds.size() - 1;
    int L = 0;
    while ((1 << L) < nleaf) ++L;
    if (L >= HODLR_MAX_LEVELS) {
        set_error("hodlr_build: %d levels exceed the limit %d", L, HODLR_MAX_LEVELS - 1);
        return HODLR_RANGE;
    }
    for (int i = 0; i < nleaf; ++i)
        if (bounds[i + 1] - bounds[i] <= 0) {
            set_error("hodlr_build: empty leaf (n too small for the leaf size)");
            return HODLR_INVALID_ARG;
        }
    hodlr_t *h = new hodlr_t();
    h->ctx = c;
    h->A = A->data;
    h->n = n;
    h->lda = A->ld;
    h->sym = A->symmetric ? 1 : 0;
    h->L = L;
    h->bounds = bounds;
    h->prec = (o.precision == HODLR_FP64) ? HODLR_FP64 : HODLR_FP32;
    h->store = o.precision;
    h->cprec = cprec;
    h->method = method;
    h->tol = tol;
    h->rank_cap = rank_cap;
    h->ldn = (n + 31) / 32 * 32;
    h->lv.resize(L + 1);
    // the Woodbury core condition guard: kappa_1 of every core (unless the
    // threshold is negative); with FP32 arithmetic the cores above the
    // threshold are re-inverted in FP64.  Default threshold: tol / 2^-24, the
    // condition at which an FP32 inversion's error bound kappa u_32 reaches the
    // compression tolerance.
    h->guard = o.core_cond_threshold >= 0.0;
    h->promote = h->guard && h->prec == HODLR_FP32;
    h->cond_thr = o.core_cond_threshold > 0.0 ? o.core_cond_threshold : tol / 5.9604644775390625e-8;
    int64_t bmax = 0;
    for (int i = 0; i < nleaf; ++i) bmax = std::max(bmax, bounds[i + 1] - bounds[i]);
    h->bmax = (int)bmax;
    auto fail = [&](hodlr_status s) {
        hodlr_destroy(h);
        return s;
    };
    auto nrange = [&](int l, int i, int64_t &r0, int64_t &m) {
        r0 = bounds[(size_t)i << (L - l)];
        m = bounds[(size_t)(i + 1) << (L - l)] - r0;
    };
    // ---- sizes of everything known before the ranks: the tree and pivot
    // metadata, the apply's tiles and the leaf inverses (one owned allocation),
    // and the compression staging (one temporary allocation)
    const size_t ce = elem_size(cprec);
    std::vector<int4> tiles;
    std::vector<int> tfirst(nleaf + 1);
    for (int i = 0; i < nleaf; ++i) {
        tfirst[i] = (int)tiles.size();
        for (int64_t r = bounds[i]; r < bounds[i + 1]; r += 32)
            tiles.push_back(make_int4(i, (int)r, (int)std::min<int64_t>(32, bounds[i + 1] - r), 0));
    }
    tfirst[nleaf] = (int)tiles.size();
    int64_t max_m = 0;
    for (int l = 1; l <= L; ++l) {
        Level &lv = h->lv[l];
        lv.nnodes = 1 << l;
        int cap = 0;
        for (int i = 0; i < lv.nnodes; ++i) {
            int64_t r0, m, c0, mc;
            nrange(l, i, r0, m);
            nrange(l, i ^ 1, c0, mc);
            cap = (int)std::max<int64_t>(cap, std::min<int64_t>(rank_cap, std::min(m, mc)));
            max_m = std::max(max_m, m);
        }
        lv.cap = std::max(cap, 1);
    }
    Arena meta, stage;
    const size_t o_bounds = meta.take(bounds.size() * sizeof(int64_t));
    const size_t o_caphit = meta.take((size_t)(2 << L) * sizeof(int32_t));
    std::vector<size_t> o_prow(L + 1), o_pcol(L + 1), o_rank(L + 1), o_ust(L + 1), o_vst(L + 1);
    const size_t o_piv0 = meta.bytes;
    for (int l = 1; l <= L; ++l) o_prow[l] = meta.take((size_t)h->lv[l].nnodes * h->lv[l].cap * sizeof(int32_t));
    for (int l = 1; l <= L; ++l) o_pcol[l] = meta.take((size_t)h->lv[l].nnodes * h->lv[l].cap * sizeof(int32_t));
    const size_t piv_bytes = meta.bytes - o_piv0;
    for (int l = 1; l <= L; ++l) o_rank[l] = meta.take((size_t)h->lv[l].nnodes * sizeof(int32_t));
    const size_t o_tiles = meta.take(std::max<size_t>(tiles.size(), 1) * sizeof(int4));
    const size_t o_tfirst = meta.take(tfirst.size() * sizeof(int));
    const size_t o_leafinv = meta.take((size_t)nleaf * bmax * bmax * elem_size(h->prec));
    for (int l = 1; l <= L; ++l) {
        o_ust[l] = stage.take((size_t)h->ldn * h->lv[l].cap * ce);
        o_vst[l] = stage.take((size_t)h->ldn * h->lv[l].cap * ce);
    }
    const size_t o_desc = stage.take((size_t)(2 << L) * sizeof(AcaBlockDesc));
    char *mbase = (char *)own(h, meta.bytes, st);
    if (!mbase) return fail(HODLR_OUT_OF_MEMORY);
    char *sbase = (char *)dalloc(c, stage.bytes, st);
    if (!sbase) return fail(HODLR_OUT_OF_MEMORY);
    std::vector<std::pair<void *, size_t>> temp{{sbase, stage.bytes}};
    h->d_bounds = (int64_t *)(mbase + o_bounds);
    // ---- compression staging and per-block descriptors
    std::vector<void *> Ust(L + 1, nullptr), Vst(L + 1, nullptr);
    h->piv_rows.assign(L + 1, nullptr);
    h->piv_cols.assign(L + 1, nullptr);
    h->d_ranks.assign(L + 1, nullptr);
    int32_t *caphit = (int32_t *)(mbase + o_caphit);
    cudaMemsetAsync(mbase + o_piv0, 0xff, piv_bytes, st);
    std::vector<AcaBlockDesc> blocks;
    for (int l = 1; l <= L; ++l) {
        Level &lv = h->lv[l];
        Ust[l] = sbase + o_ust[l];
        Vst[l] = sbase + o_vst[l];
        h->piv_rows[l] = (int32_t *)(mbase + o_prow[l]);
        h->piv_cols[l] = (int32_t *)(mbase + o_pcol[l]);
        h->d_ranks[l] = (int32_t *)(mbase + o_rank[l]);
        for (int i = 0; i < lv.nnodes; ++i) {
            AcaBlockDesc bd;
            nrange(l, i, bd.r0, bd.m);
            nrange(l, i ^ 1, bd.c0, bd.nc);
            bd.ld = h->ldn;
            bd.U = Ust[l];
            bd.V = Vst[l];
            bd.cap = lv.cap;
            bd.rank = h->d_ranks[l] + i;
            bd.prow = h->piv_rows[l] + (size_t)i * lv.cap;
            bd.pcol = h->piv_cols[l] + (size_t)i * lv.cap;
            bd.cap_hit = caphit + blocks.size();
            blocks.push_back(bd);
        }
    }
    auto free_temp = [&]() {
        for (auto &q : temp) dfree(c, q.first, q.second, st);
        temp.clear();
    };
    cudaEvent_t lfork = nullptr, ljoin = nullptr;
    cudaEventCreateWithFlags(&lfork, cudaEventDisableTiming);
    cudaEventCreateWithFlags(&ljoin, cudaEventDisableTiming);
    cudaEvent_t e0;
    cudaEventCreate(&e0);
    cudaEventRecord(e0, st);
    hodlr_status rs = HODLR_OK;
    // done[c - 1]: level c compressed; rstream[c]: the stream its ranks are read on
    std::vector<cudaEvent_t> done;
    std::vector<cudaStream_t> rstream(L + 1, st);
    // The leaf inverses depend on A only and run on a side stream.  With ACA
    // they are issued right after the top level's launch (one cluster per
    // block, few SMs), so that their CTAs are dispatched before the lower
    // levels' and every level's factor share, which waits for them, can start
    // as soon as its level is compressed.
    h->leafinv = mbase + o_leafinv;
    cudaStream_t lstream = c->side[HODLR_SIDE_STREAMS - 1];
    hodlr_status rleaf = HODLR_OK;
    bool leaf_issued = false;
    auto issue_leaf = [&]() -> hodlr_status {
        cudaEventRecord(lfork, st);
        cudaStreamWaitEvent(lstream, lfork, 0);
        rleaf = leaf_inverses(h, lstream);
        cudaEventRecord(ljoin, lstream);
        leaf_issued = true;
        return rleaf;
    };
    if (method == HODLR_ACA) {
        AcaBlockDesc *db = (AcaBlockDesc *)(sbase + o_desc);
        cudaMemcpyAsync(db, blocks.data(), blocks.size() * sizeof(AcaBlockDesc), cudaMemcpyHostToDevice, st);
        std::vector<int> first;
        std::vector<int64_t> maxdim;
        int b0 = 0;
        for (int l = 1; l <= L; ++l) {
            first.push_back(b0);
            int64_t md = 0;
            for (int i = 0; i < (1 << l); ++i) md = std::max(md, std::max(blocks[b0 + i].m, blocks[b0 + i].nc));
            maxdim.push_back(md);
            b0 += 1 << l;
        }
        first.push_back(b0);
        rs = launch_aca_levels(c, A->data, A->ld, h->sym, cprec, db, first, maxdim, tol, st, done, issue_leaf);
        for (int l = 1; l <= L; ++l) rstream[l] = c->side[(l - 1) % HODLR_SIDE_STREAMS];
    } else {
        // -2: the adaptive depth of Sec. 5.3 (run_bdlr grows it per block)
        const int depth = o.bdlr_depth >= 0 ? o.bdlr_depth
                                            : (o.bdlr_depth == -2 ? -1 : (int)std::lround(-std::log10(tol)));
        rs = run_bdlr(h, g, depth, st, Ust, Vst);
        done.assign(L, nullptr);
        for (int l = 0; l < L; ++l) {
            cudaEventCreate(&done[l]);
            cudaEventRecord(done[l], st);
        }
    }
    // ---- what the compression does not need, issued after its launch: the
    // leaf bounds, the apply's row tiles (32 rows, never straddling a leaf) and
    // the first tile of every leaf, and (without ACA levels) the leaf inverses
    // (they join the levels' streams and the caller's stream later)
    cudaMemcpyAsync(h->d_bounds, bounds.data(), bounds.size() * sizeof(int64_t), cudaMemcpyHostToDevice, st);
    h->d_tiles = (const int4 *)(mbase + o_tiles);
    h->d_tile_first = (int *)(mbase + o_tfirst);
    h->ntiles = (int)tiles.size();
    if (!tiles.empty())
        cudaMemcpyAsync((void *)h->d_tiles, tiles.data(), tiles.size() * sizeof(int4), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(h->d_tile_first, tfirst.data(), tfirst.size() * sizeof(int), cudaMemcpyHostToDevice, st);
    if (!leaf_issued) issue_leaf();
    // share_done[l]: level l's compaction and (unless deferred) its share of the
    // factorisation are complete
    std::vector<cudaEvent_t> share_done(L + 1, nullptr);
    cudaEvent_t st_mark = nullptr;
    auto drop_events = [&]() {
        if (st_mark) cudaEventDestroy(st_mark);
        st_mark = nullptr;
        for (auto e : done)
            if (e) cudaEventDestroy(e);
        done.clear();
        for (auto e : share_done)
            if (e) cudaEventDestroy(e);
        share_done.clear();
        cudaEventDestroy(lfork);
        cudaEventDestroy(ljoin);
        cudaEventDestroy(e0);
    };
    if (rs == HODLR_OK) rs = rleaf;
    if (rs != HODLR_OK) {
        cudaDeviceSynchronize();
        drop_events();
        free_temp();
        return fail(rs);
    }
    // ---- level by level from the leaves: ranks -> layout -> compaction -> the
    // level's share of the factorisation, issued while the upper levels are
    // still being compressed.  Level l's compaction and share run on its own
    // stream (the one its ranks are read on); the share waits for a deeper
    // level's share only where it starts reading that level's factors, so the
    // shares of different levels overlap.
    cudaEventCreateWithFlags(&st_mark, cudaEventDisableTiming);
    cudaEventRecord(st_mark, st);   // everything allocated so far is ordered before this
    const size_t pe = elem_size(h->prec);
    const bool q16 = (h->store == HODLR_BF16 || h->store == HODLR_FP16);
    const bool factor_now = o.defer_factor == 0;
    h->Ul.assign(L + 1, nullptr);
    h->Dl.assign(L + 1, nullptr);
    h->Vl.assign(L + 1, nullptr);
    h->El.assign(L + 1, nullptr);
    h->Vql.assign(L + 1, nullptr);
    h->Eql.assign(L + 1, nullptr);
    h->Sinv.assign(L, nullptr);
    h->core_cond.assign(L, nullptr);
    h->core_flag.assign(L, nullptr);
    h->core_count.assign(L, nullptr);
    h->Sinv64.assign(L, nullptr);
    h->vscale.assign(L + 1, nullptr);
    h->escale.assign(L + 1, nullptr);
    if (factor_now && L > 0) {
        if (!h->fev[0]) {
            cudaEventCreate(&h->fev[0]);
            cudaEventCreate(&h->fev[1]);
        }
        cudaEventRecord(h->fev[0], st);
    }
    // The factors the apply streams (E = d S^-1(half) and V, or their 16-bit
    // copies) of all levels share one region, filled from the leaves up as the
    // ranks become known: a compact span (few pages) for the apply.  It is
    // reserved for the rank caps; only the prefix the ranks need is touched.
    const size_t se = q16 ? 2 : pe;
    size_t dv_bound = 0;
    for (int l = 1; l <= L; ++l) {
        const size_t rmax = std::max((h->lv[l].cap + 7) / 8 * 8, 8);   // the padded rank's bound
        dv_bound += (((size_t)h->ldn * 2 * rmax * se + 255) & ~size_t(255)) +
                    (((size_t)h->ldn * rmax * se + 255) & ~size_t(255));
    }
    char *dvbase = L > 0 ? (char *)own(h, dv_bound, st) : nullptr;
    if (L > 0 && !dvbase) {
        cudaDeviceSynchronize();
        drop_events();
        free_temp();
        return fail(HODLR_OUT_OF_MEMORY);
    }
    size_t dv_used = 0;
    std::vector<int32_t> hcap;
    int hstat = 0, aca_status = 0;   // the status word after each level's compression
    for (int l = L; l >= 1; --l) {
        Level &lv = h->lv[l];
        lv.ranks.resize(lv.nnodes);
        hcap.resize(lv.nnodes);
        // (pageable destination: the copies return once level l is compressed)
        if (cudaMemcpyAsync(lv.ranks.data(), h->d_ranks[l], lv.nnodes * sizeof(int32_t), cudaMemcpyDeviceToHost,
                            rstream[l]) != cudaSuccess ||
            cudaMemcpyAsync(&hstat, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, rstream[l]) != cudaSuccess ||
            cudaMemcpyAsync(hcap.data(), caphit + ((1 << l) - 2), lv.nnodes * sizeof(int32_t),
                            cudaMemcpyDeviceToHost, rstream[l]) != cudaSuccess ||
            cudaStreamSynchronize(rstream[l]) != cudaSuccess) {
            cudaDeviceSynchronize();
            drop_events();
            free_temp();
            return fail(HODLR_CUDA_ERROR);
        }
        for (auto v : hcap) h->cap_hit |= v;
        aca_status |= hstat;
        int mx = 0;
        double sum = 0;
        for (int r : lv.ranks) {
            mx = std::max(mx, r);
            sum += r;
        }
        lv.rank_max = mx;
        lv.rank_mean = sum / lv.nnodes;
        lv.rp = mx == 0 ? 0 : (mx + 7) / 8 * 8;
        // storage of level l: the streamed E and V in the shared region, and
        // an arena with U, d, the cores of level l - 1 and (16-bit storage) the
        // FP32 E and V with the FP16 scales
        const size_t colb = (size_t)h->ldn * std::max(lv.rp, 1);
        const size_t sbe = ((2 * colb * se) + 255) & ~size_t(255), sbv = ((colb * se) + 255) & ~size_t(255);
        char *dv_e = dvbase + dv_used, *dv_v = dvbase + dv_used + sbe;
        dv_used += sbe + sbv;
        const int64_t s2 = 2 * (int64_t)lv.rp;
        Arena la;
        const size_t oU = la.take(colb * pe), oD = la.take(colb * pe);
        size_t oE = 0, oV = 0, ovs = 0, oes = 0;
        if (q16) {
            oE = la.take(2 * colb * pe);
            oV = la.take(colb * pe);
        }
        const size_t oS = la.take((size_t)(1 << (l - 1)) * std::max<int64_t>(s2 * s2, 1) * pe);
        const size_t oCond = h->guard ? la.take((size_t)(1 << (l - 1)) * sizeof(double)) : 0;
        const size_t oFlag = h->guard ? la.take((size_t)(1 << (l - 1)) * sizeof(int)) : 0;
        const size_t oCount = h->guard ? la.take(sizeof(unsigned)) : 0;
        const size_t oS64 = h->promote ? la.take((size_t)(1 << (l - 1)) * std::max<int64_t>(s2 * s2, 1) * 8) : 0;
        if (h->store == HODLR_FP16) {
            const size_t scb = (size_t)lv.nnodes * std::max(lv.rp, 1) * sizeof(float);
            ovs = la.take(scb);
            oes = la.take(2 * scb);
        }
        char *lb = (char *)own(h, la.bytes, st);
        if (!lb || dv_used > dv_bound) {
            cudaDeviceSynchronize();
            drop_events();
            free_temp();
            return fail(lb ? HODLR_RANGE : HODLR_OUT_OF_MEMORY);
        }
        h->Ul[l] = lb + oU;
        h->Dl[l] = lb + oD;
        h->Sinv[l - 1] = lb + oS;
        if (h->guard) {
            h->core_cond[l - 1] = (double *)(lb + oCond);
            h->core_flag[l - 1] = (int *)(lb + oFlag);
            h->core_count[l - 1] = (unsigned *)(lb + oCount);
            // a level without ranks has identity cores: kappa 1, nothing to redo
            if (lv.rp == 0) {
                std::vector<double> one((size_t)1 << (l - 1), 1.0);
                cudaMemcpyAsync(h->core_cond[l - 1], one.data(), one.size() * 8, cudaMemcpyHostToDevice, st);
                cudaMemsetAsync(h->core_flag[l - 1], 0, one.size() * sizeof(int), st);
                cudaStreamSynchronize(st);
            }
        }
        if (h->promote) h->Sinv64[l - 1] = (double *)(lb + oS64);
        if (q16) {
            h->El[l] = lb + oE;
            h->Vl[l] = lb + oV;
            h->Eql[l] = dv_e;
            h->Vql[l] = dv_v;
            if (h->store == HODLR_FP16) {
                h->vscale[l] = (float *)(lb + ovs);
                h->escale[l] = (float *)(lb + oes);
            }
        } else {
            h->El[l] = dv_e;
            h->Vl[l] = dv_v;
        }
        const cudaStream_t sl = c->side[(l - 1) % HODLR_SIDE_STREAMS];
        cudaStreamWaitEvent(sl, st_mark, 0);
        cudaStreamWaitEvent(sl, ljoin, 0);        // the leaf inverses (read by the share)
        cudaStreamWaitEvent(sl, done[l - 1], 0);  // level l compressed into the staging
        if (h->guard) cudaMemsetAsync(h->core_count[l - 1], 0, sizeof(unsigned), sl);
        if (lv.rp > 0) {
            // compaction writes the ranks' columns only: zero U and V
            cudaMemsetAsync(h->Ul[l], 0, colb * pe, sl);
            cudaMemsetAsync(h->Vl[l], 0, colb * pe, sl);
        }
        int64_t node_max = 0;
        for (int i = 0; i < lv.nnodes; ++i) {
            int64_t r0, m;
            nrange(l, i, r0, m);
            node_max = std::max(node_max, m);
        }
        char *Uc = (char *)h->Ul[l], *Vc = (char *)h->Vl[l];
        hodlr_status s3 = HODLR_OK;
        if (lv.rp > 0) {
            if (cprec == HODLR_FP64 && h->prec == HODLR_FP64) {
                s3 = launch_compact<double, double>(Ust[l], h->ldn, Uc, h->ldn, h->d_bounds, L, l, h->d_ranks[l],
                                                    lv.rp, node_max, sl);
                if (s3 == HODLR_OK)
                    s3 = launch_compact_v<double, double>(Vst[l], h->ldn, Vc, h->ldn, h->d_bounds, L, l,
                                                          h->d_ranks[l], lv.rp, node_max, sl);
            } else if (cprec == HODLR_FP64) {
                s3 = launch_compact<double, float>(Ust[l], h->ldn, Uc, h->ldn, h->d_bounds, L, l, h->d_ranks[l],
                                                   lv.rp, node_max, sl);
                if (s3 == HODLR_OK)
                    s3 = launch_compact_v<double, float>(Vst[l], h->ldn, Vc, h->ldn, h->d_bounds, L, l,
                                                         h->d_ranks[l], lv.rp, node_max, sl);
            } else if (h->prec == HODLR_FP64) {
                s3 = launch_compact<float, double>(Ust[l], h->ldn, Uc, h->ldn, h->d_bounds, L, l, h->d_ranks[l],
                                                   lv.rp, node_max, sl);
                if (s3 == HODLR_OK)
                    s3 = launch_compact_v<float, double>(Vst[l], h->ldn, Vc, h->ldn, h->d_bounds, L, l,
                                                         h->d_ranks[l], lv.rp, node_max, sl);
            } else {
                s3 = launch_compact<float, float>(Ust[l], h->ldn, Uc, h->ldn, h->d_bounds, L, l, h->d_ranks[l],
                                                  lv.rp, node_max, sl);
                if (s3 == HODLR_OK)
                    s3 = launch_compact_v<float, float>(Vst[l], h->ldn, Vc, h->ldn, h->d_bounds, L, l,
                                                        h->d_ranks[l], lv.rp, node_max, sl);
            }
        }
        if (s3 == HODLR_OK) s3 = plan_level(h, l, sl);
        if (s3 == HODLR_OK && factor_now) s3 = run_level(h, l, sl, share_done.data());
        if (s3 == HODLR_OK) {
            cudaEventCreateWithFlags(&share_done[l], cudaEventDisableTiming);
            cudaEventRecord(share_done[l], sl);
        }
        if (s3 != HODLR_OK) {
            cudaDeviceSynchronize();
            drop_events();
            free_temp();
            return fail(s3);
        }
    }
    // join on the caller's stream: the leaf inverses (a tree of one leaf has no
    // level to wait for them) and every level's share
    cudaStreamWaitEvent(st, ljoin, 0);
    for (int l = 1; l <= L; ++l) cudaStreamWaitEvent(st, share_done[l], 0);
    if (factor_now) {
        if (L > 0) cudaEventRecord(h->fev[1], st);
        h->factored = true;
    }
    int64_t coff = 0;
    for (int l = 1; l <= L; ++l) {
        h->lv[l].coff = coff;
        coff += h->lv[l].rp;
    }
    h->Wtot = coff;
    // compression time: from the launch to the last level's completion
    float ms = 0.f;
    for (auto e : done) {
        float t = 0.f;
        if (e && cudaEventElapsedTime(&t, e0, e) == cudaSuccess) ms = std::max(ms, t);
    }
    h->ms_compress = ms;
    // non-finite entries met by the compression (read with each level's ranks,
    // after its compression; a factorisation fault is reported by the next
    // synchronising call)
    {
        int w = aca_status;
        if (L == 0 && sync_leaf_status &&
            (cudaMemcpyAsync(&w, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                       cudaStreamSynchronize(st) != cudaSuccess)) {
            cudaDeviceSynchronize();
            drop_events();
            free_temp();
            return fail(HODLR_CUDA_ERROR);
        }
        if (w & (ST_NONFINITE | ST_RANGE | ST_TIMEOUT)) {
            cudaDeviceSynchronize();
            drop_events();
            free_temp();
            return fail(take_status(c, st));
        }
    }
    free_temp();
    drop_events();
    if (cudaGetLastError() != cudaSuccess) {
        set_error("hodlr_build: %s", cudaGetErrorString(cudaGetLastError()));
        return fail(HODLR_CUDA_ERROR);
    }
    *out = h;
    return HODLR_OK;
}

hodlr_status hodlr_build(hodlr_ctx *c, const hodlr_matrix *A, int leaf, double tol, int method, const hodlr_graph *g,
                         const hodlr_opts *o_in, hodlr_stream stream, hodlr_t **out) {
    return build_one(c, A, leaf, tol, method, g, o_in, stream, out, true);
}

hodlr_status hodlr_build_batched(hodlr_ctx *c, int nf, const hodlr_matrix *A, const int *leaf, double tol,
                                 int method, const hodlr_opts *o, hodlr_stream stream, hodlr_t **out) {
    if (!c || nf < 0 || (nf > 0 && (!A || !leaf || !out))) {
        set_error("hodlr_build_batched: invalid argument");
        return HODLR_INVALID_ARG;
    }
    if (method != HODLR_ACA) {
        set_error("hodlr_build_batched: only ACA (BDLR needs a graph per front)");
        return HODLR_INVALID_ARG;
    }
    for (int f = 0; f < nf; ++f) out[f] = nullptr;
    auto destroy_all = [&](int upto) {
        for (int q = 0; q < upto; ++q) {
            hodlr_destroy(out[q]);
            out[q] = nullptr;
        }
    };
    for (int f = 0; f < nf; ++f) {
        const hodlr_status r = build_one(c, &A[f], leaf[f], tol, method, nullptr, o, stream, &out[f], false);
        if (r != HODLR_OK) {
            destroy_all(f);
            return r;
        }
    }
    if (nf > 0) {
        // the single-leaf fronts' non-finite / range checks, for the batch at once
        cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
        int w = 0;
        if (cudaMemcpyAsync(&w, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            set_error("hodlr_build_batched: %s", cudaGetErrorString(cudaGetLastError()));
            destroy_all(nf);
            return HODLR_CUDA_ERROR;
        }
        if (w & (ST_NONFINITE | ST_RANGE | ST_TIMEOUT)) {
            const hodlr_status r = take_status(c, st);
            destroy_all(nf);
            return r;
        }
    }
    return HODLR_OK;
}

hodlr_status hodlr_factor_batched(int nf, hodlr_t *const *h, hodlr_stream stream) {
    if (nf < 0 || (nf > 0 && !h)) {
        set_error("hodlr_factor_batched: invalid argument");
        return HODLR_INVALID_ARG;
    }
    for (int f = 0; f < nf; ++f) HODLR_TRY(hodlr_factor(h[f], stream));
    return HODLR_OK;
}

hodlr_status hodlr_factor(hodlr_t *h, hodlr_stream stream) {
    if (!h) {
        set_error("hodlr_factor: NULL");
        return HODLR_INVALID_ARG;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    HODLR_TRY_CUDA(cudaSetDevice(h->ctx->device));
    if (h->factored) return HODLR_OK;   // factored during the build
    if (!h->fev[0]) {
        HODLR_TRY_CUDA(cudaEventCreate(&h->fev[0]));
        HODLR_TRY_CUDA(cudaEventCreate(&h->fev[1]));
    }
    HODLR_TRY_CUDA(cudaEventRecord(h->fev[0], st));
    HODLR_TRY(factor_impl(h, st));
    HODLR_TRY_CUDA(cudaEventRecord(h->fev[1], st));
    h->factored = true;
    return HODLR_OK;
}

hodlr_status hodlr_solve(hodlr_t *h, int s, double *X, int64_t ldx, hodlr_stream stream) {
    if (!h || !X || s <= 0 || ldx < h->n) {
        set_error("hodlr_solve: invalid argument");
        return HODLR_INVALID_ARG;
    }
    if (!h->factored) {
        set_error("hodlr_solve: not factored");
        return HODLR_NOT_FACTORED;
    }
    HODLR_TRY_CUDA(cudaSetDevice(h->ctx->device));
    return solve_impl(h, s, X, ldx, reinterpret_cast<cudaStream_t>(stream));
}

hodlr_status hodlr_matvec(hodlr_ctx *c, const hodlr_matrix *A, int s, const double *Z, int64_t ldz, double *W,
                          int64_t ldw, hodlr_stream stream) {
    if (!c || !Z || !W || s <= 0) {
        set_error("hodlr_matvec: invalid argument");
        return HODLR_INVALID_ARG;
    }
    HODLR_TRY(check_matrix(A));
    if (ldz < A->n || ldw < A->n) {
        set_error("hodlr_matvec: leading dimension < n");
        return HODLR_INVALID_ARG;
    }
    HODLR_TRY_CUDA(cudaSetDevice(c->device));
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (oz_eligible(A->n, s)) {
        // many right-hand sides: split A for this call and use the tensor cores
        const size_t ab = oz_a_bytes(A->n), zb = oz_z_bytes(A->n, s);
        void *abuf = dalloc(c, ab, st);
        void *zbuf = abuf ? dalloc(c, zb, st) : nullptr;
        if (zbuf) {
            hodlr_status r = oz_split_a(c, A->data, A->n, A->ld, abuf, st);
            if (r == HODLR_OK) r = oz_matvec(c, abuf, A->n, s, Z, ldz, W, ldw, zbuf, st);
            dfree(c, zbuf, zb, st);
            dfree(c, abuf, ab, st);
            HODLR_TRY(r);
            // a non-finite or out-of-range entry is reported here, and the flag
            // does not reach the context's next call
            return take_status(c, st);
        }
        if (abuf) dfree(c, abuf, ab, st);
        cudaGetLastError();   // too large for the slices: the double-float product
    }
    HODLR_TRY(matvec_impl(c, A->data, A->n, A->ld, s, Z, ldz, W, ldw, st));
    return take_status(c, st);
}

hodlr_status hodlr_stats_get(const hodlr_t *h, hodlr_stats *o) {
    if (!h || !o) {
        set_error("hodlr_stats_get: NULL");
        return HODLR_INVALID_ARG;
    }
    std::memset(o, 0, sizeof(*o));
    o->n = h->n;
    o->levels = h->L;
    o->leaf_max = h->bmax;
    for (int l = 1; l <= h->L; ++l) {
        o->rank_max[l - 1] = h->lv[l].rank_max;
        o->rank_pad[l - 1] = h->lv[l].rp;
        o->rank_mean[l - 1] = h->lv[l].rank_mean;
        o->cap[l - 1] = h->lv[l].cap;
    }
    o->cap_hit = h->cap_hit;
    o->bdlr_depth_max = h->bdlr_depth_max;
    const size_t pe = elem_size(h->prec);
    // U, d, V (ldn x rp each) and E (ldn x 2 rp) per level, the leaf inverses, the cores
    int64_t b = (int64_t)5 * h->ldn * h->Wtot * pe + ((int64_t)1 << h->L) * h->bmax * h->bmax * pe;
    for (int l = 0; l < h->L; ++l) b += ((int64_t)1 << l) * 4 * (int64_t)h->lv[l + 1].rp * h->lv[l + 1].rp * pe;
    o->bytes_factors = b;
    o->factored = h->factored ? 1 : 0;
    o->ms_compress = h->ms_compress;
    o->ms_factor = 0.0;
    o->core_cond_threshold = h->guard ? (h->promote ? h->cond_thr : INFINITY) : -1.0;
    if (h->factored && h->fev[1] && cudaEventSynchronize(h->fev[1]) == cudaSuccess) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, h->fev[0], h->fev[1]) == cudaSuccess) o->ms_factor = ms;
        if (h->guard) {
            std::vector<double> cv;
            std::vector<int> fv;
            for (int l = 0; l < h->L; ++l) {
                const size_t nn = (size_t)1 << l;
                cv.resize(nn);
                fv.resize(nn);
                if (cudaMemcpy(cv.data(), h->core_cond[l], nn * 8, cudaMemcpyDeviceToHost) != cudaSuccess ||
                    cudaMemcpy(fv.data(), h->core_flag[l], nn * sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
                    break;
                for (size_t i = 0; i < nn; ++i) {
                    o->core_cond_max[l] = std::max(o->core_cond_max[l], cv[i]);
                    o->cores_promoted[l] += fv[i];
                }
            }
        }
    }
    cudaGetLastError();
    return HODLR_OK;
}

hodlr_status hodlr_export_level(const hodlr_t *h, int level, double *U, double *d, double *V, int32_t *ranks,
                                int32_t *piv_rows, int32_t *piv_cols, hodlr_stream stream) {
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (!h || level < 1 || level > h->L) {
        set_error("hodlr_export_level: level out of range");
        return HODLR_INVALID_ARG;
    }
    if (d && !h->factored) {
        set_error("hodlr_export_level: d requested before hodlr_factor");
        return HODLR_NOT_FACTORED;
    }
    HODLR_TRY_CUDA(cudaSetDevice(h->ctx->device));
    const Level &lv = h->lv[level];
    const int64_t n = h->n, rp = lv.rp;
    if ((U || d || V) && rp > 0) {
        double *tmp = (double *)dalloc(h->ctx, (size_t)n * rp * 8, st);
        if (!tmp) return HODLR_OUT_OF_MEMORY;
        double *dst3[3] = {U, d, V};
        const void *src3[3] = {h->Ul[level], h->Dl[level], h->Vl[level]};
        for (int which = 0; which < 3; ++which) {
            double *dst = dst3[which];
            if (!dst) continue;
            const void *src = src3[which];
            int blocks = (int)std::min<int64_t>((n * rp + 255) / 256, 4096);
            if (h->prec == HODLR_FP64)
                to_double_kernel<double><<<blocks, 256, 0, st>>>((const double *)src, h->ldn, tmp, n, n, rp);
            else
                to_double_kernel<float><<<blocks, 256, 0, st>>>((const float *)src, h->ldn, tmp, n, n, rp);
            note_launch();
            HODLR_TRY_CUDA(cudaMemcpyAsync(dst, tmp, (size_t)n * rp * 8, cudaMemcpyDeviceToHost, st));
        }
        HODLR_TRY_CUDA(cudaStreamSynchronize(st));
        dfree(h->ctx, tmp, (size_t)n * rp * 8, st);
    }
    if (ranks) std::memcpy(ranks, lv.ranks.data(), lv.nnodes * sizeof(int32_t));
    if (piv_rows)
        HODLR_TRY_CUDA(cudaMemcpyAsync(piv_rows, h->piv_rows[level], (size_t)lv.nnodes * lv.cap * 4,
                                       cudaMemcpyDeviceToHost, st));
    if (piv_cols)
        HODLR_TRY_CUDA(cudaMemcpyAsync(piv_cols, h->piv_cols[level], (size_t)lv.nnodes * lv.cap * 4,
                                       cudaMemcpyDeviceToHost, st));
    HODLR_TRY_CUDA(cudaStreamSynchronize(st));
    return HODLR_OK;
}

hodlr_status hodlr_export_core(const hodlr_t *h, int level, double *Sinv, hodlr_stream stream) {
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (!h || level < 0 || level >= h->L || !Sinv) {
        set_error("hodlr_export_core: invalid argument");
        return HODLR_INVALID_ARG;
    }
    if (!h->factored) {
        set_error("hodlr_export_core: not factored");
        return HODLR_NOT_FACTORED;
    }
    HODLR_TRY_CUDA(cudaSetDevice(h->ctx->device));
    const int64_t s2 = 2 * (int64_t)h->lv[level + 1].rp;
    const int64_t cnt = ((int64_t)1 << level) * s2 * s2;
    if (cnt == 0) return HODLR_OK;
    double *tmp = (double *)dalloc(h->ctx, (size_t)cnt * 8, st);
    if (!tmp) return HODLR_OUT_OF_MEMORY;
    int blocks = (int)std::min<int64_t>((cnt + 255) / 256, 4096);
    if (h->prec == HODLR_FP64)
        to_double_kernel<double><<<blocks, 256, 0, st>>>((const double *)h->Sinv[level], cnt, tmp, cnt, cnt, 1);
    else
        to_double_kernel<float><<<blocks, 256, 0, st>>>((const float *)h->Sinv[level], cnt, tmp, cnt, cnt, 1);
    note_launch();
    if (h->promote && h->Sinv64[level]) {   // cores re-inverted in FP64: their FP64 inverse
        std::vector<int> fv((size_t)1 << level);
        HODLR_TRY_CUDA(cudaMemcpyAsync(fv.data(), h->core_flag[level], fv.size() * sizeof(int),
                                       cudaMemcpyDeviceToHost, st));
        HODLR_TRY_CUDA(cudaStreamSynchronize(st));
        for (size_t i = 0; i < fv.size(); ++i)
            if (fv[i])
                HODLR_TRY_CUDA(cudaMemcpyAsync(tmp + i * s2 * s2, h->Sinv64[level] + i * s2 * s2,
                                               (size_t)s2 * s2 * 8, cudaMemcpyDeviceToDevice, st));
    }
    HODLR_TRY_CUDA(cudaMemcpyAsync(Sinv, tmp, (size_t)cnt * 8, cudaMemcpyDeviceToHost, st));
    HODLR_TRY_CUDA(cudaStreamSynchronize(st));
    dfree(h->ctx, tmp, (size_t)cnt * 8, st);
    return HODLR_OK;
}

hodlr_status hodlr_export_core_cond(const hodlr_t *h, int level, double *cond, int32_t *promoted,
                                    hodlr_stream stream) {
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (!h || level < 0 || level >= h->L) {
        set_error("hodlr_export_core_cond: invalid argument");
        return HODLR_INVALID_ARG;
    }
    if (!h->factored) {
        set_error("hodlr_export_core_cond: not factored");
        return HODLR_NOT_FACTORED;
    }
    if (!h->guard) {
        set_error("hodlr_export_core_cond: the condition guard is off (negative core_cond_threshold)");
        return HODLR_INVALID_ARG;
    }
    HODLR_TRY_CUDA(cudaSetDevice(h->ctx->device));
    const size_t nn = (size_t)1 << level;
    if (cond) HODLR_TRY_CUDA(cudaMemcpyAsync(cond, h->core_cond[level], nn * 8, cudaMemcpyDeviceToHost, st));
    if (promoted)
        HODLR_TRY_CUDA(cudaMemcpyAsync(promoted, h->core_flag[level], nn * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    HODLR_TRY_CUDA(cudaStreamSynchronize(st));
    return HODLR_OK;
}

hodlr_status hodlr_precond_error(hodlr_t *h, int k, const double *Omega, int64_t ldo, double *out, hodlr_stream stream) {
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (!h || !Omega || !out || k <= 0 || ldo < h->n) {
        set_error("hodlr_precond_error: invalid argument");
        return HODLR_INVALID_ARG;
    }
    if (!h->factored) {
        set_error("hodlr_precond_error: not factored");
        return HODLR_NOT_FACTORED;
    }
    if (!h->A) {
        set_error("hodlr_precond_error: the object holds no matrix A (restored without one)");
        return HODLR_INVALID_ARG;
    }
    HODLR_TRY_CUDA(cudaSetDevice(h->ctx->device));
    const int64_t n = h->n;
    double *T = (double *)dalloc(h->ctx, (size_t)n * k * 8, st);
    if (!T) return HODLR_OUT_OF_MEMORY;
    hodlr_status s = matvec_impl(h->ctx, h->A, n, h->lda, k, Omega, ldo, T, n, st);
    if (s == HODLR_OK) s = solve_impl(h, k, T, n, st);
    if (s != HODLR_OK) {
        dfree(h->ctx, T, (size_t)n * k * 8, st);
        return s;
    }
    std::vector<double> ht((size_t)n * k), ho((size_t)n * k);
    cudaMemcpyAsync(ht.data(), T, (size_t)n * k * 8, cudaMemcpyDeviceToHost, st);
    cudaMemcpy2DAsync(ho.data(), n * 8, Omega, ldo * 8, n * 8, k, cudaMemcpyDeviceToHost, st);
    HODLR_TRY_CUDA(cudaStreamSynchronize(st));
    dfree(h->ctx, T, (size_t)n * k * 8, st);
    double num = 0, den = 0;
    for (size_t e = 0; e < ht.size(); ++e) {
        const double d = ho[e] - ht[e];
        num += d * d;
        den += ho[e] * ho[e];
    }
    *out = den > 0 ? std::sqrt(num / den) : 0.0;
    return take_status(h->ctx, st);
}

}  // extern "C"
