// Saving a factored HODLR matrix to host memory and restoring it
// (hodlr_save / hodlr_load).
//
// The image holds the object's scalars and per-level metadata, the contents of
// every device buffer the object owns, and each device pointer of the object
// as (buffer index, byte offset).  Loading allocates the same buffers, copies
// the contents back and rebuilds the pointers, so the restored object holds
// the same factors bit for bit.  The recorded factorisation
// plan is not part of the image: a restored object is factored and solves,
// but is not factored again.
#include <cstring>
#include <vector>

#include "internal.cuh"

namespace hodlr {
namespace {

constexpr uint64_t MAGIC = 0x31524c444f48ull;   // "HODLR1"
constexpr uint32_t VERSION = 1;

struct Ref {
    int32_t buf;      // -1: null
    uint64_t off;
};

struct Writer {
    std::vector<char> out;
    template <typename T>
    void put(const T &v) {
        const char *p = reinterpret_cast<const char *>(&v);
        out.insert(out.end(), p, p + sizeof(T));
    }
    void bytes(const void *p, size_t n) {
        const char *c = reinterpret_cast<const char *>(p);
        out.insert(out.end(), c, c + n);
    }
};

struct Reader {
    const char *p;
    size_t left;
    bool ok = true;
    template <typename T>
    T get() {
        T v{};
        if (left < sizeof(T)) {
            ok = false;
            return v;
        }
        std::memcpy(&v, p, sizeof(T));
        p += sizeof(T);
        left -= sizeof(T);
        return v;
    }
    const char *take(size_t n) {
        if (left < n) {
            ok = false;
            return nullptr;
        }
        const char *q = p;
        p += n;
        left -= n;
        return q;
    }
};

// (buffer, offset) of a device pointer inside the object's owned buffers
Ref ref_of(const hodlr_t *h, const void *ptr) {
    if (!ptr) return Ref{-1, 0};
    const char *c = reinterpret_cast<const char *>(ptr);
    for (size_t b = 0; b < h->owned.size(); ++b) {
        const char *p = reinterpret_cast<const char *>(h->owned[b].p);
        if (c >= p && c < p + h->owned[b].bytes) return Ref{(int32_t)b, (uint64_t)(c - p)};
    }
    return Ref{-2, 0};   // not owned: cannot be saved
}

// Every device pointer of the object, in a fixed order (save and load walk it alike).
template <typename F>
void for_each_pointer(hodlr_t *h, F &&f) {
    f(reinterpret_cast<void **>(&h->d_bounds));
    f(reinterpret_cast<void **>(&h->leafinv));
    f(reinterpret_cast<void **>(const_cast<int4 **>(&h->d_tiles)));
    f(reinterpret_cast<void **>(&h->d_tile_first));
    f(reinterpret_cast<void **>(&h->dinv));
    for (auto *v : {&h->Ul, &h->Dl, &h->El, &h->Vl, &h->Vql, &h->Eql, &h->Sinv})
        for (auto &p : *v) f(&p);
    for (auto *v : {&h->vscale, &h->escale})
        for (auto &p : *v) f(reinterpret_cast<void **>(&p));
    for (auto *v : {&h->piv_rows, &h->piv_cols, &h->d_ranks})
        for (auto &p : *v) f(reinterpret_cast<void **>(&p));
    for (auto &p : h->core_cond) f(reinterpret_cast<void **>(&p));
    for (auto &p : h->core_flag) f(reinterpret_cast<void **>(&p));
    for (auto &p : h->core_count) f(reinterpret_cast<void **>(&p));
    for (auto &p : h->Sinv64) f(reinterpret_cast<void **>(&p));
}

template <typename T>
void put_vec(Writer &w, const std::vector<T> &v) {
    w.put<uint64_t>(v.size());
    w.bytes(v.data(), v.size() * sizeof(T));
}

template <typename T>
bool get_vec(Reader &r, std::vector<T> &v) {
    const uint64_t n = r.get<uint64_t>();
    if (!r.ok || n > (1ull << 40) / sizeof(T)) return false;
    const char *p = r.take(n * sizeof(T));
    if (!p) return false;
    v.resize(n);
    std::memcpy(v.data(), p, n * sizeof(T));
    return true;
}

// The image of h (scalars, metadata, pointer table, buffer sizes), without the
// buffer contents; `contents` then follow in buffer order.
hodlr_status header(const hodlr_t *hc, Writer &w) {
    hodlr_t *h = const_cast<hodlr_t *>(hc);
    w.put(MAGIC);
    w.put(VERSION);
    w.put<int64_t>(h->n);
    w.put<int32_t>(h->L);
    w.put<int32_t>(h->bmax);
    w.put<int32_t>(h->prec);
    w.put<int32_t>(h->store);
    w.put<int32_t>(h->cprec);
    w.put<int32_t>(h->method);
    w.put<double>(h->tol);
    w.put<int32_t>(h->rank_cap);
    w.put<int32_t>(h->cap_hit);
    w.put<int64_t>(h->ldn);
    w.put<int64_t>(h->Wtot);
    w.put<int32_t>(h->ntiles);
    w.put<int32_t>(h->sym);
    w.put<uint8_t>(h->diag);
    w.put<uint8_t>(h->guard);
    w.put<uint8_t>(h->promote);
    w.put<double>(h->cond_thr);
    w.put<double>(h->ms_compress);
    put_vec(w, h->bounds);
    w.put<uint64_t>(h->lv.size());
    for (auto &l : h->lv) {
        w.put<int32_t>(l.nnodes);
        w.put<int32_t>(l.rp);
        w.put<int64_t>(l.coff);
        w.put<int32_t>(l.cap);
        w.put<int32_t>(l.rank_max);
        w.put<double>(l.rank_mean);
        put_vec(w, l.ranks);
    }
    // vector lengths of the pointer table, then the table
    for (auto *v : {&h->Ul, &h->Dl, &h->El, &h->Vl, &h->Vql, &h->Eql, &h->Sinv}) w.put<uint64_t>(v->size());
    w.put<uint64_t>(h->vscale.size());
    w.put<uint64_t>(h->escale.size());
    w.put<uint64_t>(h->piv_rows.size());
    w.put<uint64_t>(h->piv_cols.size());
    w.put<uint64_t>(h->d_ranks.size());
    w.put<uint64_t>(h->core_cond.size());
    w.put<uint64_t>(h->core_flag.size());
    w.put<uint64_t>(h->core_count.size());
    w.put<uint64_t>(h->Sinv64.size());
    bool bad = false;
    for_each_pointer(h, [&](void **pp) {
        const Ref r = ref_of(h, *pp);
        if (r.buf == -2) bad = true;
        w.put(r);
    });
    if (bad) {
        set_error("hodlr_save: a device pointer of the object lies outside its buffers");
        return HODLR_INVALID_ARG;
    }
    w.put<uint64_t>(h->owned.size());
    for (auto &b : h->owned) w.put<uint64_t>(b.bytes);
    return HODLR_OK;
}

}  // namespace
}  // namespace hodlr

using namespace hodlr;

extern "C" {

hodlr_status hodlr_save(const hodlr_t *h, void *buf, size_t bytes, size_t *needed, hodlr_stream stream) {
    if (!h || !needed) {
        set_error("hodlr_save: NULL argument");
        return HODLR_INVALID_ARG;
    }
    if (!h->factored) {
        set_error("hodlr_save: not factored");
        return HODLR_NOT_FACTORED;
    }
    Writer w;
    HODLR_TRY(header(h, w));
    size_t total = w.out.size();
    for (auto &b : h->owned) total += b.bytes;
    *needed = total;
    if (!buf) return HODLR_OK;   // size query
    if (bytes < total) {
        set_error("hodlr_save: buffer of %zu bytes, %zu needed", bytes, total);
        return HODLR_RANGE;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    HODLR_TRY_CUDA(cudaSetDevice(h->ctx->device));
    HODLR_TRY_CUDA(cudaStreamSynchronize(st));
    HODLR_TRY_CUDA(cudaDeviceSynchronize());   // the factorisation's side streams
    char *o = reinterpret_cast<char *>(buf);
    std::memcpy(o, w.out.data(), w.out.size());
    o += w.out.size();
    for (auto &b : h->owned) {
        HODLR_TRY_CUDA(cudaMemcpyAsync(o, b.p, b.bytes, cudaMemcpyDeviceToHost, st));
        o += b.bytes;
    }
    HODLR_TRY_CUDA(cudaStreamSynchronize(st));
    return HODLR_OK;
}

hodlr_status hodlr_load(hodlr_ctx *c, const hodlr_matrix *A, const void *buf, size_t bytes, hodlr_stream stream,
                        hodlr_t **out) {
    if (!c || !buf || !out) {
        set_error("hodlr_load: NULL argument");
        return HODLR_INVALID_ARG;
    }
    Reader r{reinterpret_cast<const char *>(buf), bytes};
    if (r.get<uint64_t>() != MAGIC || r.get<uint32_t>() != VERSION || !r.ok) {
        set_error("hodlr_load: not a saved HODLR matrix of this version");
        return HODLR_INVALID_ARG;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    HODLR_TRY_CUDA(cudaSetDevice(c->device));
    hodlr_t *h = new hodlr_t();
    h->ctx = c;
    auto fail = [&](const char *why) {
        set_error("hodlr_load: %s", why);
        hodlr_destroy(h);
        return HODLR_INVALID_ARG;
    };
    h->n = r.get<int64_t>();
    h->L = r.get<int32_t>();
    h->bmax = r.get<int32_t>();
    h->prec = r.get<int32_t>();
    h->store = r.get<int32_t>();
    h->cprec = r.get<int32_t>();
    h->method = r.get<int32_t>();
    h->tol = r.get<double>();
    h->rank_cap = r.get<int32_t>();
    h->cap_hit = r.get<int32_t>();
    h->ldn = r.get<int64_t>();
    h->Wtot = r.get<int64_t>();
    h->ntiles = r.get<int32_t>();
    h->sym = r.get<int32_t>();
    h->diag = r.get<uint8_t>() != 0;
    h->guard = r.get<uint8_t>() != 0;
    h->promote = r.get<uint8_t>() != 0;
    h->cond_thr = r.get<double>();
    h->ms_compress = r.get<double>();
    if (!r.ok || h->L < 0 || h->L >= HODLR_MAX_LEVELS || h->n <= 0) return fail("corrupt header");
    if (A && (A->n != h->n || !A->data || A->ld < A->n)) return fail("A does not match the saved matrix");
    if (!get_vec(r, h->bounds)) return fail("corrupt leaf bounds");
    const uint64_t nlv = r.get<uint64_t>();
    if (!r.ok || nlv != (uint64_t)h->L + 1) return fail("corrupt level table");
    h->lv.resize(nlv);
    for (auto &l : h->lv) {
        l.nnodes = r.get<int32_t>();
        l.rp = r.get<int32_t>();
        l.coff = r.get<int64_t>();
        l.cap = r.get<int32_t>();
        l.rank_max = r.get<int32_t>();
        l.rank_mean = r.get<double>();
        if (!get_vec(r, l.ranks)) return fail("corrupt ranks");
    }
    for (auto *v : {&h->Ul, &h->Dl, &h->El, &h->Vl, &h->Vql, &h->Eql, &h->Sinv}) {
        const uint64_t k = r.get<uint64_t>();
        if (k > 64) return fail("corrupt pointer table");
        v->assign(k, nullptr);
    }
    auto sized = [&](auto &v) {
        const uint64_t k = r.get<uint64_t>();
        if (k > 64) return false;
        v.assign(k, nullptr);
        return true;
    };
    if (!sized(h->vscale) || !sized(h->escale) || !sized(h->piv_rows) || !sized(h->piv_cols) || !sized(h->d_ranks) ||
        !sized(h->core_cond) || !sized(h->core_flag) || !sized(h->core_count) || !sized(h->Sinv64) || !r.ok)
        return fail("corrupt pointer table");
    std::vector<Ref> refs;
    for_each_pointer(h, [&](void **) { refs.push_back(r.get<Ref>()); });
    const uint64_t nb = r.get<uint64_t>();
    if (!r.ok || nb > (1u << 20)) return fail("corrupt buffer table");
    std::vector<uint64_t> sizes(nb);
    for (auto &s : sizes) s = r.get<uint64_t>();
    if (!r.ok) return fail("corrupt buffer table");
    for (uint64_t b = 0; b < nb; ++b) {
        const char *src = r.take(sizes[b]);
        if (!src) return fail("truncated image");
        void *p = own(h, sizes[b], st);
        if (!p) {
            set_error("hodlr_load: out of device memory");
            hodlr_destroy(h);
            return HODLR_OUT_OF_MEMORY;
        }
        if (cudaMemcpyAsync(p, src, sizes[b], cudaMemcpyHostToDevice, st) != cudaSuccess) {
            cudaGetLastError();
            set_error("hodlr_load: copy to the device failed");
            hodlr_destroy(h);
            return HODLR_CUDA_ERROR;
        }
    }
    size_t k = 0;
    bool bad = false;
    for_each_pointer(h, [&](void **pp) {
        const Ref ref = refs[k++];
        if (ref.buf < 0) {
            *pp = nullptr;
        } else if ((uint64_t)ref.buf >= nb || ref.off >= sizes[ref.buf]) {
            bad = true;
        } else {
            *pp = reinterpret_cast<char *>(h->owned[ref.buf].p) + ref.off;
        }
    });
    if (bad) return fail("pointer outside its buffer");
    h->A = A ? A->data : nullptr;
    h->lda = A ? A->ld : 0;
    h->factored = true;
    HODLR_TRY_CUDA(cudaStreamSynchronize(st));
    *out = h;
    return HODLR_OK;
}

}  // extern "C"
