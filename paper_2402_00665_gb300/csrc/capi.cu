// capi.cu -- the C ABI of include/lbvh.h: argument checks, device storage of
// a tree, and the order of kernel launches for a build and a query. No
// arithmetic of the method happens here; every step runs in the kernels.
#include <atomic>
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <vector>

#include "lbvh_internal.cuh"

namespace {

thread_local char g_last_error[256] = "";

void note_cuda(cudaError_t e) {
    std::snprintf(g_last_error, sizeof g_last_error, "%s: %s", cudaGetErrorName(e),
                  cudaGetErrorString(e));
}

#define LBVH_CUDA(expr)                                                    \
    do {                                                                   \
        cudaError_t e_ = (expr);                                           \
        if (e_ != cudaSuccess) {                                           \
            note_cuda(e_);                                                 \
            return e_ == cudaErrorMemoryAllocation ? LBVH_ERR_OOM : LBVH_ERR_CUDA; \
        }                                                                  \
    } while (0)

#define LBVH_LAUNCHED() LBVH_CUDA(cudaGetLastError())

// A device buffer that only grows. Growth frees the old block and allocates
// a new one on the stream (stream-ordered allocator); `zero` clears new
// storage (used for scratch that the kernels keep clean themselves).
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;

    cudaError_t ensure(size_t want, cudaStream_t s, bool zero = false) {
        if (want <= bytes) return cudaSuccess;
        if (p) cudaFreeAsync(p, s);
        p = nullptr;
        bytes = 0;
        cudaError_t e = cudaMallocAsync(&p, want, s);
        if (e != cudaSuccess) {
            p = nullptr;
            return e;
        }
        bytes = want;
        if (zero) e = cudaMemsetAsync(p, 0, want, s);
        return e;
    }
    void release(cudaStream_t s) {
        if (p) cudaFreeAsync(p, s);
        p = nullptr;
        bytes = 0;
    }
    template <typename T>
    T *as() const {
        return static_cast<T *>(p);
    }
};

bool valid_bits(int bits) { return bits >= 3 && bits <= 63 && bits % 3 == 0; }

lbvh_status flags_status(uint32_t flags) {
    if (flags & lbvh::kFlagTimeout) return LBVH_ERR_TIMEOUT;
    if (flags & lbvh::kFlagNonfinite) return LBVH_ERR_NONFINITE;
    if (flags & lbvh::kFlagCorrupt) return LBVH_ERR_CORRUPT;
    return LBVH_OK;
}

// Event pairs around each stage (see LBVH_STAGE_*), recorded only when on.
struct Profiler {
    bool on = false;
    bool ready = false;
    cudaEvent_t ev[LBVH_STAGE_COUNT][2] = {};
    bool recorded[LBVH_STAGE_COUNT] = {};

    cudaError_t enable(bool want) {
        on = want;
        if (!on || ready) return cudaSuccess;
        for (auto &pair : ev)
            for (auto &e : pair) {
                cudaError_t r = cudaEventCreate(&e);
                if (r != cudaSuccess) return r;
            }
        ready = true;
        return cudaSuccess;
    }
    void clear(int lo, int hi) {
        for (int k = lo; k < hi; ++k) recorded[k] = false;
    }
    void begin(int st, cudaStream_t s) {
        if (on) cudaEventRecord(ev[st][0], s);
    }
    void end(int st, cudaStream_t s) {
        if (!on) return;
        cudaEventRecord(ev[st][1], s);
        recorded[st] = true;
    }
    void release() {
        if (!ready) return;
        for (auto &pair : ev)
            for (auto &e : pair) cudaEventDestroy(e);
        ready = false;
    }
};

}  // namespace

struct lbvh_tree_s {
    cudaStream_t stream = nullptr;  // stream of the last build
    cudaEvent_t built = nullptr;    // recorded after the last build
    int64_t n = 0;
    int kind = LBVH_PRIM_POINTS;
    int bits = 0;
    bool has_build = false;
    bool sorted_in_b = false;
    bool store_dirty = false;  // a failed build may have left store words set
    DevBuf keys[2], vals[2];
    DevBuf nodes, store, lookback, hist, partials, bounds, ctl;
    DevBuf counts, tile_sums, overflow, slots;
    DevBuf qkeys[2], qvals[2], qlookback;  // Morton order of the queries
    const float *prims_ptr = nullptr;      // the last build's input (self-queries)
    lbvh::Control *h_ctl = nullptr;  // pinned mirror of the control block
    Profiler prof;

    const uint64_t *sorted_codes() const { return keys[sorted_in_b ? 1 : 0].as<uint64_t>(); }
    const uint32_t *perm() const { return vals[sorted_in_b ? 1 : 0].as<uint32_t>(); }
    lbvh::Control *dctl() const { return ctl.as<lbvh::Control>(); }
    lbvh::TreeView view() const {
        return lbvh::TreeView{inodes(), leaves(), n, kind};
    }
    // internal records, then the leaves (one allocation)
    float4 *inodes() const { return nodes.as<float4>(); }
    float4 *leaves() const { return nodes.as<float4>() + 2 * (n > 0 ? n - 1 : 0);
    }
};

namespace lbvh {

static std::atomic<unsigned long long> g_launches{0};

void count_launches(int k) { g_launches.fetch_add((unsigned long long)k, std::memory_order_relaxed); }

int device_sm_count() {
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    return sms;
}

}  // namespace lbvh

namespace {

// Storage for a tree of n primitives; the control block and `store` are
// zeroed when first allocated and kept clean by the kernels afterwards.
lbvh_status reserve_tree(lbvh_tree_s *t, int64_t n, int kind, cudaStream_t s) {
    using namespace lbvh;
    const size_t un = (size_t)n, ui = (size_t)(n > 0 ? n - 1 : 0);
    const int64_t tiles = sort_tiles(n);
    LBVH_CUDA(t->ctl.ensure(sizeof(Control), s, true));
    for (int k = 0; k < 2; ++k) {
        LBVH_CUDA(t->keys[k].ensure(un * 8, s));
        LBVH_CUDA(t->vals[k].ensure(un * 4, s));
    }
    LBVH_CUDA(t->nodes.ensure(ui * 32 + leaf_float4s(n, kind) * 16, s));
    LBVH_CUDA(t->store.ensure(ui * 8, s, true));
    LBVH_CUDA(t->lookback.ensure((size_t)tiles * kRadix * 4 * 2, s));
    LBVH_CUDA(t->hist.ensure((size_t)kMaxPasses * kRadix * 4, s));
    LBVH_CUDA(t->partials.ensure((size_t)bounds_blocks(n) * 8 * 4, s));
    LBVH_CUDA(t->bounds.ensure(6 * 4, s));
    if (!t->h_ctl) LBVH_CUDA(cudaMallocHost(&t->h_ctl, sizeof(Control)));
    return LBVH_OK;
}

lbvh_status check_build_args(lbvh_tree_t t, const void *prims, int64_t n, int kind) {
    if (!t || n < 0 || n > LBVH_MAX_PRIMS) return LBVH_ERR_INVALID;
    if (kind != LBVH_PRIM_POINTS && kind != LBVH_PRIM_BOXES) return LBVH_ERR_INVALID;
    if (n > 0 && !prims) return LBVH_ERR_INVALID;
    return LBVH_OK;
}

lbvh_status finish_build(lbvh_tree_t t, cudaStream_t s) {
    if (!t->built) LBVH_CUDA(cudaEventCreateWithFlags(&t->built, cudaEventDisableTiming));
    LBVH_CUDA(cudaEventRecord(t->built, s));
    t->stream = s;
    t->has_build = true;
    return LBVH_OK;
}

lbvh_status read_control(lbvh_tree_t t, cudaStream_t s) {
    LBVH_CUDA(cudaMemcpyAsync(t->h_ctl, t->ctl.p, sizeof(lbvh::Control), cudaMemcpyDeviceToHost, s));
    LBVH_CUDA(cudaStreamSynchronize(s));
    if (t->h_ctl->build_flags & (lbvh::kFlagTimeout | lbvh::kFlagCorrupt)) t->store_dirty = true;
    return LBVH_OK;
}

constexpr int64_t kOrderMinQueries = 2048;  // below this, walk in input order
constexpr int kOrderBits = 30;              // Morton bits of the query order

// The order in which threads take the queries: the Morton order of the query
// centres inside the tree's bounds (encode + radix sort, the build's own
// kernels). Queries that are the primitives of the last build (same pointer
// and count) reuse the build's permutation. Order only changes speed, never
// results.
lbvh_status query_order(lbvh_tree_t t, lbvh::QueryArgs &qa, cudaStream_t s) {
    using namespace lbvh;
    qa.order = nullptr;
    if (qa.nq < kOrderMinQueries || t->n == 0) return LBVH_OK;
    const bool same_points = qa.qkind == LBVH_Q_SPHERE && t->kind == LBVH_PRIM_POINTS;
    const bool same_boxes = qa.qkind == LBVH_Q_BOX && t->kind == LBVH_PRIM_BOXES;
    if (qa.queries == t->prims_ptr && qa.nq == t->n && (same_points || same_boxes)) {
        qa.order = t->perm();
        return LBVH_OK;
    }
    const size_t unq = (size_t)qa.nq;
    const int passes = sort_passes(kOrderBits);
    for (int k = 0; k < 2; ++k) {
        LBVH_CUDA(t->qkeys[k].ensure(unq * 8, s));
        LBVH_CUDA(t->qvals[k].ensure(unq * 4, s));
    }
    LBVH_CUDA(t->qlookback.ensure((size_t)sort_tiles(qa.nq) * kRadix * 4 * 2, s));
    LBVH_CUDA(cudaMemsetAsync(t->hist.p, 0, (size_t)passes * kRadix * 4, s));
    const int as_prims = qa.qkind == LBVH_Q_SPHERE ? LBVH_PRIM_POINTS : LBVH_PRIM_BOXES;
    launch_encode(qa.queries, qa.nq, as_prims, kOrderBits, t->bounds.as<float>(),
                  t->qkeys[0].as<uint64_t>(), t->hist.as<uint32_t>(), 1, s);
    LBVH_LAUNCHED();
    SortScratch scratch{t->hist.as<uint32_t>(), t->qlookback.as<uint32_t>(), sort_tiles(qa.nq) * kRadix};
    const bool in_b = run_onesweep(t->qkeys[0].as<uint64_t>(), t->qvals[0].as<uint32_t>(), true,
                                   t->qkeys[1].as<uint64_t>(), t->qvals[1].as<uint32_t>(), qa.nq, passes,
                                   scratch, t->dctl(), s);
    LBVH_LAUNCHED();
    qa.order = t->qvals[in_b ? 1 : 0].as<uint32_t>();
    return LBVH_OK;
}

lbvh::QueryScratch query_scratch(lbvh_tree_t t) {
    return lbvh::QueryScratch{t->counts.as<uint2>(), t->slots.as<uint32_t>(),
                              t->overflow.as<uint32_t>()};
}

// The query up to the hit count: order, collecting walk, scan; synchronises `s`.
lbvh_status query_count(lbvh_tree_t t, lbvh::QueryArgs &qa, int64_t *d_offsets,
                        cudaStream_t s, uint64_t *total) {
    using namespace lbvh;
    LBVH_CUDA(cudaStreamWaitEvent(s, t->built, 0));
    const size_t unq = (size_t)qa.nq;
    LBVH_CUDA(t->counts.ensure(unq * 8 + 8, s));
    LBVH_CUDA(t->overflow.ensure(unq * 4 + 4, s));
    LBVH_CUDA(t->tile_sums.ensure((size_t)scan_tile_count(qa.nq) * 8 + 8, s));
    LBVH_CUDA(t->slots.ensure(unq * kQueryBufferHits * 4 + 16, s));
    Control *c = t->dctl();
    LBVH_CUDA(cudaMemsetAsync(&c->query_flags, 0, offsetof(Control, pad) - offsetof(Control, query_flags), s));
    t->prof.clear(LBVH_STAGE_QCOUNT, LBVH_STAGE_COUNT);
    t->prof.begin(LBVH_STAGE_QORDER, s);
    lbvh_status ost = query_order(t, qa, s);
    if (ost != LBVH_OK) return ost;
    t->prof.end(LBVH_STAGE_QORDER, s);
    const QueryScratch qs = query_scratch(t);
    t->prof.begin(LBVH_STAGE_QCOUNT, s);
    launch_query_collect(t->view(), qa, qs, c, s);
    t->prof.end(LBVH_STAGE_QCOUNT, s);
    LBVH_LAUNCHED();
    t->prof.begin(LBVH_STAGE_QSCAN, s);
    launch_exclusive_scan(qs.count_pos, qa.nq, d_offsets, t->tile_sums.as<int64_t>(), c, s);
    t->prof.end(LBVH_STAGE_QSCAN, s);
    LBVH_LAUNCHED();
    lbvh_status st = read_control(t, s);
    if (st != LBVH_OK) return st;
    st = flags_status(t->h_ctl->build_flags);
    if (st == LBVH_OK) st = flags_status(t->h_ctl->query_flags);
    *total = t->h_ctl->total;
    return st;
}

lbvh_status query_fill(lbvh_tree_t t, const lbvh::QueryArgs &qa, const int64_t *d_offsets,
                       uint32_t *d_hits, cudaStream_t s) {
    using namespace lbvh;
    if (t->h_ctl->total == 0) return LBVH_OK;
    const QueryScratch qs = query_scratch(t);
    t->prof.begin(LBVH_STAGE_QFILL, s);
    launch_query_copy(qa, qs, d_offsets, d_hits, s);
    t->prof.end(LBVH_STAGE_QFILL, s);
    LBVH_LAUNCHED();
    if (t->h_ctl->overflow_filled > 0) {
        t->prof.begin(LBVH_STAGE_QFIXUP, s);
        launch_query_overflow(t->view(), qa, qs, t->h_ctl->overflow_filled, d_offsets, d_hits, s);
        t->prof.end(LBVH_STAGE_QFIXUP, s);
        LBVH_LAUNCHED();
    }
    return LBVH_OK;
}

lbvh_status check_query_args(lbvh_tree_t t, const float *q, int64_t nq, int qkind,
                             const float *radii, float radius) {
    if (!t || !t->has_build || nq < 0 || nq > LBVH_MAX_PRIMS) return LBVH_ERR_INVALID;
    if (qkind != LBVH_Q_SPHERE && qkind != LBVH_Q_BOX) return LBVH_ERR_INVALID;
    if (nq > 0 && !q) return LBVH_ERR_INVALID;
    if (qkind == LBVH_Q_SPHERE && !radii && !(std::isfinite(radius) && radius >= 0.0f))
        return LBVH_ERR_INVALID;
    return LBVH_OK;
}

}  // namespace

extern "C" {

lbvh_status lbvh_tree_create(lbvh_tree_t *out) {
    if (!out) return LBVH_ERR_INVALID;
    *out = new (std::nothrow) lbvh_tree_s();
    return *out ? LBVH_OK : LBVH_ERR_OOM;
}

void lbvh_tree_destroy(lbvh_tree_t t) {
    if (!t) return;
    if (t->has_build) cudaStreamSynchronize(t->stream);
    cudaStream_t s = t->stream;
    for (DevBuf *b : {&t->keys[0], &t->keys[1], &t->vals[0], &t->vals[1], &t->nodes,
                      &t->store, &t->lookback, &t->hist, &t->partials, &t->bounds, &t->ctl,
                      &t->counts, &t->tile_sums, &t->overflow, &t->qkeys[0], &t->qkeys[1],
                      &t->qvals[0], &t->qvals[1], &t->qlookback, &t->slots})
        b->release(s);
    cudaStreamSynchronize(s);
    if (t->h_ctl) cudaFreeHost(t->h_ctl);
    if (t->built) cudaEventDestroy(t->built);
    t->prof.release();
    delete t;
}

lbvh_status lbvh_build(lbvh_tree_t t, const float *d_prims, int64_t n, int kind, int morton_bits,
                       lbvh_stream_t stream) {
    using namespace lbvh;
    lbvh_status st = check_build_args(t, d_prims, n, kind);
    if (st != LBVH_OK) return st;
    if (!valid_bits(morton_bits)) return LBVH_ERR_INVALID;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    st = reserve_tree(t, n, kind, s);
    if (st != LBVH_OK) return st;
    t->n = n;
    t->kind = kind;
    t->bits = morton_bits;
    t->prims_ptr = d_prims;
    Control *c = t->dctl();
    LBVH_CUDA(cudaMemsetAsync(&c->build_flags, 0, sizeof(uint32_t), s));
    if (t->store_dirty && t->store.bytes) {
        LBVH_CUDA(cudaMemsetAsync(t->store.p, 0, t->store.bytes, s));
        t->store_dirty = false;
    }
    t->prof.clear(0, LBVH_STAGE_QCOUNT);
    if (n > 0) {
        const int passes = sort_passes(morton_bits);
        LBVH_CUDA(cudaMemsetAsync(t->hist.p, 0, (size_t)passes * kRadix * 4, s));
        t->prof.begin(LBVH_STAGE_BOUNDS, s);
        launch_bounds(d_prims, n, kind, t->partials.as<float>(), t->bounds.as<float>(), c, s);
        t->prof.end(LBVH_STAGE_BOUNDS, s);
        LBVH_LAUNCHED();
        t->prof.begin(LBVH_STAGE_ENCODE, s);
        launch_encode(d_prims, n, kind, morton_bits, t->bounds.as<float>(), t->keys[0].as<uint64_t>(),
                      t->hist.as<uint32_t>(), 1, s);
        t->prof.end(LBVH_STAGE_ENCODE, s);
        LBVH_LAUNCHED();
        SortScratch scratch{t->hist.as<uint32_t>(), t->lookback.as<uint32_t>(), sort_tiles(n) * kRadix};
        t->sorted_in_b = run_onesweep(t->keys[0].as<uint64_t>(), t->vals[0].as<uint32_t>(), true,
                                      t->keys[1].as<uint64_t>(), t->vals[1].as<uint32_t>(), n, passes,
                                      scratch, c, s, t->prof.on ? &t->prof.ev[LBVH_STAGE_SORT0] : nullptr);
        if (t->prof.on)
            for (int p = 0; p < passes; ++p) t->prof.recorded[LBVH_STAGE_SORT0 + p] = true;
        LBVH_LAUNCHED();
        t->prof.begin(LBVH_STAGE_CONSTRUCT, s);
        launch_construct(t->sorted_codes(), t->perm(), d_prims, n, kind, t->inodes(),
                         t->leaves(), t->store.as<unsigned long long>(), &c->build_flags, s);
        t->prof.end(LBVH_STAGE_CONSTRUCT, s);
        LBVH_LAUNCHED();
    }
    return finish_build(t, s);
}

lbvh_status lbvh_build_from_sorted(lbvh_tree_t t, const uint64_t *d_sorted_codes,
                                   const uint32_t *d_perm, const float *d_prims, int64_t n,
                                   int kind, lbvh_stream_t stream) {
    using namespace lbvh;
    lbvh_status st = check_build_args(t, d_prims, n, kind);
    if (st != LBVH_OK) return st;
    if (n > 0 && (!d_sorted_codes || !d_perm)) return LBVH_ERR_INVALID;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    st = reserve_tree(t, n, kind, s);
    if (st != LBVH_OK) return st;
    t->n = n;
    t->kind = kind;
    t->bits = 0;
    t->prims_ptr = d_prims;
    t->sorted_in_b = false;
    Control *c = t->dctl();
    LBVH_CUDA(cudaMemsetAsync(&c->build_flags, 0, sizeof(uint32_t), s));
    if (t->store_dirty && t->store.bytes) {
        LBVH_CUDA(cudaMemsetAsync(t->store.p, 0, t->store.bytes, s));
        t->store_dirty = false;
    }
    if (n > 0) {
        LBVH_CUDA(cudaMemcpyAsync(t->keys[0].p, d_sorted_codes, (size_t)n * 8, cudaMemcpyDeviceToDevice, s));
        LBVH_CUDA(cudaMemcpyAsync(t->vals[0].p, d_perm, (size_t)n * 4, cudaMemcpyDeviceToDevice, s));
        launch_bounds(d_prims, n, kind, t->partials.as<float>(), t->bounds.as<float>(), c, s);
        LBVH_LAUNCHED();
        launch_construct(t->sorted_codes(), t->perm(), d_prims, n, kind, t->inodes(),
                         t->leaves(), t->store.as<unsigned long long>(), &c->build_flags, s);
        LBVH_LAUNCHED();
    }
    return finish_build(t, s);
}

lbvh_status lbvh_tree_status(lbvh_tree_t t) {
    if (!t || !t->has_build) return LBVH_ERR_INVALID;
    lbvh_status st = read_control(t, t->stream);
    if (st != LBVH_OK) return st;
    return flags_status(t->h_ctl->build_flags);
}

lbvh_status lbvh_tree_size(lbvh_tree_t t, int64_t *n) {
    if (!t || !n) return LBVH_ERR_INVALID;
    *n = t->has_build ? t->n : 0;
    return LBVH_OK;
}

lbvh_status lbvh_tree_bytes(lbvh_tree_t t, uint64_t *bytes) {
    if (!t || !bytes) return LBVH_ERR_INVALID;
    uint64_t b = 0;
    for (const DevBuf *d : {&t->keys[0], &t->keys[1], &t->vals[0], &t->vals[1], &t->nodes,
                            &t->store, &t->lookback, &t->hist, &t->partials, &t->bounds, &t->ctl,
                            &t->counts, &t->tile_sums, &t->overflow, &t->qkeys[0], &t->qkeys[1],
                            &t->qvals[0], &t->qvals[1], &t->qlookback, &t->slots})
        b += d->bytes;
    *bytes = b;
    return LBVH_OK;
}

lbvh_status lbvh_tree_export(lbvh_tree_t t, uint32_t *h_perm, uint64_t *h_sorted_codes,
                             int32_t *h_left, int32_t *h_skip_internal, int32_t *h_skip_leaf,
                             float *h_internal_box, float *h_leaf_box, float *h_bounds) {
    lbvh_status st = lbvh_tree_status(t);
    if (st != LBVH_OK) return st;
    const int64_t n = t->n, ni = n > 0 ? n - 1 : 0;
    if (n == 0) return LBVH_OK;
    if (h_perm) LBVH_CUDA(cudaMemcpy(h_perm, t->perm(), n * 4, cudaMemcpyDeviceToHost));
    if (h_sorted_codes) LBVH_CUDA(cudaMemcpy(h_sorted_codes, t->sorted_codes(), n * 8, cudaMemcpyDeviceToHost));
    if (h_bounds) LBVH_CUDA(cudaMemcpy(h_bounds, t->bounds.p, 24, cudaMemcpyDeviceToHost));
    if (ni > 0 && (h_left || h_skip_internal || h_internal_box)) {
        std::vector<float4> nodes((size_t)ni * 2);
        LBVH_CUDA(cudaMemcpy(nodes.data(), t->inodes(), ni * 32, cudaMemcpyDeviceToHost));
        for (int64_t k = 0; k < ni; ++k) {
            const float4 a = nodes[2 * k], b = nodes[2 * k + 1];
            int32_t left, skip;
            std::memcpy(&left, &a.w, 4);
            std::memcpy(&skip, &b.w, 4);
            if (h_left) h_left[k] = left;
            if (h_skip_internal) h_skip_internal[k] = skip;
            if (h_internal_box) {
                const float v[6] = {a.x, a.y, a.z, b.x, b.y, b.z};
                std::memcpy(h_internal_box + 6 * k, v, sizeof v);
            }
        }
    }
    if (h_skip_leaf || h_leaf_box) {
        const int per = t->kind == LBVH_PRIM_POINTS ? 1 : 2;
        std::vector<float4> leaves((size_t)n * per);
        LBVH_CUDA(cudaMemcpy(leaves.data(), t->leaves(), n * 16 * per, cudaMemcpyDeviceToHost));
        for (int64_t k = 0; k < n; ++k) {
            const float4 a = leaves[per * k], b = leaves[per * k + per - 1];
            uint32_t word;
            std::memcpy(&word, &a.w, 4);
            if (h_skip_leaf) h_skip_leaf[k] = lbvh::leaf_skip_id(word, (int)k, (int)n);
            if (h_leaf_box) {
                const float v[6] = {a.x, a.y, a.z, b.x, b.y, b.z};
                std::memcpy(h_leaf_box + 6 * k, v, sizeof v);
            }
        }
    }
    return LBVH_OK;
}

lbvh_status lbvh_query_into(lbvh_tree_t t, const float *d_queries, int64_t nq, int qkind,
                            const float *d_radii, float radius, int64_t *d_offsets, uint32_t *d_hits,
                            uint64_t capacity, uint64_t *total, lbvh_stream_t stream) {
    lbvh_status st = check_query_args(t, d_queries, nq, qkind, d_radii, radius);
    if (st != LBVH_OK) return st;
    if (!d_offsets || !total || (capacity > 0 && !d_hits)) return LBVH_ERR_INVALID;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    lbvh::QueryArgs qa{d_queries, nq, qkind, d_radii, radius, nullptr};
    st = query_count(t, qa, d_offsets, s, total);
    if (st != LBVH_OK) return st;
    if (*total > capacity) return LBVH_ERR_CAPACITY;
    return query_fill(t, qa, d_offsets, d_hits, s);
}

lbvh_status lbvh_query(lbvh_tree_t t, const float *d_queries, int64_t nq, int qkind,
                       const float *d_radii, float radius, int64_t **d_offsets, uint32_t **d_hits,
                       uint64_t *total, lbvh_stream_t stream) {
    lbvh_status st = check_query_args(t, d_queries, nq, qkind, d_radii, radius);
    if (st != LBVH_OK) return st;
    if (!d_offsets || !d_hits || !total) return LBVH_ERR_INVALID;
    *d_offsets = nullptr;
    *d_hits = nullptr;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    LBVH_CUDA(cudaMalloc(reinterpret_cast<void **>(d_offsets), ((size_t)nq + 1) * 8));
    lbvh::QueryArgs qa{d_queries, nq, qkind, d_radii, radius, nullptr};
    st = query_count(t, qa, *d_offsets, s, total);
    if (st == LBVH_OK) {
        cudaError_t e = cudaMalloc(reinterpret_cast<void **>(d_hits), (size_t)(*total > 0 ? *total : 1) * 4);
        if (e != cudaSuccess) {
            note_cuda(e);
            st = e == cudaErrorMemoryAllocation ? LBVH_ERR_OOM : LBVH_ERR_CUDA;
        }
    }
    if (st == LBVH_OK) st = query_fill(t, qa, *d_offsets, *d_hits, s);
    if (st != LBVH_OK) {
        cudaStreamSynchronize(s);
        cudaFree(*d_offsets);
        cudaFree(*d_hits);
        *d_offsets = nullptr;
        *d_hits = nullptr;
    }
    return st;
}

void lbvh_free(void *d_ptr) {
    if (d_ptr) cudaFree(d_ptr);
}

lbvh_status lbvh_morton_codes(const float *d_prims, int64_t n, int kind, int morton_bits,
                              uint64_t *d_codes, float *d_bounds, lbvh_stream_t stream) {
    using namespace lbvh;
    if (n < 0 || n > LBVH_MAX_PRIMS || !valid_bits(morton_bits)) return LBVH_ERR_INVALID;
    if (kind != LBVH_PRIM_POINTS && kind != LBVH_PRIM_BOXES) return LBVH_ERR_INVALID;
    if (n == 0) return LBVH_OK;
    if (!d_prims || !d_codes || !d_bounds) return LBVH_ERR_INVALID;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    DevBuf ctl, partials, hist;
    lbvh_status st = LBVH_OK;
    Control h{};
    cudaError_t e = ctl.ensure(sizeof(Control), s, true);
    if (e == cudaSuccess) e = partials.ensure((size_t)bounds_blocks(n) * 32, s);
    if (e == cudaSuccess) e = hist.ensure((size_t)kMaxPasses * kRadix * 4, s);
    if (e == cudaSuccess) {
        launch_bounds(d_prims, n, kind, partials.as<float>(), d_bounds, ctl.as<Control>(), s);
        launch_encode(d_prims, n, kind, morton_bits, d_bounds, d_codes, hist.as<uint32_t>(), 0, s);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, ctl.p, sizeof h, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        note_cuda(e);
        st = e == cudaErrorMemoryAllocation ? LBVH_ERR_OOM : LBVH_ERR_CUDA;
    } else {
        st = flags_status(h.build_flags);
    }
    ctl.release(s);
    partials.release(s);
    hist.release(s);
    return st;
}

lbvh_status lbvh_sort_pairs(const uint64_t *d_keys, const uint32_t *d_vals, int64_t n, int key_bits,
                            uint64_t *d_keys_out, uint32_t *d_vals_out, lbvh_stream_t stream) {
    using namespace lbvh;
    if (n < 0 || n > LBVH_MAX_PRIMS || key_bits < 1 || key_bits > 64) return LBVH_ERR_INVALID;
    if (n == 0) return LBVH_OK;
    if (!d_keys || !d_keys_out || !d_vals_out) return LBVH_ERR_INVALID;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int passes = sort_passes(key_bits);
    const int64_t tiles = sort_tiles(n);
    DevBuf ctl, hist, lookback, tk, tv;
    Control h{};
    cudaError_t e = ctl.ensure(sizeof(Control), s, true);
    if (e == cudaSuccess) e = hist.ensure((size_t)kMaxPasses * kRadix * 4, s, true);
    if (e == cudaSuccess) e = lookback.ensure((size_t)tiles * kRadix * 8, s);
    if (e == cudaSuccess) e = tk.ensure((size_t)n * 8, s);
    if (e == cudaSuccess) e = tv.ensure((size_t)n * 4, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_keys_out, d_keys, (size_t)n * 8, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && d_vals)
        e = cudaMemcpyAsync(d_vals_out, d_vals, (size_t)n * 4, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) {
        launch_digit_histogram(d_keys_out, n, 1, hist.as<uint32_t>(), s);
        SortScratch scratch{hist.as<uint32_t>(), lookback.as<uint32_t>(), tiles * kRadix};
        const bool in_b = run_onesweep(d_keys_out, d_vals_out, d_vals == nullptr, tk.as<uint64_t>(),
                                       tv.as<uint32_t>(), n, passes, scratch, ctl.as<Control>(), s);
        e = cudaGetLastError();
        if (e == cudaSuccess && in_b) {
            e = cudaMemcpyAsync(d_keys_out, tk.p, (size_t)n * 8, cudaMemcpyDeviceToDevice, s);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(d_vals_out, tv.p, (size_t)n * 4, cudaMemcpyDeviceToDevice, s);
        }
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, ctl.p, sizeof h, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    lbvh_status st = LBVH_OK;
    if (e != cudaSuccess) {
        note_cuda(e);
        st = e == cudaErrorMemoryAllocation ? LBVH_ERR_OOM : LBVH_ERR_CUDA;
    } else {
        st = flags_status(h.build_flags);
    }
    for (DevBuf *b : {&ctl, &hist, &lookback, &tk, &tv}) b->release(s);
    return st;
}

lbvh_status lbvh_tree_set_profiling(lbvh_tree_t t, int on) {
    if (!t) return LBVH_ERR_INVALID;
    LBVH_CUDA(t->prof.enable(on != 0));
    return LBVH_OK;
}

lbvh_status lbvh_tree_stage_times(lbvh_tree_t t, float *ms) {
    if (!t || !ms) return LBVH_ERR_INVALID;
    for (int k = 0; k < LBVH_STAGE_COUNT; ++k) {
        ms[k] = NAN;
        if (!t->prof.ready || !t->prof.recorded[k]) continue;
        LBVH_CUDA(cudaEventSynchronize(t->prof.ev[k][1]));
        LBVH_CUDA(cudaEventElapsedTime(&ms[k], t->prof.ev[k][0], t->prof.ev[k][1]));
    }
    return LBVH_OK;
}

const char *lbvh_stage_name(int stage) {
    static const char *names[LBVH_STAGE_COUNT] = {
        "bounds", "encode", "sort_pass0", "sort_pass1", "sort_pass2", "sort_pass3", "sort_pass4",
        "sort_pass5", "sort_pass6", "sort_pass7", "construct", "query_walk", "query_scan",
        "query_copy", "query_overflow", "query_order"};
    return (stage >= 0 && stage < LBVH_STAGE_COUNT) ? names[stage] : "";
}

uint64_t lbvh_kernel_launches(void) { return lbvh::g_launches.load(std::memory_order_relaxed); }

const char *lbvh_status_str(lbvh_status st) {
    switch (st) {
    case LBVH_OK: return "LBVH_OK";
    case LBVH_ERR_INVALID: return "LBVH_ERR_INVALID";
    case LBVH_ERR_NONFINITE: return "LBVH_ERR_NONFINITE";
    case LBVH_ERR_OOM: return "LBVH_ERR_OOM";
    case LBVH_ERR_CUDA: return "LBVH_ERR_CUDA";
    case LBVH_ERR_TIMEOUT: return "LBVH_ERR_TIMEOUT";
    case LBVH_ERR_CORRUPT: return "LBVH_ERR_CORRUPT";
    case LBVH_ERR_CAPACITY: return "LBVH_ERR_CAPACITY";
    }
    return "LBVH_ERR_UNKNOWN";
}

const char *lbvh_last_cuda_error(void) { return g_last_error; }

}  // extern "C"
