// capi.cu -- the C ABI of include/lbvh.h: argument checks, device storage of
// a tree, and the order of kernel launches for a build and a query. No
// arithmetic of the method happens here; every step runs in the kernels.
#include <atomic>
#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "lbvh_internal.cuh"

namespace {

thread_local char g_last_error[256] = "";

// Records a runtime error that a call is about to return as its status, and
// clears the thread's last-error state: the error has been reported, and a
// later call's launch check (or the caller's own) must not take it for its
// own (an allocation that failed would otherwise fail the next call too).
void note_cuda(cudaError_t e) {
    std::snprintf(g_last_error, sizeof g_last_error, "%s: %s", cudaGetErrorName(e),
                  cudaGetErrorString(e));
    (void)cudaGetLastError();
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
        if (p) lbvh::pool_free(p, s);
        p = nullptr;
        bytes = 0;
        cudaError_t e = lbvh::pool_alloc(&p, want, s);
        if (e != cudaSuccess) {
            p = nullptr;
            return e;
        }
        bytes = want;
        if (zero) e = cudaMemsetAsync(p, 0, want, s);
        return e;
    }
    void release(cudaStream_t s) {
        if (p) lbvh::pool_free(p, s);
        p = nullptr;
        bytes = 0;
    }
    template <typename T>
    T *as() const {
        return static_cast<T *>(p);
    }
};

// Pinned host mirrors of the control block. They are carved from 64 KiB
// pinned pages that live until the process exits and are recycled, never
// freed: cudaFreeHost would wait for the whole device, which a request server
// evicting trees while other batches run cannot afford.
struct PinnedControls {
    std::mutex mu;
    std::vector<lbvh::Control *> free_list;

    cudaError_t get(lbvh::Control **out) {
        std::lock_guard<std::mutex> lock(mu);
        if (free_list.empty()) {
            constexpr size_t kPage = 64 << 10, kEach = (sizeof(lbvh::Control) + 127) & ~size_t(127);
            void *page = nullptr;
            const cudaError_t e = cudaHostAlloc(&page, kPage, cudaHostAllocPortable);
            if (e != cudaSuccess) return e;
            for (size_t off = 0; off + kEach <= kPage; off += kEach)
                free_list.push_back(reinterpret_cast<lbvh::Control *>(static_cast<char *>(page) + off));
        }
        *out = free_list.back();
        free_list.pop_back();
        return cudaSuccess;
    }
    void put(lbvh::Control *c) {
        if (!c) return;
        std::lock_guard<std::mutex> lock(mu);
        free_list.push_back(c);
    }
};

PinnedControls &pinned_controls() {
    static PinnedControls *pool = new PinnedControls();  // never destroyed (used until exit)
    return *pool;
}

bool valid_bits(int bits) { return bits >= 3 && bits <= 63 && bits % 3 == 0; }

lbvh_status flags_status(uint32_t flags) {
    if (flags & lbvh::kFlagTimeout) return LBVH_ERR_TIMEOUT;
    if (flags & lbvh::kFlagNonfinite) return LBVH_ERR_NONFINITE;
    if (flags & lbvh::kFlagCorrupt) return LBVH_ERR_CORRUPT;
    return LBVH_OK;
}

// Host-side scoped NVTX range (API calls and the sort).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

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
    // Each stage is also an NVTX range on the host thread (no-ops unless a
    // profiler is attached), so tools see where launches come from.
    void begin(int st, cudaStream_t s) {
        nvtxRangePushA(lbvh_stage_name(st));
        if (on) cudaEventRecord(ev[st][0], s);
    }
    void end(int st, cudaStream_t s) {
        nvtxRangePop();
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
    cudaEvent_t used = nullptr;     // recorded after the last query's last kernel
    bool queried = false;           // `used` has been recorded
    bool lean = false;              // nodes and bounds only (no perm / codes): queries, no export
    int64_t n = 0;
    int kind = LBVH_PRIM_POINTS;
    int bits = 0;
    bool has_build = false;
    int codes_in = 0, perm_in = 0;  // which keys[] / vals[] buffer holds the sorted codes / permutation
    int sort_choice = -1, walk_choice = -1;  // lbvh_tree_set_tuning (-1: the tuner's cache, else the default)
    int host_chunks = 0;                     // lbvh_tree_set_host_chunks (0: kHostChunksMax)
    bool store_dirty = false;  // a failed build may have left store words set
    DevBuf keys[2], vals[2];
    DevBuf nodes, store, lookback, hist, partials, bounds, ctl;
    DevBuf pend;  // climbs handed from the construct to its second kernel (zeroed, kept zero)
    DevBuf counts, tile_sums, overflow, slots, spill_head, spill;
    DevBuf qkeys[2], qvals[2], qlookback;  // Morton order of the queries
    DevBuf vscratch;                       // scratch of the Karras / Apetrei builds
    // lbvh_query_into_host: device staging of two chunks' CSR, the stream
    // that copies them to the host, and its events
    DevBuf stage_off[2], stage_hits[2];
    cudaStream_t xfer = nullptr;
    cudaEvent_t staged[2] = {nullptr, nullptr}, drained[2] = {nullptr, nullptr}, xfer_done = nullptr;
    const float *prims_ptr = nullptr;      // the last build's input (self-queries)
    int64_t spill_nq = 0;                  // query count the spill pool was sized for
    lbvh::Control *h_ctl = nullptr;  // pinned mirror of the control block (from pinned_controls())
    Profiler prof;

    const uint64_t *sorted_codes() const { return keys[codes_in].as<uint64_t>(); }
    const uint32_t *perm() const { return vals[perm_in].as<uint32_t>(); }
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

namespace {
std::mutex g_pool_mu;
std::map<int, cudaMemPool_t> g_pools;  // per device, kept until the process exits

cudaError_t device_pool(cudaMemPool_t *out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(g_pool_mu);
    auto it = g_pools.find(dev);
    if (it != g_pools.end()) {
        *out = it->second;
        return cudaSuccess;
    }
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    if ((e = cudaMemPoolCreate(&pool, &props)) != cudaSuccess) return e;
    uint64_t keep = UINT64_MAX;
    if ((e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep)) != cudaSuccess) return e;
    g_pools[dev] = pool;
    *out = pool;
    return cudaSuccess;
}
}  // namespace

cudaError_t pool_alloc(void **p, size_t bytes, cudaStream_t s) {
    cudaMemPool_t pool = nullptr;
    const cudaError_t e = device_pool(&pool);
    if (e != cudaSuccess) return e;
    return cudaMallocFromPoolAsync(p, bytes, pool, s);
}

void pool_free(void *p, cudaStream_t s) {
    if (p) cudaFreeAsync(p, s);
}

cudaError_t pool_reserve(size_t bytes, cudaStream_t s) {
    void *p = nullptr;
    cudaError_t e = pool_alloc(&p, bytes, s);
    if (e != cudaSuccess) return e;
    if ((e = cudaFreeAsync(p, s)) != cudaSuccess) return e;
    return cudaStreamSynchronize(s);
}

int device_sm_count() {
    // read once, thread-safely (function-local static initialisation)
    static const int sms = [] {
        int dev = 0, v = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        return v > 0 ? v : 1;
    }();
    return sms;
}

}  // namespace lbvh

namespace {

// Storage for a tree of n primitives; the control block and `store` are
// zeroed when first allocated and kept clean by the kernels afterwards.
lbvh_status reserve_tree(lbvh_tree_s *t, int64_t n, int kind, cudaStream_t s) {
    using namespace lbvh;
    const size_t un = (size_t)n, ui = (size_t)(n > 0 ? n - 1 : 0);
    const int64_t tiles = sort_tiles_max(n);
    LBVH_CUDA(t->ctl.ensure(sizeof(Control), s, true));
    for (int k = 0; k < 2; ++k) {
        LBVH_CUDA(t->keys[k].ensure(un * 8, s));
        LBVH_CUDA(t->vals[k].ensure(un * 4, s));
    }
    LBVH_CUDA(t->nodes.ensure(ui * 32 + leaf_float4s(n, kind) * 16, s));
    LBVH_CUDA(t->store.ensure(ui * 8, s, true));
    LBVH_CUDA(t->pend.ensure(construct_pend_bytes(n), s, true));
    LBVH_CUDA(t->lookback.ensure((size_t)tiles * kRadix * 4 * 2, s));
    LBVH_CUDA(t->hist.ensure((size_t)kMaxPasses * kRadix * 4, s));
    LBVH_CUDA(t->partials.ensure((size_t)bounds_blocks(n) * 8 * 4, s));
    LBVH_CUDA(t->bounds.ensure(6 * 4, s));
    if (!t->h_ctl) LBVH_CUDA(pinned_controls().get(&t->h_ctl));
    t->lean = false;
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
    if (!t->h_ctl) LBVH_CUDA(pinned_controls().get(&t->h_ctl));
    LBVH_CUDA(cudaMemcpyAsync(t->h_ctl, t->ctl.p, sizeof(lbvh::Control), cudaMemcpyDeviceToHost, s));
    LBVH_CUDA(cudaStreamSynchronize(s));
    if (t->h_ctl->build_flags & (lbvh::kFlagTimeout | lbvh::kFlagCorrupt)) t->store_dirty = true;
    return LBVH_OK;
}

constexpr int64_t kOrderMinQueries = 2048;  // below this, walk in input order
// Morton bits of the query order: 30 (4 sort passes) by default, or 24 (3
// passes) as the tuner's choice. 24 bits walk uniform queries as fast as 30,
// but on clustered queries (a Gaussian mixture) the coarser cells cost more
// walk time than the pass saves; order changes speed only. Batches use 30.
constexpr int order_bits() { return 30; }

// The order in which threads take the queries: the Morton order of the query
// centres inside the tree's bounds (encode + radix sort of `bits`-bit codes,
// the build's own kernels). Queries that are the primitives of the last build
// (same pointer and count) reuse the build's permutation. Order only changes
// speed, never results.
lbvh_status query_order(lbvh_tree_t t, lbvh::QueryArgs &qa, cudaStream_t s, int bits = order_bits()) {
    using namespace lbvh;
    qa.order = nullptr;
    // rays are walked in the caller's order (a camera's rays are coherent as given)
    if (qa.nq < kOrderMinQueries || t->n == 0 || qa.qkind == LBVH_Q_RAY) return LBVH_OK;
    const bool same_points = qa.qkind == LBVH_Q_SPHERE && t->kind == LBVH_PRIM_POINTS;
    const bool same_boxes = qa.qkind == LBVH_Q_BOX && t->kind == LBVH_PRIM_BOXES;
    if (qa.queries == t->prims_ptr && qa.nq == t->n && (same_points || same_boxes)) {
        qa.order = t->perm();
        return LBVH_OK;
    }
    // codes of at most 32 bits, packed with the query index (code << 32 | i):
    // one 8-byte word per query each way, and the last pass writes the order alone
    const size_t unq = (size_t)qa.nq;
    for (int k = 0; k < 2; ++k) {
        LBVH_CUDA(t->qkeys[k].ensure(unq * 8, s));
        LBVH_CUDA(t->qvals[k].ensure(unq * 4, s));
    }
    LBVH_CUDA(t->qlookback.ensure((size_t)sort_tiles_max(qa.nq) * kRadix * 4 * 2, s));
    LBVH_CUDA(cudaMemsetAsync(t->hist.p, 0, (size_t)sort_passes(bits) * kRadix * 4, s));
    const int as_prims = qa.qkind == LBVH_Q_SPHERE ? LBVH_PRIM_POINTS : LBVH_PRIM_BOXES;
    launch_encode(qa.queries, qa.nq, as_prims, bits, t->bounds.as<float>(), t->qkeys[0].as<uint64_t>(),
                  t->hist.as<uint32_t>(), 1, kCodeLow, 0, s);
    LBVH_LAUNCHED();
    SortScratch scratch{t->hist.as<uint32_t>(), t->qlookback.as<uint32_t>(), sort_tiles_max(qa.nq) * kRadix};
    qa.order = run_index_sort(t->qkeys[0].as<uint64_t>(), t->qkeys[1].as<uint64_t>(), t->qvals[0].as<uint32_t>(),
                              qa.nq, bits, scratch, t->dctl(), s);
    LBVH_LAUNCHED();
    return LBVH_OK;
}

lbvh::QueryScratch query_scratch(lbvh_tree_t t) {
    return lbvh::QueryScratch{t->counts.as<uint32_t>(), t->slots.as<uint32_t>(), t->overflow.as<uint32_t>(),
                              t->spill_head.as<uint32_t>(), t->spill.as<uint32_t>(),
                              lbvh::spill_chunks_for(t->spill_nq)};
}

// The query up to the hit count: order, collecting walk, scan; synchronises `s`.
lbvh_status query_count(lbvh_tree_t t, lbvh::QueryArgs &qa, int64_t *d_offsets,
                        cudaStream_t s, uint64_t *total) {
    using namespace lbvh;
    LBVH_CUDA(cudaStreamWaitEvent(s, t->built, 0));
    const size_t unq = (size_t)qa.nq;
    LBVH_CUDA(t->counts.ensure(unq * 4 + 4, s));
    LBVH_CUDA(t->overflow.ensure(unq * 4 + 4, s));
    LBVH_CUDA(t->spill_head.ensure(unq * 4 + 4, s));
    if (spill_chunks_for(qa.nq) > spill_chunks_for(t->spill_nq) || !t->spill.p) {
        LBVH_CUDA(t->spill.ensure((size_t)spill_chunks_for(qa.nq) * kSpillChunkWords * 4, s));
        t->spill_nq = qa.nq;
    }
    LBVH_CUDA(t->tile_sums.ensure((size_t)scan_tile_count(qa.nq) * 8 + 8, s));
    LBVH_CUDA(t->slots.ensure(unq * kQueryBufferHits * 4 + 16, s));
    Control *c = t->dctl();
    LBVH_CUDA(cudaMemsetAsync(&c->query_flags, 0, offsetof(Control, pad) - offsetof(Control, query_flags), s));
    t->prof.clear(LBVH_STAGE_QCOUNT, LBVH_STAGE_QORDER + 1);
    const int choice = t->walk_choice >= 0 ? t->walk_choice : tune_walk_choice(t->n, t->bits, t->kind, qa.qkind, 1);
    qa.walk = walk_choice_kind(choice);
    t->prof.begin(LBVH_STAGE_QORDER, s);
    lbvh_status ost = query_order(t, qa, s, walk_choice_order_bits(choice));
    t->prof.end(LBVH_STAGE_QORDER, s);
    if (ost != LBVH_OK) return ost;
    const QueryScratch qs = query_scratch(t);
    t->prof.begin(LBVH_STAGE_QCOUNT, s);
    launch_query_collect(t->view(), qa, qs, c, s);
    t->prof.end(LBVH_STAGE_QCOUNT, s);
    LBVH_LAUNCHED();
    t->prof.begin(LBVH_STAGE_QSCAN, s);
    launch_exclusive_scan(qs.counts, qa.nq, d_offsets, t->tile_sums.as<int64_t>(), c, s);
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
    launch_query_copy(qa, qs, d_offsets, d_hits, t->dctl(), s);
    t->prof.end(LBVH_STAGE_QFILL, s);
    LBVH_LAUNCHED();
    if (t->h_ctl->overflow_filled > 0) {
        t->prof.begin(LBVH_STAGE_QFIXUP, s);
        launch_query_overflow(t->view(), qa, qs, t->h_ctl->overflow_filled, d_offsets, d_hits, t->dctl(), s);
        t->prof.end(LBVH_STAGE_QFIXUP, s);
        LBVH_LAUNCHED();
    }
    // the last kernels that read this tree's buffers: destroy waits for them
    if (!t->used) LBVH_CUDA(cudaEventCreateWithFlags(&t->used, cudaEventDisableTiming));
    LBVH_CUDA(cudaEventRecord(t->used, s));
    t->queried = true;
    return LBVH_OK;
}

lbvh_status check_query_args(lbvh_tree_t t, const float *q, int64_t nq, int qkind,
                             const float *radii, float radius) {
    if (!t || !t->has_build || nq < 0 || nq > LBVH_MAX_PRIMS) return LBVH_ERR_INVALID;
    if (qkind != LBVH_Q_SPHERE && qkind != LBVH_Q_BOX && qkind != LBVH_Q_RAY) return LBVH_ERR_INVALID;
    if (nq > 0 && !q) return LBVH_ERR_INVALID;
    if (qkind == LBVH_Q_RAY && (reinterpret_cast<uintptr_t>(q) & 15u)) return LBVH_ERR_INVALID;  // float4 loads
    if (qkind == LBVH_Q_SPHERE && !radii && !(std::isfinite(radius) && radius >= 0.0f))
        return LBVH_ERR_INVALID;
    return LBVH_OK;
}

// ---------------------------------------------------------------- batches

struct BatchSignature {
    const float *prims = nullptr, *queries = nullptr, *radii = nullptr;
    int kind = 0, qkind = 0, bits = 0;
    float radius = 0.0f;
    std::vector<int64_t> prim_off, query_off;
    int64_t *offsets = nullptr;
    uint32_t *hits = nullptr;
    unsigned long long capacity = 0;
    bool operator==(const BatchSignature &o) const {
        return prims == o.prims && queries == o.queries && radii == o.radii && kind == o.kind &&
               qkind == o.qkind && bits == o.bits && radius == o.radius && prim_off == o.prim_off &&
               query_off == o.query_off && offsets == o.offsets && hits == o.hits && capacity == o.capacity;
    }
};

// The tuner's configuration of a batch: its primitives' size bucket, bits and
// kind, and its instance count rounded up to a power of two.
lbvh::TuneKey batch_tune_key(int64_t N, int bits, int kind, int64_t count) {
    return lbvh::tune_key(N, bits, kind, -1, int64_t(1) << lbvh::ceil_log2(count < 1 ? 1 : count));
}


}  // namespace

struct lbvh_batch_s {
    BatchSignature sig;
    bool ready = false;   // buffers and tables match `sig`
    int64_t count = 0, N = 0, NQ = 0, nchunks = 0, nqchunks = 0;
    int passes = 0, qpasses = 0, sort_variant = -1;
    bool self_query = false, sorted_in_b = false;
    DevBuf prim_off, query_off, node_start, store_start, chunks, chunk_first, qchunks;
    DevBuf keys[2], vals[2], nodes, store, lookback, hist, partials, bounds, ctl;
    DevBuf counts, slots, overflow, tile_sums, qkeys[2], qvals[2], qlookback, spill_head, spill;
    // Segmented-sort tile tables: row r (r < sort_variant_count(): that
    // variant; the last row: the default variant) holds count + 1 entries.
    DevBuf tile_first, qtile_first;
    std::vector<int64_t> h_tiles, h_qtiles;  // tiles per row
    int64_t max_tiles = 0, max_qtiles = 0;
    std::vector<int64_t> h_node_start;
    lbvh::Control *h_ctl = nullptr;
    cudaGraphExec_t exec = nullptr;
    int graph_kernels = 0;
    bool graphs = true;             // record and replay CUDA graphs (off: run directly every call)
    cudaStream_t stream = nullptr;  // the batch's own stream (capturable), ordered after the caller's
    cudaEvent_t ordered = nullptr;

    lbvh::BatchTables tables() const {
        return lbvh::BatchTables{prim_off.as<int64_t>(), query_off.as<int64_t>(), node_start.as<int64_t>(),
                                 store_start.as<int64_t>(), chunks.as<lbvh::BatchChunk>(),
                                 chunk_first.as<int64_t>(), qchunks.as<lbvh::BatchChunk>(), (int)count,
                                 N, NQ, nchunks, nqchunks};
    }
    const uint64_t *sorted_codes() const { return keys[sorted_in_b ? 1 : 0].as<uint64_t>(); }
    const uint32_t *perm() const { return vals[sorted_in_b ? 1 : 0].as<uint32_t>(); }
    lbvh::Control *dctl() const { return ctl.as<lbvh::Control>(); }
    // Segments of the primitive (or query) sort for tile shape `variant`.
    lbvh::SortSegments segments(bool queries, int variant) const {
        const int rows = (int)h_tiles.size();
        const int r = (variant >= 0 && variant < rows - 1) ? variant : rows - 1;
        const int64_t *tf = (queries ? qtile_first : tile_first).as<int64_t>() + (int64_t)r * (count + 1);
        return lbvh::SortSegments{(queries ? query_off : prim_off).as<int64_t>(), tf, (int)count,
                                  (queries ? h_qtiles : h_tiles)[r]};
    }
    void drop_graph() {
        if (exec) cudaGraphExecDestroy(exec);
        exec = nullptr;
    }
};

namespace {

std::vector<lbvh::BatchChunk> make_chunks(const std::vector<int64_t> &off, std::vector<int64_t> *first) {
    std::vector<lbvh::BatchChunk> out;
    if (first) first->assign(off.size(), 0);
    for (size_t b = 0; b + 1 < off.size(); ++b) {
        if (first) (*first)[b] = (int64_t)out.size();
        for (int64_t c = off[b]; c < off[b + 1]; c += lbvh::kBatchChunk)
            out.push_back(lbvh::BatchChunk{c, std::min(off[b + 1], c + (int64_t)lbvh::kBatchChunk), (int)b, 0});
    }
    if (first) first->back() = (int64_t)out.size();
    return out;
}

lbvh_status upload(DevBuf &dst, const void *src, size_t bytes, cudaStream_t s) {
    LBVH_CUDA(dst.ensure(bytes + 8, s));
    if (bytes) LBVH_CUDA(cudaMemcpyAsync(dst.p, src, bytes, cudaMemcpyHostToDevice, s));
    return LBVH_OK;
}

// Buffers and tables for the signature in b->sig (one synchronising set-up).
lbvh_status batch_setup(lbvh_batch_t b, cudaStream_t s) {
    using namespace lbvh;
    const BatchSignature &g = b->sig;
    b->count = (int64_t)g.prim_off.size() - 1;
    b->N = g.prim_off.back();
    b->NQ = g.query_off.back();
    b->passes = sort_passes(g.bits);
    b->qpasses = sort_passes(order_bits());
    const bool same_points = g.qkind == LBVH_Q_SPHERE && g.kind == LBVH_PRIM_POINTS;
    const bool same_boxes = g.qkind == LBVH_Q_BOX && g.kind == LBVH_PRIM_BOXES;
    b->self_query = g.queries == g.prims && g.query_off == g.prim_off && (same_points || same_boxes);
    std::vector<int64_t> first;
    const std::vector<BatchChunk> chunks = make_chunks(g.prim_off, &first);
    const std::vector<BatchChunk> qchunks = make_chunks(g.query_off, nullptr);
    b->nchunks = (int64_t)chunks.size();
    b->nqchunks = (int64_t)qchunks.size();
    std::vector<int64_t> node_start(b->count), store_start(b->count);
    int64_t units = 0, words = 0;
    for (int64_t k = 0; k < b->count; ++k) {
        const int64_t n = g.prim_off[k + 1] - g.prim_off[k];
        node_start[k] = units;
        store_start[k] = words;
        if (n > 0) {
            units += 2 * (n - 1) + (g.kind == LBVH_PRIM_POINTS ? n : 2 * n);
            units += units & 1;  // every tree starts on a 32-byte boundary (the walk loads 32-byte records)
            words += n - 1;
        }
    }
    b->h_node_start = node_start;
    // Tile tables of the segmented sorts, one row per tile shape.
    const int rows = sort_variant_count() + 1;
    std::vector<int64_t> tf((size_t)rows * (b->count + 1)), qtf((size_t)rows * (b->count + 1));
    b->h_tiles.assign(rows, 0);
    b->h_qtiles.assign(rows, 0);
    for (int r = 0; r < rows; ++r) {
        const int64_t tk = sort_variant_tile_keys(r < rows - 1 ? r : -1);
        int64_t t = 0, qt = 0;
        for (int64_t k = 0; k <= b->count; ++k) {
            tf[(size_t)r * (b->count + 1) + k] = t;
            qtf[(size_t)r * (b->count + 1) + k] = qt;
            if (k < b->count) {
                t += (g.prim_off[k + 1] - g.prim_off[k] + tk - 1) / tk;
                qt += (g.query_off[k + 1] - g.query_off[k] + tk - 1) / tk;
            }
        }
        b->h_tiles[r] = t;
        b->h_qtiles[r] = qt;
    }
    b->max_tiles = *std::max_element(b->h_tiles.begin(), b->h_tiles.end());
    b->max_qtiles = *std::max_element(b->h_qtiles.begin(), b->h_qtiles.end());
    lbvh_status st;
    if ((st = upload(b->tile_first, tf.data(), tf.size() * 8, s)) != LBVH_OK) return st;
    if ((st = upload(b->qtile_first, qtf.data(), qtf.size() * 8, s)) != LBVH_OK) return st;
    if ((st = upload(b->prim_off, g.prim_off.data(), g.prim_off.size() * 8, s)) != LBVH_OK) return st;
    if ((st = upload(b->query_off, g.query_off.data(), g.query_off.size() * 8, s)) != LBVH_OK) return st;
    if ((st = upload(b->node_start, node_start.data(), node_start.size() * 8, s)) != LBVH_OK) return st;
    if ((st = upload(b->store_start, store_start.data(), store_start.size() * 8, s)) != LBVH_OK) return st;
    if ((st = upload(b->chunks, chunks.data(), chunks.size() * sizeof(BatchChunk), s)) != LBVH_OK) return st;
    if ((st = upload(b->chunk_first, first.data(), first.size() * 8, s)) != LBVH_OK) return st;
    if ((st = upload(b->qchunks, qchunks.data(), qchunks.size() * sizeof(BatchChunk), s)) != LBVH_OK) return st;
    const size_t un = (size_t)b->N, unq = (size_t)b->NQ;
    LBVH_CUDA(b->ctl.ensure(sizeof(Control), s, true));
    for (int k = 0; k < 2; ++k) {
        LBVH_CUDA(b->keys[k].ensure(un * 8 + 8, s));
        LBVH_CUDA(b->vals[k].ensure(un * 4 + 4, s));
        LBVH_CUDA(b->qkeys[k].ensure(unq * 8 + 8, s));
        LBVH_CUDA(b->qvals[k].ensure(unq * 4 + 4, s));
    }
    LBVH_CUDA(b->nodes.ensure((size_t)units * 16 + 16, s));
    LBVH_CUDA(b->store.ensure((size_t)words * 8 + 8, s, true));
    LBVH_CUDA(b->lookback.ensure((size_t)b->max_tiles * kRadix * 8 + 8, s));
    LBVH_CUDA(b->qlookback.ensure((size_t)b->max_qtiles * kRadix * 8 + 8, s));
    LBVH_CUDA(b->hist.ensure((size_t)kMaxPasses * b->count * kRadix * 4 + 4, s));
    LBVH_CUDA(b->partials.ensure((size_t)b->nchunks * 32 + 32, s));
    LBVH_CUDA(b->bounds.ensure((size_t)b->count * 24 + 24, s));
    LBVH_CUDA(b->counts.ensure(unq * 4 + 4, s));
    LBVH_CUDA(b->slots.ensure(unq * kQueryBufferHits * 4 + 16, s));
    LBVH_CUDA(b->overflow.ensure(unq * 4 + 4, s));
    LBVH_CUDA(b->spill_head.ensure(unq * 4 + 4, s));
    LBVH_CUDA(b->spill.ensure((size_t)spill_chunks_for(b->NQ) * kSpillChunkWords * 4, s));
    LBVH_CUDA(b->tile_sums.ensure((size_t)scan_tile_count(b->NQ) * 8 + 8, s));
    if (!b->h_ctl) LBVH_CUDA(pinned_controls().get(&b->h_ctl));
    LBVH_CUDA(cudaStreamSynchronize(s));
    b->ready = true;
    return LBVH_OK;
}

// The whole batched pipeline on `s`, with no host synchronisation (so it can
// be captured in a CUDA graph): bounds, Morton codes, one segmented radix sort over
// all instances, the bottom-up pass of every tree, the queries' Morton order,
// the collecting walk, the scan, the checked copy and the overflow lists.
lbvh_status batch_enqueue(lbvh_batch_t b, cudaStream_t s) {
    using namespace lbvh;
    const BatchSignature &g = b->sig;
    const BatchTables bt = b->tables();
    Control *c = b->dctl();
    LBVH_CUDA(cudaMemsetAsync(&c->build_flags, 0, sizeof(uint32_t), s));
    LBVH_CUDA(cudaMemsetAsync(&c->query_flags, 0, offsetof(Control, pad) - offsetof(Control, query_flags), s));
    if (b->N > 0) {
        LBVH_CUDA(cudaMemsetAsync(b->hist.p, 0, (size_t)b->passes * b->count * kRadix * 4, s));
        launch_batch_bounds(g.prims, g.kind, bt, b->partials.as<float>(), b->bounds.as<float>(), c, s);
        launch_batch_encode(g.prims, g.kind, false, bt, g.bits, b->bounds.as<float>(), b->keys[0].as<uint64_t>(),
                            b->hist.as<uint32_t>(), s);
        SortScratch scratch{b->hist.as<uint32_t>(), b->lookback.as<uint32_t>(), b->max_tiles * kRadix};
        const SortSegments seg = b->segments(false, b->sort_variant);
        b->sorted_in_b = run_onesweep(b->keys[0].as<uint64_t>(), b->vals[0].as<uint32_t>(), true,
                                      b->keys[1].as<uint64_t>(), b->vals[1].as<uint32_t>(), b->N, b->passes,
                                      scratch, c, s, nullptr, b->sort_variant, &seg);
        launch_batch_construct(b->sorted_codes(), b->perm(), g.prims, bt, g.kind, b->nodes.as<float4>(),
                               b->store.as<unsigned long long>(), &c->build_flags, s);
        LBVH_LAUNCHED();
    }
    if (b->NQ == 0) {
        LBVH_CUDA(cudaMemsetAsync(g.offsets, 0, 8, s));
        return LBVH_OK;
    }
    QueryArgs qa{g.queries, b->NQ, g.qkind, g.radii, g.radius, nullptr};
    if (b->self_query) {
        qa.order = b->perm();
    } else {
        LBVH_CUDA(cudaMemsetAsync(b->hist.p, 0, (size_t)b->qpasses * b->count * kRadix * 4, s));
        const int as_prims = g.qkind == LBVH_Q_SPHERE ? LBVH_PRIM_POINTS : LBVH_PRIM_BOXES;
        launch_batch_encode(g.queries, as_prims, true, bt, order_bits(), b->bounds.as<float>(), b->qkeys[0].as<uint64_t>(),
                            b->hist.as<uint32_t>(), s);
        SortScratch scratch{b->hist.as<uint32_t>(), b->qlookback.as<uint32_t>(), b->max_qtiles * kRadix};
        const SortSegments seg = b->segments(true, b->sort_variant);
        const bool in_b = run_onesweep(b->qkeys[0].as<uint64_t>(), b->qvals[0].as<uint32_t>(), true,
                                       b->qkeys[1].as<uint64_t>(), b->qvals[1].as<uint32_t>(), b->NQ,
                                       b->qpasses, scratch, c, s, nullptr, b->sort_variant, &seg);
        qa.order = b->qvals[in_b ? 1 : 0].as<uint32_t>();
    }
    const QueryScratch qs{b->counts.as<uint32_t>(), b->slots.as<uint32_t>(), b->overflow.as<uint32_t>(),
                          b->spill_head.as<uint32_t>(), b->spill.as<uint32_t>(), spill_chunks_for(b->NQ)};
    launch_batch_collect(b->nodes.as<float4>(), g.kind, bt, qa, qs, c, s);
    launch_exclusive_scan(qs.counts, b->NQ, g.offsets, b->tile_sums.as<int64_t>(), c, s);
    launch_query_copy_checked(qa, qs, g.offsets, g.hits, g.capacity, c, s);
    launch_batch_overflow(b->nodes.as<float4>(), g.kind, bt, qa, qs, c, g.offsets, g.hits, g.capacity, s);
    LBVH_LAUNCHED();
    return LBVH_OK;
}

// Sort tile shape for this batch: the fastest variant on the batch's own keys
// (timed with events on `s`), kept in the tuner's cache for its configuration.
lbvh_status batch_autotune(lbvh_batch_t b, cudaStream_t s) {
    using namespace lbvh;
    if (b->sort_variant >= 0 || b->N < (1 << 20)) return LBVH_OK;
    const TuneKey key = batch_tune_key(b->N, b->sig.bits, b->sig.kind, b->count);
    {
        TuneChoice known;
        if (tune_find(key, &known) && known.sort >= 0) {
            b->sort_variant = known.sort;
            return LBVH_OK;
        }
    }
    const BatchSignature &g = b->sig;
    const BatchTables bt = b->tables();
    Control *c = b->dctl();
    cudaEvent_t e0, e1;
    LBVH_CUDA(cudaEventCreate(&e0));
    LBVH_CUDA(cudaEventCreate(&e1));
    float best = 1e30f;
    int pick = 0;
    for (int v = 0; v < sort_variant_count(); ++v) {
        float ms_total = 0.0f;
        for (int rep = 0; rep < 2; ++rep) {
            LBVH_CUDA(cudaMemsetAsync(b->hist.p, 0, (size_t)b->passes * b->count * kRadix * 4, s));
            launch_batch_encode(g.prims, g.kind, false, bt, g.bits, b->bounds.as<float>(),
                                b->keys[0].as<uint64_t>(), b->hist.as<uint32_t>(), s);
            SortScratch scratch{b->hist.as<uint32_t>(), b->lookback.as<uint32_t>(), b->max_tiles * kRadix};
            const SortSegments seg = b->segments(false, v);
            LBVH_CUDA(cudaEventRecord(e0, s));
            run_onesweep(b->keys[0].as<uint64_t>(), b->vals[0].as<uint32_t>(), true, b->keys[1].as<uint64_t>(),
                         b->vals[1].as<uint32_t>(), b->N, b->passes, scratch, c, s, nullptr, v, &seg);
            LBVH_CUDA(cudaEventRecord(e1, s));
            LBVH_CUDA(cudaEventSynchronize(e1));
            float ms = 0.0f;
            LBVH_CUDA(cudaEventElapsedTime(&ms, e0, e1));
            if (rep) ms_total += ms;  // the first repetition warms up
        }
        if (ms_total < best) {
            best = ms_total;
            pick = v;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->sort_variant = pick;
    TuneChoice made;
    made.sort = pick;
    made.sort_ms = best;
    tune_put(key, made);
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
    // Wait for this tree's own work only (its last build and its last
    // query), not for whole streams or the device; then the buffers go back
    // to the stream-ordered pool and the pinned mirror to its free list.
    if (t->has_build && t->built) cudaEventSynchronize(t->built);
    else if (t->nodes.p) cudaDeviceSynchronize();  // a build that failed part-way may still run
    if (t->queried) cudaEventSynchronize(t->used);
    for (DevBuf *b : {&t->keys[0], &t->keys[1], &t->vals[0], &t->vals[1], &t->nodes,
                      &t->store, &t->pend, &t->lookback, &t->hist, &t->partials, &t->bounds, &t->ctl,
                      &t->counts, &t->tile_sums, &t->overflow, &t->qkeys[0], &t->qkeys[1],
                      &t->qvals[0], &t->qvals[1], &t->qlookback, &t->slots, &t->vscratch, &t->spill_head,
                      &t->spill, &t->stage_off[0], &t->stage_off[1], &t->stage_hits[0], &t->stage_hits[1]})
        b->release(cudaStreamPerThread);
    pinned_controls().put(t->h_ctl);
    if (t->built) cudaEventDestroy(t->built);
    if (t->used) cudaEventDestroy(t->used);
    for (cudaEvent_t e : {t->staged[0], t->staged[1], t->drained[0], t->drained[1], t->xfer_done})
        if (e) cudaEventDestroy(e);
    if (t->xfer) cudaStreamDestroy(t->xfer);
    t->prof.release();
    delete t;
}

}  // extern "C"

namespace {

lbvh_status build_impl(lbvh_tree_t t, const float *d_prims, int64_t n, int kind, int morton_bits,
                       int algorithm, lbvh_stream_t stream) {
    NvtxRange nvtx_range("lbvh_build");
    using namespace lbvh;
    lbvh_status st = check_build_args(t, d_prims, n, kind);
    if (st != LBVH_OK) return st;
    if (!valid_bits(morton_bits)) return LBVH_ERR_INVALID;
    if (algorithm < LBVH_BUILD_MODIFIED_APETREI || algorithm > LBVH_BUILD_APETREI) return LBVH_ERR_INVALID;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    st = reserve_tree(t, n, kind, s);
    if (st != LBVH_OK) return st;
    if (algorithm != LBVH_BUILD_MODIFIED_APETREI)
        LBVH_CUDA(t->vscratch.ensure(variant_scratch_bytes(n, algorithm), s));
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
    t->prof.clear(LBVH_STAGE_SECOND, LBVH_STAGE_SECOND + 1);
    t->prof.clear(LBVH_STAGE_SORTRUNS, LBVH_STAGE_SORTRUNS + 1);
    if (n > 0) {
        const int passes = sort_passes(morton_bits);
        LBVH_CUDA(cudaMemsetAsync(t->hist.p, 0, (size_t)kMaxPasses * kRadix * 4, s));
        t->prof.begin(LBVH_STAGE_BOUNDS, s);
        launch_bounds(d_prims, n, kind, t->partials.as<float>(), t->bounds.as<float>(), c, s);
        t->prof.end(LBVH_STAGE_BOUNDS, s);
        LBVH_LAUNCHED();
        t->prof.begin(LBVH_STAGE_ENCODE, s);
        // codes of at most 30 bits are packed with the index from the start
        // (code << 32 | index); wider codes give their top bits (top << ib |
        // index) to run_code_sort
        const bool packed = morton_bits <= 30;
        const int ib = top_index_bits(n);
        // the sort choice: tile shape, and whether the top-bits sort covers
        // one byte fewer (more elements in runs of equal sorted bits)
        const int choice = t->sort_choice >= 0 ? t->sort_choice : tune_sort_choice(n, morton_bits, kind, 1);
        const int variant = sort_choice_tile(choice);
        const int skip = packed ? 0 : sort_choice_skip(choice);
        launch_encode(d_prims, n, kind, morton_bits, t->bounds.as<float>(), t->keys[0].as<uint64_t>(),
                      t->hist.as<uint32_t>(), 1, packed ? kCodeLow : kCodeTop, ib, s, skip);
        t->prof.end(LBVH_STAGE_ENCODE, s);
        LBVH_LAUNCHED();
        SortScratch scratch{t->hist.as<uint32_t>(), t->lookback.as<uint32_t>(), sort_tiles_max(n) * kRadix};
        nvtxRangePushA("sort");
        cudaEvent_t(*pass_events)[2] = t->prof.on ? &t->prof.ev[LBVH_STAGE_SORT0] : nullptr;
        // the node records are written by the construct only: until then they
        // hold run_code_sort's 2n scratch words
        const uint32_t *perm =
            packed ? run_index_sort(t->keys[0].as<uint64_t>(), t->keys[1].as<uint64_t>(), t->vals[0].as<uint32_t>(),
                                    n, morton_bits, scratch, c, s, pass_events, variant)
                   : run_code_sort(d_prims, kind, morton_bits, t->bounds.as<float>(), n, t->keys[0].as<uint64_t>(),
                                   t->keys[1].as<uint64_t>(), t->vals[0].as<uint32_t>(), t->vals[1].as<uint32_t>(),
                                   t->nodes.as<uint32_t>(), scratch, c, s, pass_events,
                                   t->prof.on ? t->prof.ev[LBVH_STAGE_SORTRUNS] : nullptr, variant, skip);
        nvtxRangePop();
        if (t->prof.on) {
            const int sorted = packed ? passes : kMaxPasses - top_first_byte(ib, skip);
            for (int p = 0; p < sorted; ++p) t->prof.recorded[LBVH_STAGE_SORT0 + p] = true;
            if (!packed) t->prof.recorded[LBVH_STAGE_SORTRUNS] = true;
        }
        LBVH_LAUNCHED();
        // the sort leaves the permutation alone; the sorted codes go to keys[0]
        t->perm_in = perm == t->vals[1].as<uint32_t>() ? 1 : 0;
        t->codes_in = 0;
        t->prof.begin(LBVH_STAGE_CONSTRUCT, s);
        if (algorithm == LBVH_BUILD_MODIFIED_APETREI) {
            launch_construct_encode(t->perm(), d_prims, t->bounds.as<float>(), morton_bits, n, kind,
                                    t->keys[0].as<uint64_t>(), t->inodes(), t->leaves(),
                                    t->store.as<unsigned long long>(), &c->build_flags, t->pend.p, s);
        } else {
            launch_sorted_codes(d_prims, t->perm(), n, kind, morton_bits, t->bounds.as<float>(),
                                t->keys[0].as<uint64_t>(), s);
            launch_variant_hierarchy(algorithm, t->sorted_codes(), t->perm(), d_prims, n, kind, t->inodes(),
                                     t->leaves(), t->vscratch.p, t->store.as<unsigned long long>(),
                                     &c->build_flags, s);
        }
        t->prof.end(LBVH_STAGE_CONSTRUCT, s);
        LBVH_LAUNCHED();
        if (algorithm != LBVH_BUILD_MODIFIED_APETREI) {
            t->prof.begin(LBVH_STAGE_SECOND, s);
            launch_variant_second(algorithm, t->sorted_codes(), t->perm(), d_prims, n, kind, t->inodes(),
                                  t->leaves(), t->vscratch.p, t->store.as<unsigned long long>(),
                                  &c->build_flags, s);
            t->prof.end(LBVH_STAGE_SECOND, s);
            LBVH_LAUNCHED();
        }
    }
    return finish_build(t, s);
}

}  // namespace

extern "C" {

lbvh_status lbvh_build(lbvh_tree_t t, const float *d_prims, int64_t n, int kind, int morton_bits,
                       lbvh_stream_t stream) {
    return build_impl(t, d_prims, n, kind, morton_bits, LBVH_BUILD_MODIFIED_APETREI, stream);
}

lbvh_status lbvh_build_variant(lbvh_tree_t t, const float *d_prims, int64_t n, int kind, int morton_bits,
                               int algorithm, lbvh_stream_t stream) {
    return build_impl(t, d_prims, n, kind, morton_bits, algorithm, stream);
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
    t->codes_in = t->perm_in = 0;
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
                         t->leaves(), t->store.as<unsigned long long>(), &c->build_flags, t->pend.p, s);
        LBVH_LAUNCHED();
    }
    return finish_build(t, s);
}

lbvh_status lbvh_refit(lbvh_tree_t t, const float *d_prims, lbvh_stream_t stream) {
    NvtxRange nvtx_range("lbvh_refit");
    using namespace lbvh;
    if (!t || !t->has_build || t->lean) return LBVH_ERR_INVALID;
    const int64_t n = t->n;
    if (n > 0 && !d_prims) return LBVH_ERR_INVALID;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    LBVH_CUDA(cudaStreamWaitEvent(s, t->built, 0));
    if (t->queried) LBVH_CUDA(cudaStreamWaitEvent(s, t->used, 0));
    t->prims_ptr = d_prims;
    Control *c = t->dctl();
    LBVH_CUDA(cudaMemsetAsync(&c->build_flags, 0, sizeof(uint32_t), s));
    if (t->store_dirty && t->store.bytes) {
        LBVH_CUDA(cudaMemsetAsync(t->store.p, 0, t->store.bytes, s));
        t->store_dirty = false;
    }
    t->prof.clear(0, LBVH_STAGE_QCOUNT);
    if (n > 0) {
        t->prof.begin(LBVH_STAGE_BOUNDS, s);
        launch_bounds(d_prims, n, t->kind, t->partials.as<float>(), t->bounds.as<float>(), c, s);
        t->prof.end(LBVH_STAGE_BOUNDS, s);
        LBVH_LAUNCHED();
        t->prof.begin(LBVH_STAGE_CONSTRUCT, s);
        launch_construct(t->sorted_codes(), t->perm(), d_prims, n, t->kind, t->inodes(), t->leaves(),
                         t->store.as<unsigned long long>(), &c->build_flags, t->pend.p, s);
        t->prof.end(LBVH_STAGE_CONSTRUCT, s);
        LBVH_LAUNCHED();
    }
    return finish_build(t, s);
}

}  // extern "C"

namespace {

constexpr char kImageMagic[8] = {'L', 'B', 'V', 'H', 'T', 'R', 'E', 'E'};
constexpr uint32_t kImageVersion = 1;

struct ImageHeader {
    char magic[8];
    uint32_t version, kind, bits, zero;
    uint64_t n;
    float bounds[6];
    uint32_t pad[2];
};
static_assert(sizeof(ImageHeader) == 64, "image header layout");

uint64_t image_node_bytes(int64_t n, int kind) {
    if (n <= 0) return 0;
    return (uint64_t)(2 * (n - 1)) * 16 + (uint64_t)lbvh::leaf_float4s(n, kind) * 16;
}

uint64_t image_bytes(int64_t n, int kind) {
    return sizeof(ImageHeader) + (uint64_t)n * 12 + image_node_bytes(n, kind);
}

}  // namespace

extern "C" {

lbvh_status lbvh_tree_save(lbvh_tree_t t, void *h_buf, uint64_t capacity, uint64_t *bytes) {
    if (!t || !bytes || !t->has_build || t->lean) return LBVH_ERR_INVALID;
    const int64_t n = t->n;
    *bytes = image_bytes(n, t->kind);
    if (!h_buf) return LBVH_OK;
    if (capacity < *bytes) return LBVH_ERR_CAPACITY;
    lbvh_status st = lbvh_tree_status(t);  // synchronises; a failed build is not saved
    if (st != LBVH_OK) return st;
    ImageHeader h{};
    std::memcpy(h.magic, kImageMagic, 8);
    h.version = kImageVersion;
    h.kind = (uint32_t)t->kind;
    h.bits = (uint32_t)t->bits;
    h.n = (uint64_t)n;
    LBVH_CUDA(cudaMemcpy(h.bounds, t->bounds.p, 24, cudaMemcpyDeviceToHost));
    char *out = static_cast<char *>(h_buf);
    std::memcpy(out, &h, sizeof h);
    out += sizeof h;
    if (n > 0) {
        LBVH_CUDA(cudaMemcpy(out, t->sorted_codes(), (size_t)n * 8, cudaMemcpyDeviceToHost));
        out += (size_t)n * 8;
        LBVH_CUDA(cudaMemcpy(out, t->perm(), (size_t)n * 4, cudaMemcpyDeviceToHost));
        out += (size_t)n * 4;
        LBVH_CUDA(cudaMemcpy(out, t->nodes.p, image_node_bytes(n, t->kind), cudaMemcpyDeviceToHost));
    }
    return LBVH_OK;
}

lbvh_status lbvh_tree_load(lbvh_tree_t t, const void *h_buf, uint64_t bytes, lbvh_stream_t stream) {
    if (!t || !h_buf || bytes < sizeof(ImageHeader)) return LBVH_ERR_INVALID;
    ImageHeader h;
    std::memcpy(&h, h_buf, sizeof h);
    if (std::memcmp(h.magic, kImageMagic, 8) != 0 || h.version != kImageVersion) return LBVH_ERR_INVALID;
    if (h.kind != LBVH_PRIM_POINTS && h.kind != LBVH_PRIM_BOXES) return LBVH_ERR_INVALID;
    if (h.n > (uint64_t)LBVH_MAX_PRIMS || (h.bits != 0 && !valid_bits((int)h.bits))) return LBVH_ERR_INVALID;
    const int64_t n = (int64_t)h.n;
    const int kind = (int)h.kind;
    if (bytes != image_bytes(n, kind)) return LBVH_ERR_INVALID;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    lbvh_status st = reserve_tree(t, n, kind, s);
    if (st != LBVH_OK) return st;
    t->n = n;
    t->kind = kind;
    t->bits = (int)h.bits;
    t->codes_in = t->perm_in = 0;
    t->prims_ptr = nullptr;
    LBVH_CUDA(cudaMemsetAsync(&t->dctl()->build_flags, 0, sizeof(uint32_t), s));
    LBVH_CUDA(cudaMemcpyAsync(t->bounds.p, h.bounds, 24, cudaMemcpyHostToDevice, s));
    const char *in = static_cast<const char *>(h_buf) + sizeof h;
    if (n > 0) {
        LBVH_CUDA(cudaMemcpyAsync(t->keys[0].p, in, (size_t)n * 8, cudaMemcpyHostToDevice, s));
        in += (size_t)n * 8;
        LBVH_CUDA(cudaMemcpyAsync(t->vals[0].p, in, (size_t)n * 4, cudaMemcpyHostToDevice, s));
        in += (size_t)n * 4;
        LBVH_CUDA(cudaMemcpyAsync(t->nodes.p, in, image_node_bytes(n, kind), cudaMemcpyHostToDevice, s));
    }
    // the bounds copy above reads a stack value: make sure it has been taken
    LBVH_CUDA(cudaStreamSynchronize(s));
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
                            &t->store, &t->pend, &t->lookback, &t->hist, &t->partials, &t->bounds, &t->ctl,
                            &t->counts, &t->tile_sums, &t->overflow, &t->qkeys[0], &t->qkeys[1],
                            &t->qvals[0], &t->qvals[1], &t->qlookback, &t->slots, &t->vscratch,
                            &t->spill_head, &t->spill})
        b += d->bytes;
    *bytes = b;
    return LBVH_OK;
}

lbvh_status lbvh_tree_export(lbvh_tree_t t, uint32_t *h_perm, uint64_t *h_sorted_codes,
                             int32_t *h_left, int32_t *h_skip_internal, int32_t *h_skip_leaf,
                             float *h_internal_box, float *h_leaf_box, float *h_bounds) {
    if (t && t->lean) return LBVH_ERR_INVALID;  // resident copy without perm and codes
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
    NvtxRange nvtx_range("lbvh_query_into");
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

}  // extern "C"

namespace {

bool page_locked(const void *h) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, h) != cudaSuccess) {
        (void)cudaGetLastError();  // not a pointer CUDA knows: leave no sticky error
        return false;
    }
    return a.type == cudaMemoryTypeHost;
}

// Queries per chunk of lbvh_query_into_host: at least 2^23, at most 4
// chunks by default. 2^25 sphere queries (17 hits each): 27.0 ms with 3 or 4
// chunks, 27.8 with 2, 29.2 with 8, 35.5 with 16, against 32.6 ms for the
// query and the copies one after the other (each chunk adds a host round
// trip, and its copy shares the link and L2 with the next chunk's walk).
// With two trees in flight (one tree's copies overlapping the other's build
// and walk), one chunk is best: 2^25 points built and queried per step at
// 1466 Mprims/s through host memory with 1 chunk, 1392 with 2, 1271 with 4.
constexpr int64_t kHostChunkMin = int64_t(1) << 23;
constexpr int64_t kHostChunksMax = 4;
constexpr int kHostChunksLimit = 16;  // lbvh_tree_set_host_chunks

lbvh_status host_stream(lbvh_tree_t t) {
    if (t->xfer) return LBVH_OK;
    LBVH_CUDA(cudaStreamCreateWithFlags(&t->xfer, cudaStreamNonBlocking));
    for (cudaEvent_t *e : {&t->staged[0], &t->staged[1], &t->drained[0], &t->drained[1], &t->xfer_done})
        LBVH_CUDA(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
    return LBVH_OK;
}

}  // namespace

extern "C" {

// Chunks of queries in index order, each through the device path into one of
// two staging areas; the copy of chunk k to the host runs on the tree's copy
// stream while the GPU works on chunk k+1 (chunk k+2 reuses the area once that
// copy is done). The caller's stream waits for the last copy.
lbvh_status lbvh_query_into_host(lbvh_tree_t t, const float *d_queries, int64_t nq, int qkind,
                                 const float *d_radii, float radius, int64_t *h_offsets, uint32_t *h_hits,
                                 uint64_t capacity, uint64_t *total, lbvh_stream_t stream) {
    NvtxRange nvtx_range("lbvh_query_into_host");
    using namespace lbvh;
    lbvh_status st = check_query_args(t, d_queries, nq, qkind, d_radii, radius);
    if (st != LBVH_OK) return st;
    if (!h_offsets || !total || (capacity > 0 && !h_hits)) return LBVH_ERR_INVALID;
    if (!page_locked(h_offsets) || (capacity > 0 && !page_locked(h_hits))) return LBVH_ERR_INVALID;
    if ((st = host_stream(t)) != LBVH_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int dim = qkind == LBVH_Q_SPHERE ? 3 : (qkind == LBVH_Q_BOX ? 6 : 8);
    const int64_t cmin = kHostChunkMin;
    const int64_t cmax = t->host_chunks > 0 ? t->host_chunks : kHostChunksMax;
    const int64_t chunks = nq <= cmin ? 1 : std::min<int64_t>(cmax, (nq + cmin - 1) / cmin);
    const int64_t per = (nq + chunks - 1) / chunks;
    uint64_t base = 0;
    bool over = false;
    auto run = [&]() -> lbvh_status {
        for (int64_t k = 0; k < chunks; ++k) {
            const int64_t q0 = k * per, m = std::min(per, nq - q0);
            if (m < 0 || (m == 0 && k > 0)) break;
            const int b = (int)(k & 1);
            if (k >= 2) LBVH_CUDA(cudaStreamWaitEvent(s, t->drained[b], 0));  // its staging area is free again
            LBVH_CUDA(t->stage_off[b].ensure((size_t)(m + 1) * 8, s));
            int64_t *soff = t->stage_off[b].as<int64_t>();
            QueryArgs qa{d_queries + q0 * dim, m, qkind, d_radii ? d_radii + q0 : nullptr, radius, nullptr};
            uint64_t tot = 0;
            lbvh_status cst = query_count(t, qa, soff, s, &tot);
            if (cst != LBVH_OK) return cst;
            const bool fits = !over && base + tot <= capacity;
            over = !fits;
            if (fits && tot > 0) {
                LBVH_CUDA(t->stage_hits[b].ensure((size_t)tot * 4, s));
                if ((cst = query_fill(t, qa, soff, t->stage_hits[b].as<uint32_t>(), s)) != LBVH_OK) return cst;
            }
            if (base > 0) launch_offsets_add(soff, m + 1, (int64_t)base, s);
            LBVH_CUDA(cudaEventRecord(t->staged[b], s));
            LBVH_CUDA(cudaStreamWaitEvent(t->xfer, t->staged[b], 0));
            LBVH_CUDA(cudaMemcpyAsync(h_offsets + q0, soff, (size_t)(m + 1) * 8, cudaMemcpyDeviceToHost, t->xfer));
            if (fits && tot > 0)
                LBVH_CUDA(cudaMemcpyAsync(h_hits + base, t->stage_hits[b].p, (size_t)tot * 4,
                                          cudaMemcpyDeviceToHost, t->xfer));
            LBVH_CUDA(cudaEventRecord(t->drained[b], t->xfer));
            base += tot;
        }
        return LBVH_OK;
    };
    st = run();
    // on every path: the caller's stream (and the tree's `used` event) cover
    // the copies already issued
    const bool tail_ok = cudaEventRecord(t->xfer_done, t->xfer) == cudaSuccess &&
                         cudaStreamWaitEvent(s, t->xfer_done, 0) == cudaSuccess &&
                         (t->used || cudaEventCreateWithFlags(&t->used, cudaEventDisableTiming) == cudaSuccess) &&
                         cudaEventRecord(t->used, s) == cudaSuccess;
    if (!tail_ok) {
        cudaStreamSynchronize(t->xfer);  // nothing may still read the staging areas
        if (st == LBVH_OK) st = LBVH_ERR_CUDA;
    }
    t->queried = t->used != nullptr;
    *total = base;
    if (st != LBVH_OK) return st;
    return over ? LBVH_ERR_CAPACITY : LBVH_OK;
}

lbvh_status lbvh_tree_walk_visits(lbvh_tree_t t, const float *d_queries, int64_t nq, int qkind,
                                  const float *d_radii, float radius, uint64_t *leaf_visits,
                                  uint64_t *internal_visits, lbvh_stream_t stream) {
    using namespace lbvh;
    lbvh_status st = check_query_args(t, d_queries, nq, qkind, d_radii, radius);
    if (st != LBVH_OK) return st;
    if (!leaf_visits || !internal_visits) return LBVH_ERR_INVALID;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    LBVH_CUDA(cudaStreamWaitEvent(s, t->built, 0));
    QueryArgs qa{d_queries, nq, qkind, d_radii, radius, nullptr};
    if ((st = query_order(t, qa, s)) != LBVH_OK) return st;  // the same order as the collecting walk
    DevBuf counts;
    LBVH_CUDA(counts.ensure(16, s, true));
    launch_visits(t->view(), qa, counts.as<unsigned long long>(), t->dctl(), s);
    LBVH_LAUNCHED();
    unsigned long long h[2] = {0, 0};
    LBVH_CUDA(cudaMemcpyAsync(h, counts.p, 16, cudaMemcpyDeviceToHost, s));
    LBVH_CUDA(cudaStreamSynchronize(s));
    counts.release(s);
    *leaf_visits = h[0];
    *internal_visits = h[1];
    return LBVH_OK;
}

lbvh_status lbvh_knn(lbvh_tree_t t, const float *d_queries, int64_t nq, int k, uint32_t *d_idx, float *d_dist2,
                     lbvh_stream_t stream) {
    NvtxRange nvtx_range("lbvh_knn");
    using namespace lbvh;
    if (!t || !t->has_build || nq < 0 || nq > LBVH_MAX_PRIMS || k < 1 || k > LBVH_KNN_MAX_K)
        return LBVH_ERR_INVALID;
    if (nq > 0 && (!d_queries || !d_idx)) return LBVH_ERR_INVALID;
    if (nq == 0) return LBVH_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    LBVH_CUDA(cudaStreamWaitEvent(s, t->built, 0));
    Control *c = t->dctl();
    LBVH_CUDA(cudaMemsetAsync(&c->query_flags, 0, offsetof(Control, pad) - offsetof(Control, query_flags), s));
    QueryArgs qa{d_queries, nq, LBVH_Q_SPHERE, nullptr, 0.0f, nullptr};
    t->prof.clear(LBVH_STAGE_QCOUNT, LBVH_STAGE_QORDER + 1);
    t->prof.begin(LBVH_STAGE_QORDER, s);
    lbvh_status st = query_order(t, qa, s);  // the Morton order of the query points
    t->prof.end(LBVH_STAGE_QORDER, s);
    if (st != LBVH_OK) return st;
    // a lean (server-resident) tree keeps no sorted codes: its walks start
    // without seeds, which is exact but slower
    const uint64_t *codes = t->lean ? nullptr : t->sorted_codes();
    t->prof.begin(LBVH_STAGE_QCOUNT, s);  // the kNN walk is timed as the query walk
    launch_knn(t->view(), codes, t->bounds.as<float>(), t->bits, qa, k, d_idx, d_dist2, c, s);
    t->prof.end(LBVH_STAGE_QCOUNT, s);
    LBVH_LAUNCHED();
    if (!t->used) LBVH_CUDA(cudaEventCreateWithFlags(&t->used, cudaEventDisableTiming));
    LBVH_CUDA(cudaEventRecord(t->used, s));
    t->queried = true;
    if ((st = read_control(t, s)) != LBVH_OK) return st;
    st = flags_status(t->h_ctl->build_flags);
    return st != LBVH_OK ? st : flags_status(t->h_ctl->query_flags);
}

lbvh_status lbvh_query(lbvh_tree_t t, const float *d_queries, int64_t nq, int qkind,
                       const float *d_radii, float radius, int64_t **d_offsets, uint32_t **d_hits,
                       uint64_t *total, lbvh_stream_t stream) {
    NvtxRange nvtx_range("lbvh_query");
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

lbvh_status lbvh_test_hold_sort_tile(int64_t tile) {
    if (tile < -1) return LBVH_ERR_INVALID;
    lbvh::sort_set_hold_tile(tile);
    return LBVH_OK;
}

lbvh_status lbvh_release_cached_memory(void) {
    std::lock_guard<std::mutex> lock(lbvh::g_pool_mu);
    for (auto &kv : lbvh::g_pools) LBVH_CUDA(cudaMemPoolTrimTo(kv.second, 0));
    return LBVH_OK;
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
        launch_encode(d_prims, n, kind, morton_bits, d_bounds, d_codes, hist.as<uint32_t>(), 0, kCodePlain, 0, s);
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
    const int64_t tiles = sort_tiles_max(n);
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

lbvh_status lbvh_batch_create(lbvh_batch_t *out) {
    if (!out) return LBVH_ERR_INVALID;
    *out = new (std::nothrow) lbvh_batch_s();
    return *out ? LBVH_OK : LBVH_ERR_OOM;
}

void lbvh_batch_destroy(lbvh_batch_t b) {
    if (!b) return;
    cudaStream_t s = b->stream;
    if (s) cudaStreamSynchronize(s);
    b->drop_graph();
    for (DevBuf *d : {&b->prim_off, &b->query_off, &b->node_start, &b->store_start, &b->chunks, &b->chunk_first,
                      &b->qchunks, &b->keys[0], &b->keys[1], &b->vals[0], &b->vals[1], &b->nodes, &b->store,
                      &b->lookback, &b->hist, &b->partials, &b->bounds, &b->ctl, &b->counts, &b->slots,
                      &b->overflow, &b->tile_sums, &b->qkeys[0], &b->qkeys[1], &b->qvals[0], &b->qvals[1],
                      &b->qlookback, &b->tile_first, &b->qtile_first, &b->spill_head, &b->spill})
        d->release(s);
    if (s) cudaStreamSynchronize(s);
    pinned_controls().put(b->h_ctl);
    if (b->ordered) cudaEventDestroy(b->ordered);
    if (s) cudaStreamDestroy(s);
    delete b;
}

lbvh_status lbvh_batch_build_query(lbvh_batch_t b, const float *d_prims, const int64_t *h_prim_offsets,
                                   int64_t count, int kind, int morton_bits, const float *d_queries,
                                   const int64_t *h_query_offsets, int qkind, const float *d_radii,
                                   float radius, int64_t *d_offsets, uint32_t *d_hits, uint64_t capacity,
                                   uint64_t *total, lbvh_stream_t stream) {
    NvtxRange nvtx_range("lbvh_batch_build_query");
    using namespace lbvh;
    if (!b || count < 1 || count > LBVH_MAX_BATCH || !h_prim_offsets || !h_query_offsets || !d_offsets || !total)
        return LBVH_ERR_INVALID;
    if (kind != LBVH_PRIM_POINTS && kind != LBVH_PRIM_BOXES) return LBVH_ERR_INVALID;
    if (qkind != LBVH_Q_SPHERE && qkind != LBVH_Q_BOX) return LBVH_ERR_INVALID;
    if (!valid_bits(morton_bits)) return LBVH_ERR_INVALID;
    if (qkind == LBVH_Q_SPHERE && !d_radii && !(std::isfinite(radius) && radius >= 0.0f)) return LBVH_ERR_INVALID;
    if (h_prim_offsets[0] != 0 || h_query_offsets[0] != 0) return LBVH_ERR_INVALID;
    for (int64_t k = 0; k < count; ++k) {
        const int64_t n = h_prim_offsets[k + 1] - h_prim_offsets[k];
        const int64_t m = h_query_offsets[k + 1] - h_query_offsets[k];
        if (n < 0 || n > LBVH_MAX_PRIMS || m < 0) return LBVH_ERR_INVALID;
    }
    if (h_prim_offsets[count] > ((int64_t)1 << 31) - 1 || h_query_offsets[count] > ((int64_t)1 << 31) - 1)
        return LBVH_ERR_INVALID;
    if ((h_prim_offsets[count] > 0 && !d_prims) || (h_query_offsets[count] > 0 && !d_queries))
        return LBVH_ERR_INVALID;
    if (capacity > 0 && !d_hits) return LBVH_ERR_INVALID;
    // run on the batch's own stream (the caller's may be the legacy default
    // stream, which cannot be captured), after the caller's pending work
    cudaStream_t caller = static_cast<cudaStream_t>(stream);
    if (!b->stream) LBVH_CUDA(cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking));
    if (!b->ordered) LBVH_CUDA(cudaEventCreateWithFlags(&b->ordered, cudaEventDisableTiming));
    LBVH_CUDA(cudaEventRecord(b->ordered, caller));
    LBVH_CUDA(cudaStreamWaitEvent(b->stream, b->ordered, 0));
    cudaStream_t s = b->stream;
    BatchSignature sig;
    sig.prims = d_prims;
    sig.queries = d_queries;
    sig.radii = d_radii;
    sig.kind = kind;
    sig.qkind = qkind;
    sig.bits = morton_bits;
    sig.radius = radius;
    sig.prim_off.assign(h_prim_offsets, h_prim_offsets + count + 1);
    sig.query_off.assign(h_query_offsets, h_query_offsets + count + 1);
    sig.offsets = d_offsets;
    sig.hits = d_hits;
    sig.capacity = capacity;
    lbvh_status st = LBVH_OK;
    if (!b->graphs) {
        // run directly: set up when the instance tables change, use a tuned
        // tile shape if one is known for this size, never capture
        const bool same_tables = b->ready && b->sig.prim_off == sig.prim_off && b->sig.query_off == sig.query_off &&
                                 b->sig.kind == sig.kind && b->sig.bits == sig.bits;
        b->sig = sig;
        if (!same_tables) {
            b->ready = false;
            if ((st = batch_setup(b, s)) != LBVH_OK) return st;
            b->sort_variant = lbvh::tune_sort_choice(b->N, sig.bits, sig.kind,
                                                     int64_t(1) << lbvh::ceil_log2(b->count < 1 ? 1 : b->count));
        } else {
            const bool same_points = qkind == LBVH_Q_SPHERE && kind == LBVH_PRIM_POINTS;
            const bool same_boxes = qkind == LBVH_Q_BOX && kind == LBVH_PRIM_BOXES;
            b->self_query = d_queries == d_prims && sig.query_off == sig.prim_off && (same_points || same_boxes);
        }
        if ((st = batch_enqueue(b, s)) != LBVH_OK) return st;
    } else if (!(b->ready && b->sig == sig)) {
        // a new shape: set up, tune, run once directly, then capture a graph
        b->drop_graph();
        const bool same_tables = b->ready && b->sig.prim_off == sig.prim_off && b->sig.query_off == sig.query_off &&
                                 b->sig.kind == sig.kind && b->sig.bits == sig.bits;
        b->sig = sig;
        if (!same_tables) {
            b->ready = false;
            b->sort_variant = -1;
            if ((st = batch_setup(b, s)) != LBVH_OK) return st;
        } else {
            b->self_query = false;
            const bool same_points = qkind == LBVH_Q_SPHERE && kind == LBVH_PRIM_POINTS;
            const bool same_boxes = qkind == LBVH_Q_BOX && kind == LBVH_PRIM_BOXES;
            b->self_query = d_queries == d_prims && sig.query_off == sig.prim_off && (same_points || same_boxes);
        }
        if ((st = batch_enqueue(b, s)) != LBVH_OK) return st;  // bounds for the autotuner, and a first result
        if ((st = batch_autotune(b, s)) != LBVH_OK) return st;
        if ((st = batch_enqueue(b, s)) != LBVH_OK) return st;
        const unsigned long long before = lbvh_kernel_launches();
        cudaGraph_t graph = nullptr;
        LBVH_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        st = batch_enqueue(b, s);
        const cudaError_t ce = cudaStreamEndCapture(s, &graph);
        if (st != LBVH_OK) {
            if (graph) cudaGraphDestroy(graph);
            return st;
        }
        LBVH_CUDA(ce);
        b->graph_kernels = (int)(lbvh_kernel_launches() - before);
        const cudaError_t ie = cudaGraphInstantiate(&b->exec, graph, 0);
        cudaGraphDestroy(graph);
        LBVH_CUDA(ie);
    } else {
        LBVH_CUDA(cudaGraphLaunch(b->exec, s));
        lbvh::count_launches(b->graph_kernels);
    }
    LBVH_CUDA(cudaMemcpyAsync(b->h_ctl, b->ctl.p, sizeof(Control), cudaMemcpyDeviceToHost, s));
    LBVH_CUDA(cudaStreamSynchronize(s));
    *total = b->h_ctl->total;
    st = flags_status(b->h_ctl->build_flags);
    if (st == LBVH_OK) st = flags_status(b->h_ctl->query_flags);
    if (st == LBVH_OK && (b->h_ctl->query_flags & kFlagCapacity)) st = LBVH_ERR_CAPACITY;
    if (st == LBVH_OK && *total > capacity) st = LBVH_ERR_CAPACITY;
    if (b->h_ctl->build_flags & (kFlagTimeout | kFlagCorrupt)) {  // re-zero the store before the next run
        cudaMemsetAsync(b->store.p, 0, b->store.bytes, s);
        cudaStreamSynchronize(s);
    }
    return st;
}

lbvh_status lbvh_batch_export(lbvh_batch_t b, int64_t instance, uint32_t *h_perm, uint64_t *h_sorted_codes,
                              int32_t *h_left, int32_t *h_skip_internal, int32_t *h_skip_leaf,
                              float *h_internal_box, float *h_leaf_box, float *h_bounds) {
    if (!b || !b->ready || instance < 0 || instance >= b->count) return LBVH_ERR_INVALID;
    LBVH_CUDA(cudaStreamSynchronize(b->stream));
    const int64_t o = b->sig.prim_off[instance];
    const int64_t n = b->sig.prim_off[instance + 1] - o, ni = n > 0 ? n - 1 : 0;
    if (h_bounds) LBVH_CUDA(cudaMemcpy(h_bounds, b->bounds.as<float>() + 6 * instance, 24, cudaMemcpyDeviceToHost));
    if (n == 0) return LBVH_OK;
    if (h_perm) {
        LBVH_CUDA(cudaMemcpy(h_perm, b->perm() + o, n * 4, cudaMemcpyDeviceToHost));
        for (int64_t k = 0; k < n; ++k) h_perm[k] -= (uint32_t)o;
    }
    if (h_sorted_codes) {
        LBVH_CUDA(cudaMemcpy(h_sorted_codes, b->sorted_codes() + o, n * 8, cudaMemcpyDeviceToHost));
    }
    const int per = b->sig.kind == LBVH_PRIM_POINTS ? 1 : 2;
    std::vector<float4> rec((size_t)(2 * ni + per * n));
    LBVH_CUDA(cudaMemcpy(rec.data(), b->nodes.as<float4>() + b->h_node_start[instance], rec.size() * 16,
                         cudaMemcpyDeviceToHost));
    for (int64_t k = 0; k < ni; ++k) {
        const float4 a = rec[2 * k], c = rec[2 * k + 1];
        int32_t left, skip;
        std::memcpy(&left, &a.w, 4);
        std::memcpy(&skip, &c.w, 4);
        if (h_left) h_left[k] = left;
        if (h_skip_internal) h_skip_internal[k] = skip;
        if (h_internal_box) {
            const float v[6] = {a.x, a.y, a.z, c.x, c.y, c.z};
            std::memcpy(h_internal_box + 6 * k, v, sizeof v);
        }
    }
    for (int64_t k = 0; k < n; ++k) {
        const float4 a = rec[2 * ni + per * k], c = rec[2 * ni + per * k + per - 1];
        uint32_t word;
        std::memcpy(&word, &a.w, 4);
        if (h_skip_leaf) h_skip_leaf[k] = lbvh::leaf_skip_id(word, (int)k, (int)n);
        if (h_leaf_box) {
            const float v[6] = {a.x, a.y, a.z, c.x, c.y, c.z};
            std::memcpy(h_leaf_box + 6 * k, v, sizeof v);
        }
    }
    return LBVH_OK;
}

lbvh_status lbvh_batch_sort_variant(lbvh_batch_t b, int *variant) {
    if (!b || !variant) return LBVH_ERR_INVALID;
    *variant = b->sort_variant;
    return LBVH_OK;
}

}  // extern "C"

namespace lbvh {

void batch_set_graphs(lbvh_batch_t b, bool on) {
    if (b->graphs != on) b->drop_graph();
    b->graphs = on;
}

lbvh_status tree_from_batch(lbvh_batch_t b, int64_t instance, lbvh_tree_t t, cudaStream_t s) {
    // A lean copy: what queries read (nodes, scene bounds, control block, the
    // query-order histogram) and nothing that only exports or rebuilds need.
    if (!b || !b->ready || !t || instance < 0 || instance >= b->count) return LBVH_ERR_INVALID;
    const int64_t o = b->sig.prim_off[instance];
    const int64_t n = b->sig.prim_off[instance + 1] - o;
    const int kind = b->sig.kind;
    const int64_t units = n > 0 ? 2 * (n - 1) + (kind == LBVH_PRIM_POINTS ? n : 2 * n) : 0;
    LBVH_CUDA(t->ctl.ensure(sizeof(Control), s, true));
    LBVH_CUDA(t->nodes.ensure((size_t)units * 16 + 16, s));
    LBVH_CUDA(t->hist.ensure((size_t)kMaxPasses * kRadix * 4, s));
    LBVH_CUDA(t->bounds.ensure(6 * 4, s));
    t->lean = true;
    t->n = n;
    t->kind = kind;
    t->bits = b->sig.bits;
    t->codes_in = t->perm_in = 0;
    t->prims_ptr = nullptr;
    LBVH_CUDA(cudaMemsetAsync(&t->dctl()->build_flags, 0, sizeof(uint32_t), s));
    LBVH_CUDA(cudaMemcpyAsync(t->bounds.p, b->bounds.as<float>() + 6 * instance, 24, cudaMemcpyDeviceToDevice, s));
    if (units > 0)
        LBVH_CUDA(cudaMemcpyAsync(t->nodes.p, b->nodes.as<float4>() + b->h_node_start[instance], units * 16,
                                  cudaMemcpyDeviceToDevice, s));
    return finish_build(t, s);
}

void tree_release_query_scratch(lbvh_tree_t t, cudaStream_t s) {
    for (DevBuf *b : {&t->counts, &t->tile_sums, &t->overflow, &t->slots, &t->qkeys[0], &t->qkeys[1],
                      &t->qvals[0], &t->qvals[1], &t->qlookback, &t->spill_head, &t->spill,
                      &t->stage_off[0], &t->stage_off[1], &t->stage_hits[0], &t->stage_hits[1]})
        b->release(s);
    t->spill_nq = 0;
}

}  // namespace lbvh

extern "C" {

lbvh_status lbvh_tree_set_host_chunks(lbvh_tree_t t, int max_chunks) {
    if (!t || max_chunks < 0 || max_chunks > kHostChunksLimit) return LBVH_ERR_INVALID;
    t->host_chunks = max_chunks;
    return LBVH_OK;
}

lbvh_status lbvh_tree_set_tuning(lbvh_tree_t t, int sort_variant, int walk_variant) {
    if (!t || sort_variant < -1 || sort_variant >= lbvh::build_sort_choices() || walk_variant < -1 ||
        walk_variant >= lbvh::kWalkChoices)
        return LBVH_ERR_INVALID;
    t->sort_choice = sort_variant;
    t->walk_choice = walk_variant;
    return LBVH_OK;
}

}  // extern "C"

namespace {

// Device milliseconds of stages [lo, hi) of the tree's last build or query
// (the tree's profiling must be on); synchronises the recording streams.
float stages_ms(lbvh_tree_t t, int lo, int hi) {
    float sum = 0.0f;
    for (int k = lo; k < hi; ++k) {
        if (!t->prof.recorded[k]) continue;
        if (cudaEventSynchronize(t->prof.ev[k][1]) != cudaSuccess) return -1.0f;
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, t->prof.ev[k][0], t->prof.ev[k][1]) != cudaSuccess) return -1.0f;
        sum += ms;
    }
    return sum;
}

}  // namespace

extern "C" {

lbvh_status lbvh_tree_autotune(lbvh_tree_t t, const float *d_prims, int64_t n, int kind, int morton_bits,
                               const float *d_queries, int64_t nq, int qkind, const float *d_radii, float radius,
                               lbvh_stream_t stream, int *sort_variant, int *walk_variant) {
    using namespace lbvh;
    NvtxRange nvtx_range("lbvh_tree_autotune");
    lbvh_status st = check_build_args(t, d_prims, n, kind);
    if (st != LBVH_OK) return st;
    if (!valid_bits(morton_bits) || nq < 0 || (nq > 0 && !d_queries)) return LBVH_ERR_INVALID;
    if (nq > 0 && qkind != LBVH_Q_SPHERE && qkind != LBVH_Q_BOX && qkind != LBVH_Q_RAY) return LBVH_ERR_INVALID;
    if (qkind == LBVH_Q_SPHERE && nq > 0 && !d_radii && !(std::isfinite(radius) && radius >= 0.0f))
        return LBVH_ERR_INVALID;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const bool prof_was = t->prof.on;
    const int keep_sort = t->sort_choice, keep_walk = t->walk_choice;
    LBVH_CUDA(t->prof.enable(true));
    auto finish = [&](lbvh_status r) {
        t->sort_choice = keep_sort;
        t->walk_choice = keep_walk;
        t->prof.on = prof_was;
        return r;
    };
    // the sort: every choice on this build's own keys (tile shapes; for codes
    // wider than 30 bits also one top-bits pass fewer), the best of two runs
    // each, timed over the passes and the runs stage
    float best_sort = 1e30f;
    int pick_sort = 0;
    const int choices = morton_bits <= 30 ? sort_variant_count() : build_sort_choices();
    for (int v = 0; v < choices && n > 0; ++v) {
        t->sort_choice = v;
        for (int rep = 0; rep < 2; ++rep) {
            if ((st = lbvh_build(t, d_prims, n, kind, morton_bits, stream)) != LBVH_OK) return finish(st);
            const float mp = stages_ms(t, LBVH_STAGE_SORT0, LBVH_STAGE_SORT0 + kMaxPasses);
            const float mr = stages_ms(t, LBVH_STAGE_SORTRUNS, LBVH_STAGE_SORTRUNS + 1);
            const float ms = mp < 0.0f || mr < 0.0f ? -1.0f : mp + mr;
            if (ms < 0.0f) return finish(LBVH_ERR_CUDA);
            if (ms < best_sort) {
                best_sort = ms;
                pick_sort = v;
            }
        }
    }
    if (n > 0) {
        TuneChoice made;
        made.sort = pick_sort;
        made.sort_ms = best_sort;
        tune_put(tune_key(n, morton_bits, kind, -1, 1), made);
    }
    t->sort_choice = pick_sort;
    if ((st = lbvh_build(t, d_prims, n, kind, morton_bits, stream)) != LBVH_OK) return finish(st);
    if ((st = lbvh_tree_status(t)) != LBVH_OK) return finish(st);
    int pick_walk = kWalkThread;
    if (nq > 0 && n > 0) {
        DevBuf offsets;
        LBVH_CUDA(offsets.ensure((size_t)(nq + 1) * 8, s));
        float best_walk = 1e30f;
        for (int w = 0; w < kWalkChoices; ++w) {
            t->walk_choice = w;
            for (int rep = 0; rep < 2; ++rep) {
                QueryArgs qa{d_queries, nq, qkind, d_radii, radius, nullptr};
                uint64_t total = 0;
                st = query_count(t, qa, offsets.as<int64_t>(), s, &total);
                if (st != LBVH_OK) {
                    offsets.release(s);
                    return finish(st);
                }
                // the walk and the query order (whose bits are part of the choice)
                const float mw = stages_ms(t, LBVH_STAGE_QCOUNT, LBVH_STAGE_QCOUNT + 1);
                const float mo = stages_ms(t, LBVH_STAGE_QORDER, LBVH_STAGE_QORDER + 1);
                const float ms = mw < 0.0f || mo < 0.0f ? -1.0f : mw + mo;
                if (ms >= 0.0f && ms < best_walk) {
                    best_walk = ms;
                    pick_walk = w;
                }
            }
        }
        offsets.release(s);
        TuneChoice made;
        made.walk = pick_walk;
        made.walk_ms = best_walk;
        tune_put(tune_key(n, morton_bits, kind, qkind, 1), made);
    }
    if (sort_variant) *sort_variant = pick_sort;
    if (walk_variant) *walk_variant = pick_walk;
    return finish(LBVH_OK);
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
        "query_copy", "query_overflow", "query_order", "build_second_pass", "sort_runs"};
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
