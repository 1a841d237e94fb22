// server.cu -- a request server over the batched build + query: requests
// arrive at any time (lbvh_server_submit), a scheduler thread admits them
// against an HBM byte budget and packs compatible ones into batches
// (continuous batching: whatever arrived while other batches ran is admitted
// as soon as a slot and memory are free), slot workers run the batches on
// their own streams so that several batches overlap on the device, and built
// trees can stay resident (under the same budget, evicted least recently used
// first) for later query-only requests.
//
// Nothing here computes the method: builds and queries are the library's
// kernels (lbvh_batch_build_query, lbvh_query_into); this file moves request
// data in and out of batches (copy, rebase of offsets) and keeps the books.
#include <algorithm>
#include <cmath>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <list>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "lbvh_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

double seconds_since(Clock::time_point t0, Clock::time_point t) {
    return std::chrono::duration<double>(t - t0).count();
}

// ---------------------------------------------------------------- kernels

__global__ void fill_kernel(float *out, int64_t n, float v) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = v;
}

// out[j] = off[base + j] - off[base], j in [0, nq]
__global__ void rebase_offsets_kernel(const int64_t *__restrict__ off, int64_t base, int64_t nq,
                                      int64_t *__restrict__ out) {
    const int64_t first = off[base];
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j <= nq; j += (int64_t)gridDim.x * blockDim.x)
        out[j] = off[base + j] - first;
}

// hits of queries [base, base + nq) of the batch CSR -> out, if they fit
__global__ void copy_hits_kernel(const int64_t *__restrict__ off, int64_t base, int64_t nq,
                                 const uint32_t *__restrict__ hits, uint32_t *__restrict__ out,
                                 unsigned long long capacity) {
    const int64_t a = off[base], e = off[base + nq];
    if ((unsigned long long)(e - a) > capacity) return;
    for (int64_t i = a + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < e; i += (int64_t)gridDim.x * blockDim.x)
        out[i - a] = hits[i];
}

// totals[k] = off[qbase[k+1]] - off[qbase[k]]
__global__ void request_totals_kernel(const int64_t *__restrict__ off, const int64_t *__restrict__ qbase, int count,
                                      unsigned long long *__restrict__ totals) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < count) totals[k] = (unsigned long long)(off[qbase[k + 1]] - off[qbase[k]]);
}

unsigned grid_for(int64_t n) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 8192)); }

// ---------------------------------------------------------------- buffers

struct Buf {
    void *p = nullptr;
    size_t bytes = 0;
    lbvh_status ensure(size_t want, cudaStream_t s) {
        if (want <= bytes) return LBVH_OK;
        if (p) lbvh::pool_free(p, s);
        p = nullptr;
        bytes = 0;
        want = std::max<size_t>(want, 256);
        if (lbvh::pool_alloc(&p, want, s) != cudaSuccess) {
            p = nullptr;
            (void)cudaGetLastError();  // reported as LBVH_ERR_OOM: no later launch check may see it
            return LBVH_ERR_OOM;
        }
        bytes = want;
        return LBVH_OK;
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

struct Request {
    lbvh_request req;
    uint64_t ticket = 0;
    uint64_t est_bytes = 0;
    Clock::time_point submitted;
};

struct Outcome {
    bool done = false;
    lbvh_result result{};
};

struct Resident {
    lbvh_tree_t tree = nullptr;
    uint64_t bytes = 0;
    int in_use = 0;
    std::list<uint64_t>::iterator lru;  // position in the LRU list (front = most recent)
};

struct Job {
    std::vector<Request> reqs;
    bool query_only = false;
    uint64_t bytes = 0;
    int64_t work = 0;  // primitives built (build jobs) or queries walked (query-only jobs)
};

// A batch of at least this many primitives (queries for a query-only job)
// starts only when no other batch runs: a batch of a few million points
// already fills the GPU, and two large batches in flight at once (two trees'
// nodes competing for L1 and L2 in a walk bound by its load latency) took
// longer together than one after the other (the 400 requests offered at
// once, two slots: 723 Mprims/s, against 1,228 with one slot). Smaller
// batches still start beside running ones and overlap their launch gaps and
// host round trips.
constexpr int64_t kOverlapWork = int64_t(1) << 23;

struct Slot {
    int index = 0;
    std::thread worker;
    cudaStream_t stream = nullptr;
    cudaEvent_t began = nullptr, ended = nullptr;  // device span of the slot's current job
    lbvh_batch_t batch = nullptr;
    Buf prims, queries, radii, offsets, hits, qbase, totals;
    std::vector<unsigned long long> h_totals;
    bool busy = false;
    std::unique_ptr<Job> job;
};

// Device bytes one build + query request needs while it runs (inputs staged,
// sort buffers, nodes, store, query scratch, output): an upper estimate.
uint64_t estimate_bytes(const lbvh_request &r) {
    const uint64_t n = (uint64_t)r.n, nq = (uint64_t)r.nq;
    const uint64_t prim = r.kind == LBVH_PRIM_POINTS ? 12 : 24;
    const uint64_t qsz = r.qkind == LBVH_Q_SPHERE ? 12 : (r.qkind == LBVH_Q_BOX ? 24 : 32);
    const uint64_t build = n * (prim + 24 + 24 + 48 + 8 + 16);
    const uint64_t query = nq * (qsz + 4 + 8 + lbvh::kQueryBufferHits * 4 + 4 + 8 + 24 + 8) + r.capacity * 4;
    return std::max<uint64_t>(build + query, 1);  // a running job always counts as in flight
}

// Device bytes of a resident tree: its nodes (2(n-1) internal records of
// 32 bytes, leaves of 16 or 32 bytes) plus the control block, bounds and the
// query-order histogram.
uint64_t resident_bytes_of(int64_t n, int kind) {
    const uint64_t un = (uint64_t)std::max<int64_t>(n, 1);
    return (2 * (un - 1) + (kind == LBVH_PRIM_POINTS ? un : 2 * un)) * 16 + 16 + 8192 + 512;
}

bool same_batch_kind(const lbvh_request &a, const lbvh_request &b) {
    return a.kind == b.kind && a.morton_bits == b.morton_bits && a.qkind == b.qkind;
}

}  // namespace

struct lbvh_server_s {
    uint64_t budget = 0;
    int max_batch = 0;
    int64_t max_batch_prims = 0;
    std::mutex mu;
    std::condition_variable cv_sched, cv_done;
    std::deque<Request> pending;
    std::unordered_map<uint64_t, Outcome> outcomes;
    std::unordered_map<uint64_t, Resident> resident;
    std::list<uint64_t> lru;
    uint64_t resident_total = 0, inflight = 0, next_ticket = 1;
    uint64_t evictions = 0, batches = 0, requests_done = 0, jobs_finished = 0;
    double phase_s[LBVH_SERVER_PHASES] = {};  // see lbvh_server_phase_seconds
    std::vector<double> latencies;            // of every answered request, seconds
    cudaEvent_t ref = nullptr;                // recorded once at creation: the origin of device spans
    std::vector<double> spans;                // (slot, begin s, end s) of every job on the device
    bool stop = false;
    Clock::time_point t0 = Clock::now();
    std::vector<std::unique_ptr<Slot>> slots;
    std::condition_variable cv_slot;
    std::thread scheduler;

    void complete(Request &r, lbvh_status st, uint64_t total, Clock::time_point start, int batch_size) {
        const Clock::time_point now = Clock::now();
        Outcome &o = outcomes[r.ticket];
        o.done = true;
        o.result.status = st;
        o.result.total = total;
        o.result.queued_s = seconds_since(r.submitted, start);
        o.result.service_s = seconds_since(start, now);
        o.result.latency_s = seconds_since(r.submitted, now);
        o.result.batch_size = batch_size;
        latencies.push_back(o.result.latency_s);
        ++requests_done;
    }

    // Evict least recently used resident trees that are not in use until
    // `need` more bytes fit. Called with `mu` held.
    bool make_room(uint64_t need) {
        while (resident_total + inflight + need > budget) {
            auto it = std::find_if(lru.rbegin(), lru.rend(), [&](uint64_t k) { return resident[k].in_use == 0; });
            if (it == lru.rend()) return false;
            const uint64_t key = *it;
            Resident &r = resident[key];
            lbvh_tree_destroy(r.tree);
            resident_total -= r.bytes;
            lru.erase(r.lru);
            resident.erase(key);
            ++evictions;
        }
        return true;
    }

    // The device span of the job that just finished on `slot` (its events
    // have completed: the worker synchronised the slot's stream). Called
    // with `mu` held.
    void record_span(const Slot *slot) {
        float b = 0.0f, e = 0.0f;
        if (cudaEventElapsedTime(&b, ref, slot->began) != cudaSuccess ||
            cudaEventElapsedTime(&e, ref, slot->ended) != cudaSuccess) {
            (void)cudaGetLastError();
            return;
        }
        spans.push_back((double)slot->index);
        spans.push_back(b * 1e-3);
        spans.push_back(e * 1e-3);
    }

    void schedule_loop();
    void worker_loop(Slot *slot);
    void run_build_job(Slot *slot, Job &job);
    void run_query_job(Slot *slot, Job &job);
};

void lbvh_server_s::schedule_loop() {
    std::unique_lock<std::mutex> lk(mu);
    while (true) {
        cv_sched.wait(lk, [&] {
            if (stop) return true;
            if (pending.empty()) return false;
            return std::any_of(slots.begin(), slots.end(), [](const std::unique_ptr<Slot> &s) { return !s->busy; });
        });
        if (stop) return;
        auto job = std::make_unique<Job>();
        int64_t prims = 0;
        while (!pending.empty() && (int)job->reqs.size() < max_batch) {
            Request &r = pending.front();
            const bool query_only = r.req.n == 0;
            if (query_only) {
                if (!job->reqs.empty()) break;  // a query-only request runs on its own
                auto it = resident.find(r.req.key);
                if (it == resident.end()) {  // not resident (never built, or evicted)
                    complete(r, LBVH_ERR_INVALID, 0, Clock::now(), 1);
                    pending.pop_front();
                    cv_done.notify_all();
                    continue;
                }
                if (it->second.in_use > 0) break;  // another query is using this tree: one at a time
                it->second.in_use++;  // pinned: make_room must not evict the tree this request needs
                if (!make_room(r.est_bytes)) {
                    it->second.in_use--;
                    if (inflight == 0) {  // can never fit the budget
                        complete(r, LBVH_ERR_OOM, 0, Clock::now(), 1);
                        pending.pop_front();
                        cv_done.notify_all();
                        continue;
                    }
                    break;
                }
                lru.splice(lru.begin(), lru, it->second.lru);
                job->query_only = true;
                job->bytes = r.est_bytes;
                job->work = r.req.nq;
                inflight += r.est_bytes;
                job->reqs.push_back(r);
                pending.pop_front();
                break;
            }
            if (!job->reqs.empty() && (!same_batch_kind(job->reqs[0].req, r.req) || prims + r.req.n > max_batch_prims))
                break;
            if (!make_room(r.est_bytes)) {
                if (job->reqs.empty() && inflight == 0) {  // can never fit the budget
                    complete(r, LBVH_ERR_OOM, 0, Clock::now(), 1);
                    pending.pop_front();
                    cv_done.notify_all();
                    continue;
                }
                break;
            }
            inflight += r.est_bytes;
            job->bytes += r.est_bytes;
            job->work += r.req.n;
            prims += r.req.n;
            job->reqs.push_back(r);
            pending.pop_front();
        }
        if (job->reqs.empty()) {
            if (pending.empty()) continue;  // every queued request was answered at admission
            // the oldest request does not fit yet; a job is running (else the
            // request would have been refused above): wait until one ends
            const uint64_t seen = jobs_finished;
            cv_sched.wait(lk, [&] { return stop || jobs_finished != seen || inflight == 0; });
            continue;
        }
        if (job->work >= kOverlapWork)  // a large batch runs alone (see kOverlapWork)
            cv_sched.wait(lk, [&] {
                return stop || std::none_of(slots.begin(), slots.end(),
                                            [](const std::unique_ptr<Slot> &s) { return s->busy; });
            });
        Slot *free_slot = nullptr;
        for (auto &s : slots)
            if (!s->busy) {
                free_slot = s.get();
                break;
            }
        free_slot->busy = true;
        free_slot->job = std::move(job);
        ++batches;
        cv_slot.notify_all();
    }
}

void lbvh_server_s::worker_loop(Slot *slot) {
    std::unique_lock<std::mutex> lk(mu);
    while (true) {
        cv_slot.wait(lk, [&] { return stop || (slot->busy && slot->job); });
        if (stop && !(slot->busy && slot->job)) return;
        std::unique_ptr<Job> job = std::move(slot->job);
        lk.unlock();
        if (job->query_only) run_query_job(slot, *job);
        else run_build_job(slot, *job);
        lk.lock();
        inflight -= job->bytes;
        ++jobs_finished;
        slot->busy = false;
        cv_done.notify_all();
        cv_sched.notify_all();
    }
}

void lbvh_server_s::run_query_job(Slot *slot, Job &job) {
    nvtxRangePushA("lbvh_server query");
    struct PopAtExit {
        ~PopAtExit() { nvtxRangePop(); }
    } pop_at_exit;
    Request &r = job.reqs[0];
    const Clock::time_point start = Clock::now();
    lbvh_tree_t tree;
    {
        std::lock_guard<std::mutex> lk(mu);
        tree = resident[r.req.key].tree;
    }
    uint64_t total = 0;
    cudaEventRecord(slot->began, slot->stream);
    const lbvh_status st = lbvh_query_into(tree, r.req.d_queries, r.req.nq, r.req.qkind, r.req.d_radii,
                                           r.req.radius, r.req.d_offsets, r.req.d_hits, r.req.capacity, &total,
                                           slot->stream);
    cudaEventRecord(slot->ended, slot->stream);
    lbvh::tree_release_query_scratch(tree, slot->stream);  // resident bytes stay those of the tree
    cudaStreamSynchronize(slot->stream);
    std::lock_guard<std::mutex> lk(mu);
    record_span(slot);
    auto it = resident.find(r.req.key);
    if (it != resident.end()) it->second.in_use--;
    complete(r, st, total, start, 1);
    phase_s[3] += seconds_since(start, Clock::now());
}

void lbvh_server_s::run_build_job(Slot *slot, Job &job) {
    nvtxRangePushA("lbvh_server batch");
    struct PopAtExit {
        ~PopAtExit() { nvtxRangePop(); }
    } pop_at_exit;
    const Clock::time_point start = Clock::now();
    const int count = (int)job.reqs.size();
    const lbvh_request &k0 = job.reqs[0].req;
    cudaStream_t s = slot->stream;
    const int pdim = k0.kind == LBVH_PRIM_POINTS ? 3 : 6;
    const int qdim = k0.qkind == LBVH_Q_SPHERE ? 3 : 6;
    std::vector<int64_t> po(count + 1, 0), qo(count + 1, 0);
    bool self_query = true;
    uint64_t cap = 0;
    for (int k = 0; k < count; ++k) {
        const lbvh_request &r = job.reqs[k].req;
        po[k + 1] = po[k] + r.n;
        qo[k + 1] = qo[k] + r.nq;
        cap += r.capacity;
        const bool same = (r.kind == LBVH_PRIM_POINTS && r.qkind == LBVH_Q_SPHERE) ||
                          (r.kind == LBVH_PRIM_BOXES && r.qkind == LBVH_Q_BOX);
        self_query = self_query && same && r.d_queries == r.d_prims && r.nq == r.n;
    }
    lbvh_status st = LBVH_OK;
    auto fail_all = [&](lbvh_status e) {
        std::lock_guard<std::mutex> lk(mu);
        for (Request &r : job.reqs) complete(r, e, 0, start, count);
    };
    // stage inputs (device to device) into one concatenated batch
    if ((st = slot->prims.ensure((size_t)po[count] * pdim * 4, s)) != LBVH_OK) return fail_all(st);
    if (!self_query && (st = slot->queries.ensure((size_t)qo[count] * qdim * 4, s)) != LBVH_OK) return fail_all(st);
    if (k0.qkind == LBVH_Q_SPHERE && (st = slot->radii.ensure((size_t)qo[count] * 4, s)) != LBVH_OK)
        return fail_all(st);
    if ((st = slot->offsets.ensure((size_t)(qo[count] + 1) * 8, s)) != LBVH_OK) return fail_all(st);
    if ((st = slot->hits.ensure((size_t)std::max<uint64_t>(cap, 1) * 4, s)) != LBVH_OK) return fail_all(st);
    if ((st = slot->qbase.ensure((size_t)(count + 1) * 8, s)) != LBVH_OK) return fail_all(st);
    if ((st = slot->totals.ensure((size_t)count * 8, s)) != LBVH_OK) return fail_all(st);
    for (int k = 0; k < count; ++k) {
        const lbvh_request &r = job.reqs[k].req;
        if (r.n) cudaMemcpyAsync(slot->prims.as<float>() + po[k] * pdim, r.d_prims, (size_t)r.n * pdim * 4,
                                 cudaMemcpyDeviceToDevice, s);
        if (!self_query && r.nq)
            cudaMemcpyAsync(slot->queries.as<float>() + qo[k] * qdim, r.d_queries, (size_t)r.nq * qdim * 4,
                            cudaMemcpyDeviceToDevice, s);
        if (k0.qkind == LBVH_Q_SPHERE && r.nq) {
            if (r.d_radii)
                cudaMemcpyAsync(slot->radii.as<float>() + qo[k], r.d_radii, (size_t)r.nq * 4,
                                cudaMemcpyDeviceToDevice, s);
            else
                fill_kernel<<<grid_for(r.nq), 256, 0, s>>>(slot->radii.as<float>() + qo[k], r.nq, r.radius);
        }
    }
    cudaMemcpyAsync(slot->qbase.p, qo.data(), (size_t)(count + 1) * 8, cudaMemcpyHostToDevice, s);
    const Clock::time_point staged = Clock::now();
    const float *queries = self_query ? slot->prims.as<float>() : slot->queries.as<float>();
    const float *radii = k0.qkind == LBVH_Q_SPHERE ? slot->radii.as<float>() : nullptr;
    uint64_t total = 0;
    cudaEventRecord(slot->began, s);
    st = lbvh_batch_build_query(slot->batch, slot->prims.as<float>(), po.data(), count, k0.kind, k0.morton_bits,
                                queries, qo.data(), k0.qkind, radii, 0.0f, slot->offsets.as<int64_t>(),
                                slot->hits.as<uint32_t>(), std::max<uint64_t>(cap, 1), &total, s);
    if (st == LBVH_ERR_CAPACITY) {  // requests under-sized their buffers: rerun to learn each one's need
        if ((st = slot->hits.ensure((size_t)total * 4 + 4, s)) != LBVH_OK) return fail_all(st);
        st = lbvh_batch_build_query(slot->batch, slot->prims.as<float>(), po.data(), count, k0.kind,
                                    k0.morton_bits, queries, qo.data(), k0.qkind, radii, 0.0f,
                                    slot->offsets.as<int64_t>(), slot->hits.as<uint32_t>(), total + 1, &total, s);
    }
    if (st != LBVH_OK) return fail_all(st);
    cudaEventRecord(slot->ended, s);
    const Clock::time_point batched = Clock::now();
    request_totals_kernel<<<(count + 255) / 256, 256, 0, s>>>(slot->offsets.as<int64_t>(), slot->qbase.as<int64_t>(),
                                                              count, slot->totals.as<unsigned long long>());
    slot->h_totals.resize(count);
    cudaMemcpyAsync(slot->h_totals.data(), slot->totals.p, (size_t)count * 8, cudaMemcpyDeviceToHost, s);
    for (int k = 0; k < count; ++k) {
        const lbvh_request &r = job.reqs[k].req;
        rebase_offsets_kernel<<<grid_for(r.nq + 1), 256, 0, s>>>(slot->offsets.as<int64_t>(), qo[k], r.nq,
                                                                 r.d_offsets);
        if (r.d_hits && r.capacity)
            copy_hits_kernel<<<grid_for(r.nq * 16), 256, 0, s>>>(slot->offsets.as<int64_t>(), qo[k], r.nq,
                                                                 slot->hits.as<uint32_t>(), r.d_hits, r.capacity);
    }
    // trees that stay resident
    std::vector<std::pair<uint64_t, lbvh_tree_t>> keep;
    for (int k = 0; k < count; ++k) {
        const lbvh_request &r = job.reqs[k].req;
        if (!r.key) continue;
        lbvh_tree_t t = nullptr;
        if (lbvh_tree_create(&t) != LBVH_OK) continue;
        if (lbvh::tree_from_batch(slot->batch, k, t, s) != LBVH_OK) {
            lbvh_tree_destroy(t);
            continue;
        }
        keep.emplace_back(r.key, t);
    }
    cudaStreamSynchronize(s);
    std::lock_guard<std::mutex> lk(mu);
    record_span(slot);
    phase_s[0] += seconds_since(start, staged);
    phase_s[1] += seconds_since(staged, batched);
    phase_s[2] += seconds_since(batched, Clock::now());
    for (auto &kt : keep) {
        const uint64_t key = kt.first;
        auto old = resident.find(key);
        if (old != resident.end() && old->second.in_use == 0) {
            lbvh_tree_destroy(old->second.tree);
            resident_total -= old->second.bytes;
            lru.erase(old->second.lru);
            resident.erase(old);
        } else if (old != resident.end()) {
            lbvh_tree_destroy(kt.second);  // the old tree is being queried: keep it
            continue;
        }
        int64_t n = 0;
        lbvh_tree_size(kt.second, &n);
        Resident rs;
        rs.tree = kt.second;
        rs.bytes = resident_bytes_of(n, k0.kind);
        lru.push_front(key);
        rs.lru = lru.begin();
        resident[key] = rs;
        resident_total += rs.bytes;
    }
    for (int k = 0; k < count; ++k) {
        Request &r = job.reqs[k];
        const uint64_t need = slot->h_totals[k];
        complete(r, need > r.req.capacity ? LBVH_ERR_CAPACITY : LBVH_OK, need, start, count);
    }
    // the budget is exceeded only until the next admission evicts
}

extern "C" {

lbvh_status lbvh_server_create(uint64_t hbm_budget_bytes, int slots, int max_batch, lbvh_server_t *out) {
    if (!out || slots < 1 || slots > 16 || max_batch < 1 || hbm_budget_bytes == 0) return LBVH_ERR_INVALID;
    auto *srv = new (std::nothrow) lbvh_server_s();
    if (!srv) return LBVH_ERR_OOM;
    srv->budget = hbm_budget_bytes;
    srv->max_batch = max_batch;
    srv->max_batch_prims = (int64_t)1 << 25;
    for (int k = 0; k < slots; ++k) {
        auto slot = std::make_unique<Slot>();
        slot->index = k;
        if (cudaStreamCreateWithFlags(&slot->stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreate(&slot->began) != cudaSuccess || cudaEventCreate(&slot->ended) != cudaSuccess ||
            lbvh_batch_create(&slot->batch) != LBVH_OK) {
            srv->stop = true;
            lbvh_server_destroy(srv);
            return LBVH_ERR_CUDA;
        }
        lbvh::batch_set_graphs(slot->batch, false);
        srv->slots.push_back(std::move(slot));
    }
    if (cudaEventCreate(&srv->ref) != cudaSuccess || cudaEventRecord(srv->ref, srv->slots[0]->stream) != cudaSuccess ||
        cudaEventSynchronize(srv->ref) != cudaSuccess) {
        srv->stop = true;
        lbvh_server_destroy(srv);
        return LBVH_ERR_CUDA;
    }
    for (auto &slot : srv->slots) {
        Slot *sp = slot.get();
        slot->worker = std::thread([srv, sp] { srv->worker_loop(sp); });
    }
    srv->scheduler = std::thread([srv] { srv->schedule_loop(); });
    *out = srv;
    return LBVH_OK;
}

lbvh_status lbvh_server_submit(lbvh_server_t srv, const lbvh_request *req, uint64_t *ticket) {
    if (!srv || !req || !ticket) return LBVH_ERR_INVALID;
    const lbvh_request &r = *req;
    if (r.n < 0 || r.n > LBVH_MAX_PRIMS || r.nq < 0 || r.nq > LBVH_MAX_PRIMS) return LBVH_ERR_INVALID;
    if (r.kind != LBVH_PRIM_POINTS && r.kind != LBVH_PRIM_BOXES) return LBVH_ERR_INVALID;
    if (r.qkind != LBVH_Q_SPHERE && r.qkind != LBVH_Q_BOX && r.qkind != LBVH_Q_RAY) return LBVH_ERR_INVALID;
    if (r.qkind == LBVH_Q_RAY && r.n > 0) return LBVH_ERR_INVALID;  // rays: query-only requests
    if (r.n > 0 && (!r.d_prims || r.morton_bits < 3 || r.morton_bits > 63 || r.morton_bits % 3)) return LBVH_ERR_INVALID;
    if (r.n == 0 && r.key == 0) return LBVH_ERR_INVALID;  // query-only needs a resident tree
    if (r.nq > 0 && !r.d_queries) return LBVH_ERR_INVALID;
    if (!r.d_offsets || (r.capacity > 0 && !r.d_hits)) return LBVH_ERR_INVALID;
    if (r.qkind == LBVH_Q_SPHERE && !r.d_radii && !(r.radius >= 0.0f && r.radius <= 3.0e38f)) return LBVH_ERR_INVALID;
    Request q;
    q.req = r;
    q.est_bytes = estimate_bytes(r);
    q.submitted = Clock::now();
    std::lock_guard<std::mutex> lk(srv->mu);
    q.ticket = srv->next_ticket++;
    srv->outcomes[q.ticket] = Outcome{};
    srv->pending.push_back(q);
    *ticket = q.ticket;
    srv->cv_sched.notify_all();
    return LBVH_OK;
}

lbvh_status lbvh_server_wait(lbvh_server_t srv, uint64_t ticket, lbvh_result *out) {
    if (!srv || !out) return LBVH_ERR_INVALID;
    std::unique_lock<std::mutex> lk(srv->mu);
    auto it = srv->outcomes.find(ticket);
    if (it == srv->outcomes.end()) return LBVH_ERR_INVALID;
    srv->cv_done.wait(lk, [&] { return srv->outcomes[ticket].done; });
    *out = srv->outcomes[ticket].result;
    srv->outcomes.erase(ticket);
    return LBVH_OK;
}

lbvh_status lbvh_server_stats(lbvh_server_t srv, uint64_t *resident_bytes, uint64_t *resident_trees,
                              uint64_t *evictions, uint64_t *batches) {
    if (!srv) return LBVH_ERR_INVALID;
    std::lock_guard<std::mutex> lk(srv->mu);
    if (resident_bytes) *resident_bytes = srv->resident_total;
    if (resident_trees) *resident_trees = srv->resident.size();
    if (evictions) *evictions = srv->evictions;
    if (batches) *batches = srv->batches;
    return LBVH_OK;
}

lbvh_status lbvh_server_latency(lbvh_server_t srv, double *p50_s, double *p99_s, uint64_t *count) {
    if (!srv) return LBVH_ERR_INVALID;
    std::vector<double> v;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        v = srv->latencies;
    }
    if (count) *count = v.size();
    // nearest-rank percentiles
    auto pct = [&](double p) {
        if (v.empty()) return 0.0;
        size_t k = (size_t)std::ceil(p / 100.0 * (double)v.size());
        k = k == 0 ? 0 : k - 1;
        std::nth_element(v.begin(), v.begin() + k, v.end());
        return v[k];
    };
    if (p50_s) *p50_s = pct(50.0);
    if (p99_s) *p99_s = pct(99.0);
    return LBVH_OK;
}

lbvh_status lbvh_server_device_spans(lbvh_server_t srv, double *spans, uint64_t capacity, uint64_t *count) {
    if (!srv || !count || (capacity > 0 && !spans)) return LBVH_ERR_INVALID;
    std::lock_guard<std::mutex> lk(srv->mu);
    const uint64_t have = srv->spans.size() / 3;
    *count = have;
    const uint64_t n = std::min<uint64_t>(have, capacity);
    std::copy(srv->spans.begin(), srv->spans.begin() + 3 * n, spans);
    return LBVH_OK;
}

lbvh_status lbvh_server_phase_seconds(lbvh_server_t srv, double *seconds) {
    if (!srv || !seconds) return LBVH_ERR_INVALID;
    std::lock_guard<std::mutex> lk(srv->mu);
    for (int k = 0; k < LBVH_SERVER_PHASES; ++k) seconds[k] = srv->phase_s[k];
    return LBVH_OK;
}

void lbvh_server_destroy(lbvh_server_t srv) {
    if (!srv) return;
    {
        std::unique_lock<std::mutex> lk(srv->mu);
        // finish queued and running work first
        srv->cv_done.wait(lk, [&] {
            return srv->pending.empty() &&
                   std::none_of(srv->slots.begin(), srv->slots.end(), [](const std::unique_ptr<Slot> &s) { return s->busy; });
        });
        srv->stop = true;
    }
    srv->cv_sched.notify_all();
    srv->cv_slot.notify_all();
    if (srv->scheduler.joinable()) srv->scheduler.join();
    for (auto &slot : srv->slots)
        if (slot->worker.joinable()) slot->worker.join();
    for (auto &kv : srv->resident) lbvh_tree_destroy(kv.second.tree);
    for (auto &slot : srv->slots) {
        for (Buf *b : {&slot->prims, &slot->queries, &slot->radii, &slot->offsets, &slot->hits, &slot->qbase,
                       &slot->totals})
            b->release(slot->stream);
        lbvh_batch_destroy(slot->batch);
        cudaStreamSynchronize(slot->stream);
        cudaStreamDestroy(slot->stream);
        if (slot->began) cudaEventDestroy(slot->began);
        if (slot->ended) cudaEventDestroy(slot->ended);
    }
    if (srv->ref) cudaEventDestroy(srv->ref);
    delete srv;
}

}  // extern "C"
