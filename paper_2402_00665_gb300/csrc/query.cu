// query.cu -- stackless range queries (Algorithm 1) and CSR assembly.
//
// Each thread walks the tree for one query: start at the root (id 0); when
// the predicate holds on an internal node go to its left child, on a leaf
// report it and go to its skip; when it fails go to the skip; stop at the
// sentinel. Every step runs the same code for internal nodes and leaves: a
// 16-byte load (internal: lo + left; point leaf: xyz + index word), a second
// one for internal nodes and box leaves (hi + skip), the box test, and a
// select. A leaf's skip is position k+1, leaf or internal by one bit.
//
// Predicates (closed, FP32, fixed operation order):
//   sphere  e_a = max(lo_a - c_a, c_a - hi_a, 0);
//           d2 = fma(ez, ez, fma(ey, ey, ex*ex)) (each step rounded once);
//           hit iff d2 <= r*r. Every step is monotone in e_a >= 0, so a
//           node's d2 never exceeds the d2 of a primitive inside it: the walk
//           prunes nothing a brute-force scan would report. e_a is computed
//           as c_a - clamp(c_a, lo_a, hi_a), which has the same magnitude
//           because fl(x - y) = -fl(y - x).
//   box     lo_q <= hi_b and lo_b <= hi_q on every axis.
//   ray     the slab test of a segment {origin, tmin, direction, tmax}
//           (see hits(const Ray &...)); rays are walked in input order.
//
// Threads take the queries in the order given by QueryArgs::order (the
// queries sorted by the Morton code of their centre, so that a warp's walks
// visit the same nodes), and write results at the query's own index.
//
// CSR in one walk:
//   collect   each thread walks sorted position i (query q = order[i]; groups
//             of lanes walking together are a tuning option) and writes up
//             to kQueryBufferHits primitive ids, in walk order, into slot q
//             of a scratch array (no shared memory: L1 stays with the tree),
//             and the hit count at q. Slot q rather than slot i: the copy
//             then reads the slots in order (copy 1.86 -> 1.45 ms on 2^25
//             uniform points; the walk's stores are scattered either way).
//   scan      exclusive scan of the counts -> offsets, total (host reads it).
//   copy      in query order: each thread loads one slot of up to 32 hits
//             into registers and sorts it with a bitonic network; the warp
//             writes its 32 lists, adjacent in the CSR, through shared
//             memory, one coalesced list per step; lists of 33..64 hits are
//             sorted by the whole warp (two values per lane, shuffles).
//   overflow  hits past the slot go on, during the same walk, to chunks of a
//             shared spill pool; those lists are copied (slot + chunks) to
//             their CSR ranges; only when the pool runs out does a query walk
//             a second time, writing straight into the CSR. A fix-up kernel
//             then sorts every such list, one warp per list (one CTA per list
//             above 1024 hits).
#include <algorithm>
#include <cstdlib>
#include <type_traits>

#include "lbvh_internal.cuh"
#include "morton.cuh"

namespace lbvh {

namespace {

constexpr int kThreads = 256;

struct Sphere {
    float3 c;
    float r2;
};
struct Box {
    float3 lo, hi;
};
// A ray segment: origin, 1/direction per axis (IEEE division), which axes
// are parallel (direction 0, or a reciprocal that overflows), and [tmin, tmax].
struct Ray {
    float3 o, inv;
    float tmin, tmax;
    uint32_t parallel;  // bit a: axis a
};

// |gap| between c and [lo, hi]: c - clamp(c, lo, hi) (sign irrelevant: squared)
__device__ __forceinline__ float gap(float lo, float c, float hi) {
    return __fsub_rn(c, fminf(fmaxf(c, lo), hi));
}

// Squared distance from c to the box: ex*ex, then + ey*ey and + ez*ez each
// as one fused multiply-add.
__device__ __forceinline__ float box_d2(float3 c, float3 lo, float3 hi) {
    const float ex = gap(lo.x, c.x, hi.x);
    const float ey = gap(lo.y, c.y, hi.y);
    const float ez = gap(lo.z, c.z, hi.z);
    return __fmaf_rn(ez, ez, __fmaf_rn(ey, ey, __fmul_rn(ex, ex)));
}

__device__ __forceinline__ bool hits(const Sphere &s, float3 lo, float3 hi) { return box_d2(s.c, lo, hi) <= s.r2; }

// Slab test, each operation rounded once: per axis t1 = (lo - o) * inv and
// t2 = (hi - o) * inv; tnear = max(tmin, min(t1, t2)), tfar = min(tmax,
// max(t1, t2)); a parallel axis instead requires lo <= o <= hi. Hit iff
// tnear <= tfar. Monotone in the box, like the other predicates.
__device__ __forceinline__ bool slab(float lo, float hi, float o, float inv, bool parallel, float &tn,
                                     float &tf) {
    if (parallel) return lo <= o && o <= hi;
    const float t1 = __fmul_rn(__fsub_rn(lo, o), inv), t2 = __fmul_rn(__fsub_rn(hi, o), inv);
    tn = fmaxf(tn, fminf(t1, t2));
    tf = fminf(tf, fmaxf(t1, t2));
    return true;
}

__device__ __forceinline__ bool hits(const Ray &r, float3 lo, float3 hi) {
    float tn = r.tmin, tf = r.tmax;
    if (!slab(lo.x, hi.x, r.o.x, r.inv.x, r.parallel & 1u, tn, tf)) return false;
    if (!slab(lo.y, hi.y, r.o.y, r.inv.y, r.parallel & 2u, tn, tf)) return false;
    if (!slab(lo.z, hi.z, r.o.z, r.inv.z, r.parallel & 4u, tn, tf)) return false;
    return tn <= tf;
}

__device__ __forceinline__ bool hits(const Box &q, float3 lo, float3 hi) {
    return q.lo.x <= hi.x && lo.x <= q.hi.x && q.lo.y <= hi.y && lo.y <= q.hi.y &&
           q.lo.z <= hi.z && lo.z <= q.hi.z;
}

template <int kQ>
struct QueryOf;
template <>
struct QueryOf<LBVH_Q_SPHERE> {
    using type = Sphere;
    static __device__ __forceinline__ Sphere load(const QueryArgs &a, int64_t q) {
        const float *p = a.queries + 3 * q;
        const float r = a.radii ? __ldcs(a.radii + q) : a.radius;
        return Sphere{make_float3(__ldcs(p), __ldcs(p + 1), __ldcs(p + 2)), __fmul_rn(r, r)};
    }
};
template <>
struct QueryOf<LBVH_Q_RAY> {
    using type = Ray;
    static __device__ __forceinline__ float axis_inv(float d, uint32_t bit, uint32_t &parallel) {
        const float inv = __fdiv_rn(1.0f, d);
        if (d == 0.0f || isinf(inv)) parallel |= bit;
        return inv;
    }
    static __device__ __forceinline__ Ray load(const QueryArgs &a, int64_t q) {
        const float4 *p = reinterpret_cast<const float4 *>(a.queries) + 2 * q;
        const float4 u = __ldcs(p), v = __ldcs(p + 1);
        Ray r;
        r.parallel = 0;
        r.o = make_float3(u.x, u.y, u.z);
        r.inv = make_float3(axis_inv(v.x, 1u, r.parallel), axis_inv(v.y, 2u, r.parallel),
                            axis_inv(v.z, 4u, r.parallel));
        r.tmin = u.w;
        r.tmax = v.w;
        const bool finite = isfinite(u.x) && isfinite(u.y) && isfinite(u.z) && isfinite(v.x) && isfinite(v.y) &&
                            isfinite(v.z) && !isnan(u.w) && !isnan(v.w);
        if (!finite) {  // hits nothing: an empty parameter interval on every axis
            r.tmin = 1.0f;
            r.tmax = 0.0f;
            r.parallel = 0;
            r.o = make_float3(0.0f, 0.0f, 0.0f);
            r.inv = make_float3(1.0f, 1.0f, 1.0f);
        }
        return r;
    }
};
template <>
struct QueryOf<LBVH_Q_BOX> {
    using type = Box;
    static __device__ __forceinline__ Box load(const QueryArgs &a, int64_t q) {
        const float *p = a.queries + 6 * q;
        return Box{make_float3(__ldcs(p), __ldcs(p + 1), __ldcs(p + 2)),
                   make_float3(__ldcs(p + 3), __ldcs(p + 4), __ldcs(p + 5))};
    }
};

__device__ __forceinline__ float3 xyz(float4 v) { return make_float3(v.x, v.y, v.z); }

// A node record as one 32-byte load (two float4 halves), read-only path.
// Records of two float4 start on 32-byte boundaries (internal nodes and box
// leaves; batches pad every tree to an even float4 offset).
__device__ __forceinline__ void ld_node32(const float4 *p, float4 &a, float4 &b) {
    asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
        : "l"(p));
}

// The node at `unit` (float4 units). In a box tree every record is 32 bytes:
// one 32-byte load per step (measured: D3's walk 10.14 -> 8.39 ms). In a
// point tree a leaf is one float4 (its box is its point): a first 16-byte
// load common to every lane and a second one for internal nodes measured
// faster than splitting the warp between a 16- and a 32-byte load.
template <int kP>
__device__ __forceinline__ void load_node(const float4 *base, int unit, bool leaf, float4 &a, float4 &b) {
    if (kP == LBVH_PRIM_BOXES) {
        ld_node32(base + unit, a, b);
    } else {
        a = __ldg(base + unit);
        b = a;
        if (!leaf) b = __ldg(base + unit + 1);
    }
}

// Algorithm 1. on_leaf(id) is called with the primitive index of every leaf
// that satisfies the predicate, leaves in increasing sorted position. Returns
// false if the walk ran past 2(2n-1) steps or met an id outside the tree (a
// corrupt tree).
template <int kP, typename Q, typename F>
__device__ __forceinline__ bool walk(const TreeView &t, const Q &q, F &&on_leaf) {
    const int ni = (int)t.n - 1;
    const int nodes = 2 * (int)t.n - 1;
    const uint32_t max_steps = 2u * (uint32_t)nodes;
    const float4 *base = t.inodes;  // leaves follow the internal records
    int node = 0;
    uint32_t steps = 0;
    // ids outside [0, nodes) end the loop: the sentinel, one past the last
    // leaf (the last leaf's skip), or a corrupt id (reported below)
    while ((uint32_t)node < (uint32_t)nodes) {
        if (++steps > max_steps) return false;
        const bool leaf = node >= ni;
        const int unit = kP == LBVH_PRIM_BOXES ? 2 * node : (leaf ? node + ni : 2 * node);
        float4 a, b;
        load_node<kP>(base, unit, leaf, a, b);
        const bool hit = hits(q, xyz(a), xyz(b));
        const uint32_t word = __float_as_uint(a.w);
        if (hit && leaf) on_leaf(word & kLeafIndexMask);
        // internal: left child on a hit, else skip; leaf k: position k+1
        node = leaf ? node + 1 - ((word & kLeafSkipInternal) ? ni : 0)
                    : __float_as_int(hit ? a.w : b.w);
    }
    return node == kSentinel || node == nodes;
}

// Algorithm 1 walked by a group of kLanes adjacent lanes together (8, 16 or
// 32): the group stands at one node, every lane tests its own query there,
// and at an internal node the group goes to the left child if any lane's
// predicate holds, else to the skip. Every lane calls on_leaf for each leaf
// its own predicate accepts. The group's walk visits every node that one of
// its lanes' own walks visits (a leaf a lane accepts has all its ancestors
// accepted by that lane, the predicates being monotone), in the same
// pre-order, so each lane reports exactly its own walk's hits, in the same
// order. A step loads one node for the whole group (a broadcast) instead of
// one per lane, and walks the union of the lanes' paths. Lanes without a
// query (active false) walk along and report nothing.
template <int kP, int kLanes, typename Q, typename F>
__device__ __forceinline__ bool walk_group(const TreeView &t, const Q &q, bool active, F &&on_leaf) {
    const int ni = (int)t.n - 1;
    const int nodes = 2 * (int)t.n - 1;
    const uint32_t max_steps = 2u * (uint32_t)nodes;
    const float4 *base = t.inodes;
    const int lane = threadIdx.x & 31;
    const uint32_t gmask =
        kLanes == 32 ? 0xffffffffu : (((1u << kLanes) - 1u) << (lane & ~(kLanes - 1)));
    int node = 0;
    uint32_t steps = 0;
    while ((uint32_t)node < (uint32_t)nodes) {
        if (++steps > max_steps) return false;
        const bool leaf = node >= ni;
        const int unit = kP == LBVH_PRIM_BOXES ? 2 * node : (leaf ? node + ni : 2 * node);
        float4 a, b;
        load_node<kP>(base, unit, leaf, a, b);
        const bool hit = active && hits(q, xyz(a), xyz(b));
        const uint32_t word = __float_as_uint(a.w);
        if (leaf) {
            if (hit) on_leaf(word & kLeafIndexMask);
            node = node + 1 - ((word & kLeafSkipInternal) ? ni : 0);
        } else {
            node = __float_as_int((__ballot_sync(gmask, hit) & gmask) ? a.w : b.w);
        }
    }
    return node == kSentinel || node == nodes;
}

constexpr int kSlot = kQueryBufferHits;  // ids kept per walk (slot size)
constexpr int kRegSort = 32;             // lists up to this long are sorted in one thread's registers

__device__ __forceinline__ int64_t thread_query(const QueryArgs &qa, int64_t i) {
    return qa.order ? (int64_t)__ldcs(qa.order + i) : i;
}

// Hits past a walk's slot: appended to chunks from the shared pool, the first
// chunk recorded in spill_head[q], each chunk's word 0 linking to the next.
// `cur` is the walk's current chunk (kNoChunk before the first); it becomes
// kSpillFailed when the pool is exhausted, and the query then takes the
// second walk.
constexpr uint32_t kNoChunk = 0xffffffffu, kSpillFailed = 0xfffffffeu;

__device__ __forceinline__ void spill_put(const QueryScratch &qs, Control *ctl, int64_t i, uint32_t cnt,
                                          uint32_t id, uint32_t &cur) {
    if (cur == kSpillFailed) return;
    const uint32_t sidx = cnt - (uint32_t)kSlot;                   // index among the spilled hits
    const uint32_t off = sidx % (uint32_t)(kSpillChunkWords - 1);  // slot in the chunk (after the link)
    if (off == 0) {
        const uint32_t fresh = atomicAdd(&ctl->spill_used, 1u);
        if (fresh >= qs.spill_chunks) {
            cur = kSpillFailed;
            return;
        }
        if (cur == kNoChunk) qs.spill_head[i] = fresh;
        else qs.spill[(int64_t)cur * kSpillChunkWords] = fresh;
        cur = fresh;
    }
    qs.spill[(int64_t)cur * kSpillChunkWords + 1 + off] = id;
}

// One query's collecting walk at walk position i (query qi): the first kSlot
// hits go to the slot, later ones to spill chunks. Writes (count, i) and, for
// a long list, its overflow-list entry (tagged when all its hits are in slot
// + chunks).
// kLanes = 0: the thread walks alone (walk); else with its group of kLanes
// lanes (walk_group; every lane of the warp must call this, `has_query`
// false for lanes past the last query).
template <int kQ, int kP, bool kPairs, int kLanes = 0>
__device__ __forceinline__ void collect_walk(const TreeView &t, const QueryArgs &qa, const QueryScratch &qs,
                                             Control *ctl, int64_t i, int64_t qi, bool walk_ok,
                                             bool has_query = true) {
    uint32_t cnt = 0;
    uint32_t cur = kNoChunk;
    if (walk_ok) {
        const auto q = has_query ? QueryOf<kQ>::load(qa, qi) : typename QueryOf<kQ>::type{};
        uint32_t *slot = qs.slots + qi * kSlot;
        // kPairs: hits go to the slot two at a time (one 8-byte store; words
        // past the count are never read). Point trees, one tree: walk 16.19
        // -> 15.87 ms on 2^25 uniform points (held to 32 registers, with an
        // 8-byte spill; 16.00 ms at 40 registers); on box trees it cost more
        // (D3 walk 8.39 -> 8.49 ms at 40 registers).
        uint2 buf = make_uint2(0u, 0u);
        auto keep = [&](uint32_t id) {
            if (cnt < (uint32_t)kSlot) {
                if (!kPairs) {
                    __stcs(slot + cnt, id);
                } else if (cnt & 1u) {
                    buf.y = id;
                    __stcs(reinterpret_cast<uint2 *>(slot + cnt - 1), buf);
                } else {
                    buf.x = id;
                }
            } else {
                spill_put(qs, ctl, qi, cnt, id, cur);
            }
            ++cnt;
        };
        bool ok;
        if constexpr (kLanes == 0)
            ok = walk<kP>(t, q, keep);
        else
            ok = walk_group<kP, kLanes>(t, q, has_query, keep);
        if (!has_query) return;
        if (kPairs && cnt < (uint32_t)kSlot && (cnt & 1u)) __stcs(reinterpret_cast<uint2 *>(slot + cnt - 1), buf);
        if (!ok) atomicOr(&ctl->query_flags, kFlagCorrupt);
    }
    if (!has_query) return;
    __stcs(qs.counts + qi, cnt);  // streamed: keep L2 for the tree
    if (cnt > (uint32_t)kSlot)
        qs.overflow_list[atomicAdd(&ctl->overflow_filled, 1u)] =
            (uint32_t)qi | (cur != kSpillFailed ? kSpilledTag : 0u);
}

// The collecting walk with groups of kLanes lanes walking together
// (walk_group); thread i takes walk position i as in collect_kernel.
template <int kQ, int kP, int kLanes>
__global__ void __launch_bounds__(kThreads, 8)
    collect_group_kernel(TreeView t, QueryArgs qa, QueryScratch qs, Control *ctl) {
    const int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    const int64_t warp_first = i - (threadIdx.x & 31);
    if (warp_first >= qa.nq) return;  // whole warps leave together
    const bool has = i < qa.nq;
    const bool walk_ok = t.n > 0 && ctl->build_flags == 0;
    collect_walk<kQ, kP, kP == LBVH_PRIM_POINTS, kLanes>(t, qa, qs, ctl, i, has ? thread_query(qa, i) : 0, walk_ok,
                                                       has);
}

// One thread per walk position: thread i walks position i (query order[i]).
// At most 32 registers (2048 threads per SM): the walk hides its load latency
// with occupancy. Several walks per thread in lock step (K independent loads
// in flight per thread) measured slower on GB300: the walk is bound by L1
// wavefronts (distinct sectors per load), which more walks per thread only
// increase. kT threads per CTA (256 or 512, a tuner choice): the CTAs that
// share an SM's L1 walk kT adjacent queries each, so larger CTAs put more
// neighbouring walks on one SM (D2 walk 15.93 -> 15.66 ms with 512; 1024
// measured slower on D2 and D3).
template <int kQ, int kP, int kT>
__global__ void __launch_bounds__(kT, 2048 / kT)
    collect_kernel(TreeView t, QueryArgs qa, QueryScratch qs, Control *ctl) {
    const int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x;
    if (i >= qa.nq) return;
    const bool walk_ok = t.n > 0 && ctl->build_flags == 0;
    collect_walk<kQ, kP, kP == LBVH_PRIM_POINTS>(t, qa, qs, ctl, i, thread_query(qa, i), walk_ok);
}

// Batcher's odd-even merge sort of v[0..kN) (kN a power of two), keeping only
// the comparators inside v[0..kAct). Every comparator puts the smaller value
// at the lower index, so padding values ~0u at the top never move and the
// comparators that reach them do nothing: the pruned network sorts kAct
// values (8: 19 comparators, 16: 63, 24: 132, 32: 191; a bitonic network
// over 32 takes 240). Written as templates so that every index is a
// compile-time constant and v stays in registers.
template <int kAct>
__device__ __forceinline__ void compare_swap(uint32_t (&v)[32], int x, int y) {
    if (y < kAct) {
        const uint32_t a = v[x], b = v[y];
        v[x] = min(a, b);
        v[y] = max(a, b);
    }
}

// merges the two sorted halves of the elements lo, lo + r, lo + 2r, ... of v[lo, lo + n)
template <int kLo, int kN, int kR, int kAct>
struct OddEvenMerge {
    static __device__ __forceinline__ void run(uint32_t (&v)[32]) {
        constexpr int m = 2 * kR;
        if constexpr (m < kN) {
            OddEvenMerge<kLo, kN, m, kAct>::run(v);
            OddEvenMerge<kLo + kR, kN, m, kAct>::run(v);
#pragma unroll
            for (int i = kLo + kR; i + kR < kLo + kN; i += m) compare_swap<kAct>(v, i, i + kR);
        } else {
            compare_swap<kAct>(v, kLo, kLo + kR);
        }
    }
};

template <int kLo, int kN, int kAct>
struct OddEvenSort {
    static __device__ __forceinline__ void run(uint32_t (&v)[32]) {
        if constexpr (kN > 1) {
            OddEvenSort<kLo, kN / 2, kAct>::run(v);
            OddEvenSort<kLo + kN / 2, kN / 2, kAct>::run(v);
            OddEvenMerge<kLo, kN, 1, kAct>::run(v);
        }
    }
};

template <int kN, int kAct>
__device__ __forceinline__ void merge_sort_net(uint32_t (&v)[32]) {
    OddEvenSort<0, kN, kAct>::run(v);
}

// Ascending bitonic sort of 64 values held by a warp, value e in lane e % 32
// (v0: e < 32, v1: e >= 32). Steps with partner distance 32 compare a lane's
// two values; the others exchange with lane ^ j by shuffle.
__device__ __forceinline__ void warp_sort64(uint32_t &v0, uint32_t &v1) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 2; k <= 64; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j == 32) {  // k == 64: one ascending merge
                const uint32_t lo = min(v0, v1), hi = max(v0, v1);
                v0 = lo;
                v1 = hi;
            } else {
                const bool lower = (lane & j) == 0;
                const uint32_t p0 = __shfl_xor_sync(0xffffffffu, v0, j);
                const uint32_t p1 = __shfl_xor_sync(0xffffffffu, v1, j);
                const bool up0 = (lane & k) == 0, up1 = ((lane + 32) & k) == 0;
                v0 = lower == up0 ? min(v0, p0) : max(v0, p0);
                v1 = lower == up1 ? min(v1, p1) : max(v1, p1);
            }
        }
    }
}

// Thread q sorts query q's list in registers if it has at most 32 hits; the
// warp then writes its 32 lists, which are adjacent in the CSR, one list per
// step with lanes on consecutive hits. Lists of 33..64 hits are then sorted
// and written by the whole warp, one after the other.
__global__ void __launch_bounds__(kThreads)
    copy_kernel(int64_t nq, const uint32_t *__restrict__ counts, const int64_t *__restrict__ offsets,
                const uint32_t *__restrict__ slots, uint32_t *__restrict__ hits,
                unsigned long long capacity, Control *ctl) {
    __shared__ uint32_t s_lists[kThreads / 32][32][kRegSort + 1];
    if (ctl->total > capacity) {  // the caller's buffer is too small: write nothing
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&ctl->query_flags, kFlagCapacity);
        return;
    }
    const int64_t q = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t c = 0, mid = 0;
    int64_t dst = 0, pos = 0;
    if (q < nq) {
        const uint32_t cq = counts[q];
        c = cq > (uint32_t)kRegSort ? 0u : cq;
        mid = cq > (uint32_t)kRegSort && cq <= (uint32_t)kSlot ? cq : 0u;  // longer: the overflow walk
        pos = q;
        dst = offsets[q];
    }
    uint32_t mids = __ballot_sync(0xffffffffu, mid != 0);
    if (!__any_sync(0xffffffffu, c != 0) && mids == 0) return;
    uint32_t v[kRegSort];
    const uint4 *src = reinterpret_cast<const uint4 *>(slots + pos * kSlot);
#pragma unroll
    for (int j4 = 0; j4 < kRegSort / 4; ++j4) {
        uint4 w = make_uint4(~0u, ~0u, ~0u, ~0u);
        if (4 * j4 < (int)c) w = src[j4];
        v[4 * j4] = 4 * j4 < (int)c ? w.x : ~0u;
        v[4 * j4 + 1] = 4 * j4 + 1 < (int)c ? w.y : ~0u;
        v[4 * j4 + 2] = 4 * j4 + 2 < (int)c ? w.z : ~0u;
        v[4 * j4 + 3] = 4 * j4 + 3 < (int)c ? w.w : ~0u;
    }
    // the network for the warp's longest list (lists are padded with ~0u)
    const uint32_t cmax = __reduce_max_sync(0xffffffffu, c);
    if (cmax > 24)
        merge_sort_net<32, 32>(v);
    else if (cmax > 16)
        merge_sort_net<32, 24>(v);
    else if (cmax > 8)
        merge_sort_net<16, 16>(v);
    else if (cmax > 1)
        merge_sort_net<8, 8>(v);
#pragma unroll
    for (int j = 0; j < kRegSort; ++j)
        if (j < (int)cmax) s_lists[warp][lane][j] = v[j];
    __syncwarp();
    for (int s = 0; s < 32; ++s) {
        const uint32_t cs = __shfl_sync(0xffffffffu, c, s);
        const int64_t ds = __shfl_sync(0xffffffffu, dst, s);
        if ((uint32_t)lane < cs) hits[ds + lane] = s_lists[warp][s][lane];
    }
    while (mids) {
        const int s = __ffs(mids) - 1;
        mids &= mids - 1;
        const uint32_t m = __shfl_sync(0xffffffffu, mid, s);
        const int64_t ps = __shfl_sync(0xffffffffu, pos, s);
        const int64_t ds = __shfl_sync(0xffffffffu, dst, s);
        const uint32_t *slot = slots + ps * kSlot;
        uint32_t v0 = (uint32_t)lane < m ? slot[lane] : ~0u;
        uint32_t v1 = (uint32_t)lane + 32 < m ? slot[lane + 32] : ~0u;
        warp_sort64(v0, v1);
        if ((uint32_t)lane < m) hits[ds + lane] = v0;
        if ((uint32_t)lane + 32 < m) hits[ds + lane + 32] = v1;
    }
}

// Second walk for the overflow list: hits go straight to the CSR in walk
// order (sorted afterwards by the list sorts).
template <int kQ, int kP>
__global__ void __launch_bounds__(kThreads)
    overflow_walk_kernel(TreeView t, QueryArgs qa, const uint32_t *__restrict__ list, uint32_t count,
                         const int64_t *__restrict__ offsets, uint32_t *__restrict__ hits) {
    const int64_t j = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (j >= count) return;
    const uint32_t e = list[j];
    if (e & kSpilledTag) return;  // its hits are in its slot and spill chunks
    const int64_t qi = e;
    const int64_t base = offsets[qi];
    const int64_t total = offsets[qi + 1] - base;
    const auto q = QueryOf<kQ>::load(qa, qi);
    int64_t c = 0;
    walk<kP>(t, q, [&](uint32_t id) {
        if (c < total) hits[base + c] = id;
        ++c;
    });
}

// ---------------------------------------------------------------- scan
constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ int64_t block_scan_exclusive(int64_t v, int64_t *s_warp, int64_t &total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t x = v;
    for (int off = 1; off < 32; off <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, x, off);
        if (lane >= off) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    int64_t before = 0, all = 0;
    for (int w = 0; w < kScanThreads / 32; ++w) {
        if (w < warp) before += s_warp[w];
        all += s_warp[w];
    }
    __syncthreads();
    total = all;
    return before + x - v;
}

__global__ void __launch_bounds__(kScanThreads)
    scan_reduce_kernel(const uint32_t *__restrict__ counts, int64_t nq, int64_t *tile_sums) {
    __shared__ int64_t s_warp[kScanThreads / 32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    int64_t sum = 0;
    for (int j = 0; j < kScanItems; ++j) {
        const int64_t i = base + j * kScanThreads + threadIdx.x;
        if (i < nq) sum += counts[i];
    }
    int64_t total;
    block_scan_exclusive(sum, s_warp, total);
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanThreads)
    scan_tiles_kernel(int64_t *tile_sums, int64_t tiles, int64_t *offsets, int64_t nq,
                      unsigned long long *total_out) {
    __shared__ int64_t s_warp[kScanThreads / 32];
    int64_t carry = 0;
    for (int64_t base = 0; base < tiles; base += kScanThreads) {
        const int64_t i = base + threadIdx.x;
        const int64_t v = i < tiles ? tile_sums[i] : 0;
        int64_t total;
        const int64_t ex = block_scan_exclusive(v, s_warp, total);
        if (i < tiles) tile_sums[i] = carry + ex;
        carry += total;
    }
    if (threadIdx.x == 0) {
        offsets[nq] = carry;
        *total_out = (unsigned long long)carry;
    }
}

// Loads and stores run across the block (thread t at t, t + 256, ...); each
// thread scans kScanItems consecutive counts, which it reads from and writes
// back to shared memory (rows padded by one element against bank conflicts).
__global__ void __launch_bounds__(kScanThreads)
    scan_apply_kernel(const uint32_t *__restrict__ counts, int64_t nq,
                      const int64_t *__restrict__ tile_sums, int64_t *__restrict__ offsets) {
    constexpr int kRow = kScanItems + 1;
    __shared__ int64_t s_warp[kScanThreads / 32];
    __shared__ int64_t s_o[kScanThreads * kRow];  // the offsets; first the counts (the scan's barriers
                                                  // separate the last read of a count from the first offset)
    uint32_t *s_c = reinterpret_cast<uint32_t *>(s_o);
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        const int p = j * kScanThreads + threadIdx.x;
        const int64_t i = base + p;
        s_c[(p / kScanItems) * kRow + p % kScanItems] = i < nq ? counts[i] : 0u;
    }
    __syncthreads();
    uint32_t c[kScanItems];
    int64_t sum = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        c[j] = s_c[threadIdx.x * kRow + j];
        sum += c[j];
    }
    int64_t total;
    int64_t run = tile_sums[blockIdx.x] + block_scan_exclusive(sum, s_warp, total);
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        s_o[threadIdx.x * kRow + j] = run;
        run += c[j];
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        const int p = j * kScanThreads + threadIdx.x;
        const int64_t i = base + p;
        if (i < nq) offsets[i] = s_o[(p / kScanItems) * kRow + p % kScanItems];
    }
}

// ---------------------------------------------------------------- fix-up sort
constexpr int kFixThreads = 512;
constexpr int kFixSmem = 8192;

__device__ __forceinline__ void order_pair(uint32_t *a, int64_t lo, int64_t hi) {
    const uint32_t x = a[lo], y = a[hi];
    if (x > y) {
        a[lo] = y;
        a[hi] = x;
    }
}

// Bitonic sorting network in its one-direction form: every comparator puts
// the smaller value at the lower index (the first step of each merge pairs i
// with the mirror position in its block, later steps pair i with i + j).
// Positions >= m act as +infinity and their comparators are skipped, which
// leaves the network correct for any m.
__device__ void bitonic_sort(uint32_t *a, int64_t m) {
    int64_t pow2 = 1;
    while (pow2 < m) pow2 <<= 1;
    for (int64_t k = 2; k <= pow2; k <<= 1) {
        const int64_t half = k >> 1;
        for (int64_t i = threadIdx.x; i < pow2 / 2; i += blockDim.x) {
            const int64_t blk = i / half, off = i % half;
            const int64_t lo = blk * k + off, hi = blk * k + k - 1 - off;
            if (hi < m) order_pair(a, lo, hi);
        }
        __syncthreads();
        for (int64_t j = k >> 2; j >= 1; j >>= 1) {
            for (int64_t i = threadIdx.x; i < pow2 / 2; i += blockDim.x) {
                const int64_t blk = i / j, off = i % j;
                const int64_t lo = blk * 2 * j + off, hi = lo + j;
                if (hi < m) order_pair(a, lo, hi);
            }
            __syncthreads();
        }
    }
}

// One warp per overflow list (the common case: a few dozen to a few hundred
// hits): the warp loads the list into its own shared-memory region, runs the
// network with __syncwarp between steps and writes it back. Lists longer than
// kWarpSortMax go to a second list (kept in the then unused slot buffer) for
// sort_big_lists_kernel. Both kernels stride over counts held on the device
// and write nothing when the hits did not fit the caller's buffer.
constexpr int kWarpSortMax = 1024;
constexpr int kSortWarps = kThreads / 32;

__device__ void warp_bitonic_sort(uint32_t *a, int m) {
    const int lane = threadIdx.x & 31;
    int lg = 0;
    while ((1 << lg) < m) ++lg;
    const int pairs = (1 << lg) >> 1;
    for (int lk = 1; lk <= lg; ++lk) {
        // first step of the merge of blocks of 2^lk: i pairs with its mirror
        const int lh = lk - 1;
        for (int i = lane; i < pairs; i += 32) {
            const int blk = i >> lh, off = i & ((1 << lh) - 1);
            const int lo = (blk << lk) + off, hi = (blk << lk) + (1 << lk) - 1 - off;
            if (hi < m) order_pair(a, lo, hi);
        }
        __syncwarp();
        for (int lj = lk - 2; lj >= 0; --lj) {
            for (int i = lane; i < pairs; i += 32) {
                const int blk = i >> lj, off = i & ((1 << lj) - 1);
                const int lo = (blk << (lj + 1)) + off, hi = lo + (1 << lj);
                if (hi < m) order_pair(a, lo, hi);
            }
            __syncwarp();
        }
    }
}

__global__ void __launch_bounds__(kThreads)
    warp_sort_lists_kernel(const int64_t *__restrict__ offsets, uint32_t *hits,
                           const uint32_t *__restrict__ list, uint32_t *__restrict__ big_list, Control *ctl,
                           unsigned long long capacity) {
    __shared__ uint32_t s[kSortWarps][kWarpSortMax];
    if (ctl->total > capacity) return;
    const uint32_t count = ctl->overflow_filled;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t *a = s[warp];
    for (int64_t j = (int64_t)blockIdx.x * kSortWarps + warp; j < count; j += (int64_t)gridDim.x * kSortWarps) {
        const uint32_t q = list[j] & ~kSpilledTag;
        const int64_t base = offsets[q];
        const int64_t m = offsets[q + 1] - base;
        if (m > kWarpSortMax) {
            if (lane == 0) big_list[atomicAdd(&ctl->overflow_big, 1u)] = q;
            continue;
        }
        uint32_t *seg = hits + base;
        for (int i = lane; i < m; i += 32) a[i] = seg[i];
        __syncwarp();
        warp_bitonic_sort(a, (int)m);
        for (int i = lane; i < m; i += 32) seg[i] = a[i];
        __syncwarp();
    }
}

__global__ void __launch_bounds__(kFixThreads)
    sort_big_lists_kernel(const int64_t *__restrict__ offsets, uint32_t *hits,
                          const uint32_t *__restrict__ big_list, const Control *ctl,
                          unsigned long long capacity) {
    __shared__ uint32_t s[kFixSmem];
    if (ctl->total > capacity) return;
    const uint32_t count = ctl->overflow_big;
    for (uint32_t j = blockIdx.x; j < count; j += gridDim.x) {
        const uint32_t q = big_list[j];
        const int64_t base = offsets[q];
        const int64_t m = offsets[q + 1] - base;
        uint32_t *seg = hits + base;
        if (m <= kFixSmem) {
            for (int64_t i = threadIdx.x; i < m; i += blockDim.x) s[i] = seg[i];
            __syncthreads();
            bitonic_sort(s, m);
            for (int64_t i = threadIdx.x; i < m; i += blockDim.x) seg[i] = s[i];
        } else {
            bitonic_sort(seg, m);  // in global memory; one CTA owns the list
        }
        __syncthreads();
    }
}

// Lists whose hits past the slot all went to spill chunks: one warp per list
// copies the slot and then each chunk of its chain to the list's CSR range
// (in walk order; the list sorts follow).
__global__ void __launch_bounds__(kThreads)
    spill_gather_kernel(QueryScratch qs, const int64_t *__restrict__ offsets, uint32_t *__restrict__ hits,
                        const Control *ctl, unsigned long long capacity) {
    if (ctl->total > capacity) return;
    const uint32_t count = ctl->overflow_filled;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int kWarps = kThreads / 32;
    for (int64_t j = (int64_t)blockIdx.x * kWarps + warp; j < count; j += (int64_t)gridDim.x * kWarps) {
        const uint32_t e = qs.overflow_list[j];
        if (!(e & kSpilledTag)) continue;  // walks a second time instead
        const uint32_t q = e & ~kSpilledTag;
        const int64_t base = offsets[q];
        const int64_t m = offsets[q + 1] - base;
        uint32_t *dst = hits + base;
        const uint32_t *slot = qs.slots + (int64_t)q * kSlot;
        for (int k = lane; k < kSlot; k += 32) dst[k] = slot[k];
        int64_t done = kSlot;
        uint32_t c = qs.spill_head[q];
        while (done < m) {
            if (c >= qs.spill_chunks) break;  // cannot happen for a tagged list; guards the reads
            const uint32_t *chunk = qs.spill + (int64_t)c * kSpillChunkWords;
            const int64_t take = min((int64_t)(kSpillChunkWords - 1), m - done);
            for (int k = lane; k < take; k += 32) dst[done + k] = chunk[1 + k];
            done += take;
            c = chunk[0];
        }
    }
}

// ---- batches: the same walk, on the tree of the query's instance

template <int kQ, int kP>
__global__ void __launch_bounds__(kThreads, 8)  // at most 32 registers: full occupancy for the walk
    batch_collect_kernel(const float4 *__restrict__ nodes, BatchTables bt, QueryArgs qa, QueryScratch qs,
                         Control *ctl) {
    const int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (i >= qa.nq) return;
    const int64_t qi = thread_query(qa, i);
    const int b = instance_of(bt.query_off, bt.count, qi);
    const int64_t n = bt.prim_off[b + 1] - bt.prim_off[b];
    const TreeView t{nodes + bt.node_start[b], nullptr, n, kP};
    collect_walk<kQ, kP, false>(t, qa, qs, ctl, i, qi, n > 0 && ctl->build_flags == 0);
}

// Overflow lists whose number is known only on the device: a fixed grid
// strides over them.
template <int kQ, int kP>
__global__ void __launch_bounds__(kThreads)
    batch_overflow_kernel(const float4 *__restrict__ nodes, BatchTables bt, QueryArgs qa,
                          const uint32_t *__restrict__ list, const Control *ctl,
                          const int64_t *__restrict__ offsets, uint32_t *__restrict__ hits,
                          unsigned long long capacity) {
    if (ctl->total > capacity) return;  // nothing is written into a buffer that is too small
    const uint32_t count = ctl->overflow_filled;
    for (int64_t j = (int64_t)blockIdx.x * kThreads + threadIdx.x; j < count; j += (int64_t)gridDim.x * kThreads) {
        const uint32_t e = list[j];
        if (e & kSpilledTag) continue;  // its hits are in its slot and spill chunks
        const int64_t qi = e;
        const int b = instance_of(bt.query_off, bt.count, qi);
        const int64_t n = bt.prim_off[b + 1] - bt.prim_off[b];
        const TreeView t{nodes + bt.node_start[b], nullptr, n, kP};
        const int64_t base = offsets[qi];
        const int64_t total = offsets[qi + 1] - base;
        const auto q = QueryOf<kQ>::load(qa, qi);
        int64_t c = 0;
        walk<kP>(t, q, [&](uint32_t id) {
            if (c < total) hits[base + c] = id;
            ++c;
        });
    }
}

// ---- walk statistics

// Algorithm 1 for every query, counting the leaves and internal nodes it
// visits (no hits are kept): the walk's work per query, for measurement.
template <int kQ, int kP>
__global__ void __launch_bounds__(kThreads)
    visits_kernel(TreeView t, QueryArgs qa, unsigned long long *counts, Control *ctl) {
    const int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    uint32_t leaves = 0, internal = 0;
    if (i < qa.nq && t.n > 0 && ctl->build_flags == 0) {
        const auto q = QueryOf<kQ>::load(qa, thread_query(qa, i));
        const int ni = (int)t.n - 1;
        const int nodes = 2 * (int)t.n - 1;
        const uint32_t max_steps = 2u * (uint32_t)nodes;
        int node = 0;
        while ((uint32_t)node < (uint32_t)nodes && leaves + internal < max_steps) {
            const bool leaf = node >= ni;
            const int unit = kP == LBVH_PRIM_BOXES ? 2 * node : (leaf ? node + ni : 2 * node);
            float4 a, b;
            load_node<kP>(t.inodes, unit, leaf, a, b);
            const bool hit = hits(q, xyz(a), xyz(b));
            const uint32_t word = __float_as_uint(a.w);
            leaves += leaf;
            internal += !leaf;
            node = leaf ? node + 1 - ((word & kLeafSkipInternal) ? ni : 0) : __float_as_int(hit ? a.w : b.w);
        }
    }
    // one add per warp
    for (int off = 16; off > 0; off >>= 1) {
        leaves += __shfl_xor_sync(0xffffffffu, leaves, off);
        internal += __shfl_xor_sync(0xffffffffu, internal, off);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(counts, (unsigned long long)leaves);
        atomicAdd(counts + 1, (unsigned long long)internal);
    }
}

// ---- k nearest neighbours

// Max-heap of (squared distance bits << 32 | primitive index) keys in the
// thread's local memory: keys order like (distance, index), distances being
// non-negative floats.
template <int kCap>
struct KnnHeap {
    uint64_t h[kCap];
    int cnt;

    __device__ __forceinline__ void push(uint64_t key) {
        int i = cnt++;
        while (i > 0) {
            const int p = (i - 1) >> 1;
            if (h[p] >= key) break;
            h[i] = h[p];
            i = p;
        }
        h[i] = key;
    }
    // the largest key leaves and `key` (smaller than it) enters
    __device__ __forceinline__ void sift_from_top(uint64_t key, int size) {
        int i = 0;
        while (true) {
            const int l = 2 * i + 1;
            if (l >= size) break;
            const int r = l + 1;
            const int c = (r < size && h[r] > h[l]) ? r : l;
            if (h[c] <= key) break;
            h[i] = h[c];
            i = c;
        }
        h[i] = key;
    }
    // heap sort: ascending keys in h[0..cnt)
    __device__ __forceinline__ void sort() {
        for (int e = cnt - 1; e > 0; --e) {
            const uint64_t top = h[0];
            sift_from_top(h[e], e);
            h[e] = top;
        }
    }
};

constexpr int kKnnSeedFactor = 4;

__device__ __forceinline__ uint64_t knn_key(float d2, uint32_t id) {
    return ((uint64_t)__float_as_uint(d2) << 32) | id;
}

// The k nearest primitives of each query point: Algorithm 1 with a ball
// whose radius is the current k-th best distance. The radius only shrinks
// during the walk, so a subtree the walk skips (its box farther than the
// radius then) holds no primitive that could enter the list later: the walk
// stays exact. A node is entered when its box distance is <= the radius (a
// primitive at exactly that distance may still win on its index). The list
// starts from the m = min(k, n) leaves around the query's place in the
// sorted Morton codes (a lower-bound search of the query's own code): the
// best m of the 4m leaves there, so the walk starts with a tight radius; the
// seed leaves are not considered again (a seed that left the list cannot
// come back, the radius only shrinking). 4m seeds: 16-nearest-neighbour
// walk of 2^25 uniform points 123 ms with m seeds.
// Queries with a non-finite coordinate get no neighbours. Row qi of out_idx
// / out_d2 holds the neighbours in the order (d2, index), padded with
// 0xffffffff / +inf.
template <int kP, int kCap>
__global__ void __launch_bounds__(128)
    knn_kernel(TreeView t, const uint64_t *__restrict__ codes, const float *__restrict__ bounds, int bits,
               QueryArgs qa, int k, uint32_t *__restrict__ out_idx, float *__restrict__ out_d2, Control *ctl) {
    const int64_t i = (int64_t)blockIdx.x * 128 + threadIdx.x;
    if (i >= qa.nq) return;
    const int64_t qi = thread_query(qa, i);
    const float3 c = make_float3(__ldcs(qa.queries + 3 * qi), __ldcs(qa.queries + 3 * qi + 1),
                                 __ldcs(qa.queries + 3 * qi + 2));
    const int n = (int)t.n;
    const int m = k < n ? k : n;
    KnnHeap<kCap> hp;
    hp.cnt = 0;
    const bool finite = isfinite(c.x) && isfinite(c.y) && isfinite(c.z);
    if (finite && n > 0 && ctl->build_flags == 0) {
        const int ni = n - 1;
        const float4 *base = t.inodes;  // leaves follow the internal records
        // the seed leaves [s0, s0 + S): S = 4m around the query's place in
        // Morton order (the best m of them start the list)
        const int S = min(n, kKnnSeedFactor * m);
        int s0 = 0;
        if (codes && bits > 0 && S < n) {
            const uint64_t qc = morton(c.x, c.y, c.z, make_grid(bounds, bits / 3));
            int lo = 0, hi = n;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (__ldg(codes + mid) < qc) lo = mid + 1;
                else hi = mid;
            }
            s0 = min(max(lo - S / 2, 0), n - S);
        }
        for (int j = s0; j < s0 + S; ++j) {
            const int unit = kP == LBVH_PRIM_BOXES ? 2 * (ni + j) : ni + j + ni;
            float4 a, b;
            load_node<kP>(base, unit, true, a, b);
            const uint64_t key = knn_key(box_d2(c, xyz(a), xyz(b)), __float_as_uint(a.w) & kLeafIndexMask);
            if (hp.cnt < m) hp.push(key);
            else if (key < hp.h[0]) hp.sift_from_top(key, m);
        }
        if (S < n) {
            const int nodes = 2 * n - 1;
            const uint32_t max_steps = 2u * (uint32_t)nodes;
            uint32_t steps = 0;
            int node = 0;
            while ((uint32_t)node < (uint32_t)nodes) {
                if (++steps > max_steps) break;
                const bool leaf = node >= ni;
                const int unit = kP == LBVH_PRIM_BOXES ? 2 * node : (leaf ? node + ni : 2 * node);
                float4 a, b;
                load_node<kP>(base, unit, leaf, a, b);
                const float d2 = box_d2(c, xyz(a), xyz(b));
                const uint64_t worst = hp.h[0];  // the list is full (m entries) from the seeds on
                const bool inside = d2 <= __uint_as_float((uint32_t)(worst >> 32));
                const uint32_t word = __float_as_uint(a.w);
                if (leaf) {
                    const int pos = node - ni;
                    if (inside && (pos < s0 || pos >= s0 + S)) {
                        const uint64_t key = knn_key(d2, word & kLeafIndexMask);
                        if (key < worst) hp.sift_from_top(key, m);
                    }
                    node = node + 1 - ((word & kLeafSkipInternal) ? ni : 0);
                } else {
                    node = __float_as_int(inside ? a.w : b.w);
                }
            }
            if (!(node == kSentinel || node == nodes)) atomicOr(&ctl->query_flags, kFlagCorrupt);
        }
        hp.sort();
    }
    uint32_t *ri = out_idx + qi * k;
    float *rd = out_d2 ? out_d2 + qi * k : nullptr;
    for (int r = 0; r < k; ++r) {
        const bool have = r < hp.cnt;
        const uint64_t key = have ? hp.h[r] : ~0ull;
        __stcs(ri + r, have ? (uint32_t)key : 0xffffffffu);
        if (rd) __stcs(rd + r, have ? __uint_as_float((uint32_t)(key >> 32)) : __int_as_float(0x7f800000));
    }
}

}  // namespace

template <typename F>
void dispatch_kinds(int qkind, int pkind, F &&f) {
    if (qkind == LBVH_Q_RAY) {
        if (pkind == LBVH_PRIM_POINTS)
            f(std::integral_constant<int, LBVH_Q_RAY>{}, std::integral_constant<int, LBVH_PRIM_POINTS>{});
        else
            f(std::integral_constant<int, LBVH_Q_RAY>{}, std::integral_constant<int, LBVH_PRIM_BOXES>{});
    } else if (qkind == LBVH_Q_SPHERE) {
        if (pkind == LBVH_PRIM_POINTS)
            f(std::integral_constant<int, LBVH_Q_SPHERE>{}, std::integral_constant<int, LBVH_PRIM_POINTS>{});
        else
            f(std::integral_constant<int, LBVH_Q_SPHERE>{}, std::integral_constant<int, LBVH_PRIM_BOXES>{});
    } else {
        if (pkind == LBVH_PRIM_POINTS)
            f(std::integral_constant<int, LBVH_Q_BOX>{}, std::integral_constant<int, LBVH_PRIM_POINTS>{});
        else
            f(std::integral_constant<int, LBVH_Q_BOX>{}, std::integral_constant<int, LBVH_PRIM_BOXES>{});
    }
}

void launch_query_collect(const TreeView &t, const QueryArgs &q, const QueryScratch &qs, Control *ctl,
                          cudaStream_t s) {
    if (q.nq <= 0) return;
    const unsigned blocks = (unsigned)((q.nq + kThreads - 1) / kThreads);
    dispatch_kinds(q.qkind, t.kind, [&](auto qk, auto pk) {
        constexpr int Q = decltype(qk)::value, P = decltype(pk)::value;
        switch (q.walk) {
        case kWalkGroup8: collect_group_kernel<Q, P, 8><<<blocks, kThreads, 0, s>>>(t, q, qs, ctl); break;
        case kWalkGroup16: collect_group_kernel<Q, P, 16><<<blocks, kThreads, 0, s>>>(t, q, qs, ctl); break;
        case kWalkGroup32: collect_group_kernel<Q, P, 32><<<blocks, kThreads, 0, s>>>(t, q, qs, ctl); break;
        case kWalkThread512:
            collect_kernel<Q, P, 512><<<(unsigned)((q.nq + 511) / 512), 512, 0, s>>>(t, q, qs, ctl);
            break;
        default: collect_kernel<Q, P, kThreads><<<blocks, kThreads, 0, s>>>(t, q, qs, ctl); break;
        }
    });
    count_launches(1);
}

void launch_query_copy_checked(const QueryArgs &q, const QueryScratch &qs, const int64_t *offsets,
                               uint32_t *hits, unsigned long long capacity, Control *ctl, cudaStream_t s) {
    if (q.nq <= 0) return;
    const unsigned blocks = (unsigned)((q.nq + kThreads - 1) / kThreads);
    copy_kernel<<<blocks, kThreads, 0, s>>>(q.nq, qs.counts, offsets, qs.slots, hits, capacity, ctl);
    count_launches(1);
}

void launch_query_copy(const QueryArgs &q, const QueryScratch &qs, const int64_t *offsets,
                       uint32_t *hits, Control *ctl, cudaStream_t s) {
    launch_query_copy_checked(q, qs, offsets, hits, ~0ull, ctl, s);
}

// Sorts the overflow lists: warps for the lists, CTAs for the long ones.
// `bound`: an upper bound of the overflow count (sizes the warp kernel's grid).
// First copies the spilled lists (slot + chunks) to their CSR ranges; the
// big-list sort then reuses the slot buffer, which nothing reads any more.
static void launch_sort_lists(const QueryScratch &qs, uint64_t bound, const int64_t *offsets, uint32_t *hits,
                              unsigned long long capacity, Control *ctl, cudaStream_t s) {
    const uint64_t want = (bound + kSortWarps - 1) / kSortWarps;
    const uint64_t cap = (uint64_t)device_sm_count() * 8;
    const unsigned blocks = (unsigned)std::max<uint64_t>(1, std::min(want, cap));
    spill_gather_kernel<<<blocks, kThreads, 0, s>>>(qs, offsets, hits, ctl, capacity);
    warp_sort_lists_kernel<<<blocks, kThreads, 0, s>>>(offsets, hits, qs.overflow_list, qs.slots, ctl, capacity);
    sort_big_lists_kernel<<<(unsigned)device_sm_count(), kFixThreads, 0, s>>>(offsets, hits, qs.slots, ctl,
                                                                              capacity);
    count_launches(3);
}

void launch_query_overflow(const TreeView &t, const QueryArgs &q, const QueryScratch &qs,
                           uint32_t count, const int64_t *offsets, uint32_t *hits, Control *ctl,
                           cudaStream_t s) {
    if (count == 0) return;
    const unsigned blocks = (unsigned)((count + kThreads - 1) / kThreads);
    dispatch_kinds(q.qkind, t.kind, [&](auto qk, auto pk) {
        overflow_walk_kernel<decltype(qk)::value, decltype(pk)::value><<<blocks, kThreads, 0, s>>>(
            t, q, qs.overflow_list, count, offsets, hits);
    });
    launch_sort_lists(qs, count, offsets, hits, ~0ull, ctl, s);
    count_launches(1);
}

void launch_batch_collect(const float4 *nodes, int kind, const BatchTables &bt, const QueryArgs &q,
                          const QueryScratch &qs, Control *ctl, cudaStream_t s) {
    if (q.nq <= 0) return;
    const unsigned blocks = (unsigned)((q.nq + kThreads - 1) / kThreads);
    dispatch_kinds(q.qkind, kind, [&](auto qk, auto pk) {
        batch_collect_kernel<decltype(qk)::value, decltype(pk)::value><<<blocks, kThreads, 0, s>>>(nodes, bt, q, qs,
                                                                                                    ctl);
    });
    count_launches(1);
}

void launch_batch_overflow(const float4 *nodes, int kind, const BatchTables &bt, const QueryArgs &q,
                           const QueryScratch &qs, Control *ctl, const int64_t *offsets, uint32_t *hits,
                           unsigned long long capacity, cudaStream_t s) {
    if (q.nq <= 0) return;
    const unsigned blocks = (unsigned)device_sm_count() * 8;
    dispatch_kinds(q.qkind, kind, [&](auto qk, auto pk) {
        batch_overflow_kernel<decltype(qk)::value, decltype(pk)::value><<<blocks, kThreads, 0, s>>>(
            nodes, bt, q, qs.overflow_list, ctl, offsets, hits, capacity);
    });
    count_launches(1);
    launch_sort_lists(qs, (uint64_t)q.nq, offsets, hits, capacity, ctl, s);
}

void launch_visits(const TreeView &t, const QueryArgs &q, unsigned long long *counts, Control *ctl, cudaStream_t s) {
    if (q.nq <= 0) return;
    const unsigned blocks = (unsigned)((q.nq + kThreads - 1) / kThreads);
    dispatch_kinds(q.qkind, t.kind, [&](auto qk, auto pk) {
        visits_kernel<decltype(qk)::value, decltype(pk)::value><<<blocks, kThreads, 0, s>>>(t, q, counts, ctl);
    });
    count_launches(1);
}

void launch_knn(const TreeView &t, const uint64_t *codes, const float *bounds, int bits, const QueryArgs &q, int k,
                uint32_t *out_idx, float *out_d2, Control *ctl, cudaStream_t s) {
    if (q.nq <= 0) return;
    const unsigned blocks = (unsigned)((q.nq + 127) / 128);
    auto go = [&](auto cap) {
        constexpr int C = decltype(cap)::value;
        if (t.kind == LBVH_PRIM_POINTS)
            knn_kernel<LBVH_PRIM_POINTS, C><<<blocks, 128, 0, s>>>(t, codes, bounds, bits, q, k, out_idx, out_d2, ctl);
        else
            knn_kernel<LBVH_PRIM_BOXES, C><<<blocks, 128, 0, s>>>(t, codes, bounds, bits, q, k, out_idx, out_d2, ctl);
    };
    if (k <= 16) go(std::integral_constant<int, 16>{});
    else if (k <= 64) go(std::integral_constant<int, 64>{});
    else go(std::integral_constant<int, kKnnMaxK>{});
    count_launches(1);
}

int64_t scan_tile_count(int64_t nq) { return (nq + kScanTile - 1) / kScanTile; }

namespace {
__global__ void __launch_bounds__(kThreads) offsets_add_kernel(int64_t *off, int64_t n, int64_t base) {
    const int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (i < n) off[i] += base;
}
}  // namespace

void launch_offsets_add(int64_t *offsets, int64_t n, int64_t base, cudaStream_t s) {
    if (n <= 0) return;
    offsets_add_kernel<<<(unsigned)((n + kThreads - 1) / kThreads), kThreads, 0, s>>>(offsets, n, base);
    count_launches(1);
}

void launch_exclusive_scan(const uint32_t *counts, int64_t nq, int64_t *offsets,
                           int64_t *tile_sums, Control *ctl, cudaStream_t s) {
    const int64_t tiles = scan_tile_count(nq);
    if (tiles > 0)
        scan_reduce_kernel<<<(unsigned)tiles, kScanThreads, 0, s>>>(counts, nq, tile_sums);
    scan_tiles_kernel<<<1, kScanThreads, 0, s>>>(tile_sums, tiles, offsets, nq, &ctl->total);
    if (tiles > 0)
        scan_apply_kernel<<<(unsigned)tiles, kScanThreads, 0, s>>>(counts, nq, tile_sums, offsets);
    count_launches(tiles > 0 ? 3 : 1);
}

}  // namespace lbvh
