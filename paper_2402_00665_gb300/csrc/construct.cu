// construct.cu -- the single bottom-up pass of Algorithm 4 (Sec. 4): modified
// Apetrei merge that writes every internal node in Karras' ordering (Sec. 3.1)
// with its left child, its skip connection (Algorithm 2) and its box (Karras
// step 4, which Algorithm 4 leaves out; here the second thread up writes the
// union of its own box, held in registers, and its sibling's).
//
// One thread per leaf i:
//   1. delta*(i-1), delta*(i), delta*(i+1) from the sorted codes. delta is the
//      XOR reading of Sec. 3.2 with keys augmented by their sorted position:
//      64 + highest differing code bit, else the highest differing bit of the
//      positions; +inf (255) at -1 and n-1. Only comparisons are made and no
//      two compared gaps can share a highest bit, so this order is exact.
//   2. The leaf's skip (Algorithm 4's leaf lines) and box are written.
//   3. Climb: the parent's split p is range_right (left child: delta_right <
//      delta_left) or range_left - 1 (right child). The thread swaps its half
//      of the parent's description into store[p]. The first arrival reads
//      "empty" and exits; the second receives the other half, so it now knows
//      the parent's full range [l, r] and delta*(l-1), delta*(r), delta*(r+1).
//      It computes the Karras index q = r if delta*(r) < delta*(l-1) else l,
//      the left child (L_p if l == p else I_p: the children of split p are p
//      and p+1), the skip (sentinel if r == n-1, else L_{r+1} if delta*(r) <
//      delta*(r+1), else I_{r+1}), and the box, writes node q, and continues
//      with i = q until q == 0 (I_0 is the root in Karras' ordering).
//
// Differences from the listing, with the same result:
//   - store[p] carries, besides the range end, the delta* values the other
//     thread needs (packed into 64 bits), so no thread re-reads codes while
//     it climbs; only the leaf step reads codes, coalesced.
//   - an atomic exchange replaces compare-and-swap: exactly two threads
//     ever touch store[p], so the one that reads "empty" is the first. The
//     second writes "empty" back, leaving the scratch clean for the next build
//     (it is zeroed once, when allocated).
//   - release/acquire: the exchange is an acq_rel atomic, so a thread's node
//     is visible before its half of the parent is, and the second thread
//     reads the sibling's box only after it has seen that half.
//   - two phases (construct_block_kernel): splits whose two children both
//     lie inside one group of consecutive leaves (128 by default) meet in
//     shared memory (block-scope exchange, sibling box from shared memory);
//     only the nodes spanning a group's edge meet in the device-scope
//     `store` words (sibling box through L2, ld.global.cg). Batches group
//     their global sorted positions the same way (a group may hold several
//     trees; a split only ever joins leaves of one).
#include <cuda/atomic>

#include <cstdlib>
#include <mutex>

#include "lbvh_internal.cuh"

namespace lbvh {

namespace {

constexpr int kThreads = 256;
constexpr uint32_t kInf = 255;  // above every finite delta* (<= 127)

__device__ __forceinline__ uint32_t delta_star(uint64_t a, uint64_t b, uint32_t pos) {
    const uint64_t x = a ^ b;
    if (x) return 127u - (uint32_t)__clzll((long long)x);  // 64 + highest differing bit
    return 31u - (uint32_t)__clz((int)(pos ^ (pos + 1u)));
}

// store word: bit 63 set = occupied.
//   left child's half (its range start l and delta*(l-1)):   l | d << 32
//   right child's half (range end r, delta*(r), delta*(r+1)): r | d << 32 | dn << 40
__device__ __forceinline__ unsigned long long pack(uint32_t end, uint32_t d, uint32_t dn) {
    return (1ull << 63) | ((unsigned long long)dn << 40) | ((unsigned long long)d << 32) | end;
}

template <int kKind>
__device__ __forceinline__ void load_node_box(const float4 *inodes, const float4 *leaves, int ni,
                                              int id, float3 &lo, float3 &hi) {
    if (id < ni) {
        const float4 a = __ldcg(inodes + 2 * (int64_t)id);
        const float4 b = __ldcg(inodes + 2 * (int64_t)id + 1);
        lo = make_float3(a.x, a.y, a.z);
        hi = make_float3(b.x, b.y, b.z);
    } else if (kKind == LBVH_PRIM_POINTS) {
        const float4 a = __ldcg(leaves + (id - ni));
        lo = make_float3(a.x, a.y, a.z);
        hi = lo;
    } else {
        const float4 a = __ldcg(leaves + 2 * (int64_t)(id - ni));
        const float4 b = __ldcg(leaves + 2 * (int64_t)(id - ni) + 1);
        lo = make_float3(a.x, a.y, a.z);
        hi = make_float3(b.x, b.y, b.z);
    }
}

// The exchange on store[p] publishes this thread's finished node (release)
// and, for the second thread, makes the sibling's node visible (acquire):
// either as one acq_rel atomic, or as a relaxed atomic between two fences.
template <bool kAcqRel>
__device__ __forceinline__ unsigned long long publish_exchange(unsigned long long *slot,
                                                               unsigned long long v) {
    if (kAcqRel) {
        cuda::atomic_ref<unsigned long long, cuda::thread_scope_device> a(*slot);
        return a.exchange(v, cuda::memory_order_acq_rel);
    }
    __threadfence();
    const unsigned long long old = atomicExch(slot, v);
    __threadfence();
    return old;
}

// A thread's finished node while it climbs: leaf range [l, r], delta*(l-1),
// delta*(r), delta*(r+1), and its box.
struct Climb {
    uint32_t l, r, d_left, d_right, d_next;
    float3 lo, hi;
};

// delta*(i-1), delta*(i), delta*(i+1) around leaf i (255 = +inf at -1 and n-1).
__device__ __forceinline__ void leaf_deltas(int i, int n, const uint64_t *__restrict__ codes, uint32_t &dl,
                                            uint32_t &dr, uint32_t &drn) {
    const uint64_t c0 = codes[i];
    dl = i > 0 ? delta_star(codes[i - 1], c0, (uint32_t)(i - 1)) : kInf;
    dr = kInf;
    drn = kInf;
    if (i + 1 < n) {
        const uint64_t c1 = codes[i + 1];
        dr = delta_star(c0, c1, (uint32_t)i);
        if (i + 2 < n) drn = delta_star(c1, codes[i + 2], (uint32_t)(i + 1));
    }
}

// Algorithm 4's leaf step for leaf i of one tree of n leaves, given its
// delta* values: the leaf's skip and box (written out) and the climb state.
// perm holds primitive indices into `prims`, the tree's own indices being
// perm - perm_base. False (and kFlagCorrupt) if perm is not a permutation of
// this tree.
template <int kKind>
__device__ __forceinline__ bool leaf_write(int i, int n, const uint32_t *__restrict__ perm, uint32_t perm_base,
                                           const float *__restrict__ prims, float4 *leaves, uint32_t *flags,
                                           uint32_t dl, uint32_t dr, uint32_t drn, Climb &c) {
    const int ni = n - 1;
    const int leaf_skip = i == n - 1 ? kSentinel : (dr < drn ? ni + i + 1 : i + 1);
    const uint32_t p_id = perm[i];
    const uint32_t p_own = p_id - perm_base;
    if (p_own >= (uint32_t)n) {  // not a permutation of this tree: the sort failed
        atomicOr(flags, kFlagCorrupt);
        return false;
    }
    float3 lo, hi;
    if (kKind == LBVH_PRIM_POINTS) {
        lo = make_float3(prims[3 * (int64_t)p_id], prims[3 * (int64_t)p_id + 1],
                         prims[3 * (int64_t)p_id + 2]);
        hi = lo;
    } else {
        const float *b = prims + 6 * (int64_t)p_id;
        lo = make_float3(b[0], b[1], b[2]);
        hi = make_float3(b[3], b[4], b[5]);
    }
    // the leaf's skip is position i+1: one bit says I_{i+1} rather than L_{i+1}
    const uint32_t word = p_own | (leaf_skip >= 0 && leaf_skip < ni ? kLeafSkipInternal : 0u);
    if (kKind == LBVH_PRIM_POINTS) {
        leaves[i] = make_float4(lo.x, lo.y, lo.z, __uint_as_float(word));
    } else {
        leaves[2 * (int64_t)i] = make_float4(lo.x, lo.y, lo.z, __uint_as_float(word));
        leaves[2 * (int64_t)i + 1] = make_float4(hi.x, hi.y, hi.z, 0.0f);
    }
    c = Climb{(uint32_t)i, (uint32_t)i, dl, dr, drn, lo, hi};
    return true;
}

template <int kKind>
__device__ __forceinline__ bool leaf_step(int i, int n, const uint64_t *__restrict__ codes,
                                          const uint32_t *__restrict__ perm, uint32_t perm_base,
                                          const float *__restrict__ prims, float4 *leaves, uint32_t *flags,
                                          Climb &c) {
    uint32_t dl, dr, drn;
    leaf_deltas(i, n, codes, dl, dr, drn);
    return leaf_write<kKind>(i, n, perm, perm_base, prims, leaves, flags, dl, dr, drn, c);
}

// The parent's split p of c's node (range_right for a left child, range_left
// - 1 for a right child) and the half of the parent's description c gives.
__device__ __forceinline__ bool parent_split(const Climb &c, uint32_t &p, unsigned long long &mine) {
    const bool is_left = c.d_right < c.d_left;
    p = is_left ? c.r : c.l - 1;
    mine = is_left ? pack(c.l, c.d_left, 0) : pack(c.r, c.d_right, c.d_next);
    return is_left;
}

// The second thread up at split p takes the sibling's half: c becomes the
// parent's range; returns the sibling's node id (leaves from ni up).
__device__ __forceinline__ int take_half(Climb &c, bool is_left, uint32_t p, unsigned long long other,
                                         int ni) {
    if (is_left) {
        c.r = (uint32_t)other;
        c.d_right = (uint32_t)(other >> 32) & 0xffu;
        c.d_next = (uint32_t)(other >> 40) & 0xffu;
        return (p + 1 == c.r) ? ni + (int)p + 1 : (int)p + 1;
    }
    c.l = (uint32_t)other;
    c.d_left = (uint32_t)(other >> 32) & 0xffu;
    return (c.l == p) ? ni + (int)p : (int)p;
}

// The parent of split p: box = union with the sibling's, Karras index q = r
// if delta*(r) < delta*(l-1) else l, left child (L_p if l == p else I_p),
// skip (sentinel if r == n-1, else L_{r+1} if delta*(r) < delta*(r+1), else
// I_{r+1}). Writes node q and returns q.
__device__ __forceinline__ int write_parent(Climb &c, uint32_t p, int n, float3 slo, float3 shi,
                                            float4 *inodes) {
    const int ni = n - 1;
    c.lo = make_float3(min_ordered(c.lo.x, slo.x), min_ordered(c.lo.y, slo.y), min_ordered(c.lo.z, slo.z));
    c.hi = make_float3(max_ordered(c.hi.x, shi.x), max_ordered(c.hi.y, shi.y), max_ordered(c.hi.z, shi.z));
    const int q = c.d_right < c.d_left ? (int)c.r : (int)c.l;
    const int left_child = (c.l == p) ? ni + (int)p : (int)p;
    const int skip = (c.r == (uint32_t)(n - 1)) ? kSentinel
                                                : (c.d_right < c.d_next ? ni + (int)c.r + 1 : (int)c.r + 1);
    inodes[2 * (int64_t)q] = make_float4(c.lo.x, c.lo.y, c.lo.z, __int_as_float(left_child));
    inodes[2 * (int64_t)q + 1] = make_float4(c.hi.x, c.hi.y, c.hi.z, __int_as_float(skip));
    return q;
}

// Climb from c's node with device-scope exchanges on store[p] until this
// thread is the first up at a split, or has written the root I_0.
template <int kKind, bool kAcqRel>
__device__ __forceinline__ void climb_global(Climb c, int n, float4 *inodes, const float4 *leaves,
                                             unsigned long long *store, uint32_t *flags) {
    const int ni = n - 1;
    // The augmented keys have at most 64 + 32 bits, so no leaf is deeper than
    // 96 levels; the bound only guards against a corrupt input order.
    for (int level = 0; level < 128; ++level) {
        uint32_t p;
        unsigned long long mine;
        const bool is_left = parent_split(c, p, mine);
        if (p >= (uint32_t)ni) {
            atomicOr(flags, kFlagCorrupt);
            return;
        }
        const unsigned long long other = publish_exchange<kAcqRel>(store + p, mine);
        if (other == 0ull) return;  // first thread up
        store[p] = 0ull;            // second thread up: leave the slot empty again
        if ((uint32_t)other >= (uint32_t)n) {
            atomicOr(flags, kFlagCorrupt);
            return;
        }
        const int sibling = take_half(c, is_left, p, other, ni);
        float3 slo, shi;
        load_node_box<kKind>(inodes, leaves, ni, sibling, slo, shi);
        if (write_parent(c, p, n, slo, shi, inodes) == 0) return;  // the root
    }
    atomicOr(flags, kFlagCorrupt);
}

// Algorithm 4 for leaf i, every exchange at device scope (batched trees).
template <int kKind, bool kAcqRel>
__device__ __forceinline__ void construct_leaf(int i, int n, const uint64_t *__restrict__ codes,
                                               const uint32_t *__restrict__ perm, uint32_t perm_base,
                                               const float *__restrict__ prims, float4 *inodes,
                                               float4 *leaves, unsigned long long *store,
                                               uint32_t *flags) {
    Climb c;
    if (!leaf_step<kKind>(i, n, codes, perm, perm_base, prims, leaves, flags, c)) return;
    if (n == 1) return;
    climb_global<kKind, kAcqRel>(c, n, inodes, leaves, store, flags);
}

// Algorithm 4 with the climb split in two phases. The leaves are cut into
// groups of kGroup consecutive leaves [a, a + kGroup) (a warp, or a whole
// CTA). A node whose leaf range lies inside a group has both children there,
// so its split p has a <= p and p + 1 < a + kGroup; such splits meet in a
// shared-memory word with a block-scope exchange, and the sibling's box is
// read from shared memory. A thread stops phase 1 at a split on the group's
// edge, or as the first up at a word. After the group's barrier every node
// inside the group is finished; a word still holding its first thread's half
// has a sibling that spans the group's edge, and that thread, like one stopped
// at the edge, continues with the device-scope exchanges of climb_global.
// Each node is still written once, by the second thread up at its split, with
// the same fields: only where the two halves meet changes.
template <int kGroup>
struct GroupShape {
    static constexpr int kCta = kGroup == 32 ? 256 : kGroup;  // warp groups: eight per CTA
};

template <int kCta>
struct GroupSmem {
    unsigned long long word[kCta];  // split at global position a + j: word[g0 + j]
    float3 lo[2][kCta], hi[2][kCta];  // boxes: [0] leaf, [1] internal node, by global position / index
    int failed;
};

// Both phases for the thread of leaf i of a tree of n leaves whose leaf 0 sits
// at global position o (0 for a single tree; trees of a batch follow each
// other), in the group whose first global position is a (shared slots from
// g0). A split joins two leaves of one tree, so groups may hold several trees.
template <int kKind, int kGroup, int kCta>
__device__ __forceinline__ void two_phase(GroupSmem<kCta> &sm, bool active, int i, int n, int64_t o, int64_t a,
                                          int g0, int t, const uint64_t *__restrict__ codes,
                                          const uint32_t *__restrict__ perm, uint32_t perm_base,
                                          const float *__restrict__ prims, float4 *inodes, float4 *leaves,
                                          unsigned long long *store, uint32_t *flags) {
    const int ni = n - 1;
    Climb c;
    bool pending = false, in_word = false;
    int word_at = 0;
    if (active && leaf_step<kKind>(i, n, codes, perm, perm_base, prims, leaves, flags, c) && n > 1) {
        sm.lo[0][t] = c.lo;
        sm.hi[0][t] = c.hi;
        for (int level = 0; level < 128; ++level) {
            uint32_t p;
            unsigned long long mine;
            const bool is_left = parent_split(c, p, mine);
            if (p >= (uint32_t)ni) {
                atomicOr(flags, kFlagCorrupt);
                break;
            }
            const int64_t rel = o + (int64_t)p - a;  // the split's place in the group
            if (rel < 0 || rel >= kGroup - 1) {       // on the group's edge
                pending = true;
                break;
            }
            const int at = (int)rel;
            cuda::atomic_ref<unsigned long long, cuda::thread_scope_block> w(sm.word[g0 + at]);
            const unsigned long long other = w.exchange(mine, cuda::memory_order_acq_rel);
            if (other == 0ull) {  // first up: the sibling may come in this phase, or never
                pending = in_word = true;
                word_at = at;
                break;
            }
            w.store(0ull, cuda::memory_order_relaxed);  // taken
            if ((uint32_t)other >= (uint32_t)n) {
                atomicOr(flags, kFlagCorrupt);
                break;
            }
            const int sibling = take_half(c, is_left, p, other, ni);
            const int k = sibling < ni ? 1 : 0;
            const int sat = g0 + (int)(o + (sibling < ni ? sibling : sibling - ni) - a);  // g0 + at or + at + 1
            const int q = write_parent(c, p, n, sm.lo[k][sat], sm.hi[k][sat], inodes);
            if (q == 0) break;  // the root: the whole tree lies in this group
            const int qat = g0 + (int)(o + q - a);  // q is l or r, inside the group
            sm.lo[1][qat] = c.lo;
            sm.hi[1][qat] = c.hi;
        }
    }
    if (kGroup == 32)
        __syncwarp();
    else
        __syncthreads();
    if (!pending) return;
    if (in_word && sm.word[g0 + word_at] == 0ull) return;  // the sibling came and carried on
    // this thread wrote its own node, so its device-scope release covers it
    climb_global<kKind, true>(c, n, inodes, leaves, store, flags);
}

template <int kKind, int kGroup>
__global__ void __launch_bounds__(GroupShape<kGroup>::kCta, 2048 / GroupShape<kGroup>::kCta)
    construct_block_kernel(const uint64_t *__restrict__ codes, const uint32_t *__restrict__ perm,
                           const float *__restrict__ prims, int n, float4 *inodes, float4 *leaves,
                           unsigned long long *store, uint32_t *flags) {
    constexpr int kCta = GroupShape<kGroup>::kCta;
    __shared__ GroupSmem<kCta> sm;
    const int t = threadIdx.x;
    const int g0 = t / kGroup * kGroup;  // the group's first thread
    const int i = blockIdx.x * kCta + t;
    sm.word[t] = 0ull;
    if (t == 0) sm.failed = (__ldcg(flags) & (kFlagTimeout | kFlagCorrupt)) != 0;
    __syncthreads();
    if (sm.failed) return;  // the sort failed: leave store untouched (the whole CTA returns)
    two_phase<kKind, kGroup, kCta>(sm, i < n, i, n, 0, (int64_t)blockIdx.x * kCta + g0, g0, t, codes, perm, 0u,
                                   prims, inodes, leaves, store, flags);
}

// Many trees at once, grouped by global sorted position: global position g
// belongs to the instance b with off[b] <= g < off[b+1]; its tree's records
// start at node_start[b] (float4 units) and its store words at store_start[b].
template <int kKind, int kGroup>
__global__ void __launch_bounds__(GroupShape<kGroup>::kCta, 2048 / GroupShape<kGroup>::kCta)
    batch_construct_block_kernel(const uint64_t *__restrict__ codes, const uint32_t *__restrict__ perm,
                                 const float *__restrict__ prims, const int64_t *__restrict__ off,
                                 const int64_t *__restrict__ node_start, const int64_t *__restrict__ store_start,
                                 int count, int64_t total, float4 *nodes, unsigned long long *store,
                                 uint32_t *flags) {
    constexpr int kCta = GroupShape<kGroup>::kCta;
    __shared__ GroupSmem<kCta> sm;
    const int t = threadIdx.x;
    const int g0 = t / kGroup * kGroup;
    const int64_t g = (int64_t)blockIdx.x * kCta + t;
    sm.word[t] = 0ull;
    if (t == 0) sm.failed = (__ldcg(flags) & (kFlagTimeout | kFlagCorrupt)) != 0;
    __syncthreads();
    if (sm.failed) return;
    const bool active = g < total;
    const int b = active ? instance_of(off, count, g) : 0;
    const int64_t o = active ? off[b] : 0;
    const int n = active ? (int)(off[b + 1] - o) : 1;
    float4 *inodes = nodes + (active ? node_start[b] : 0);
    float4 *leaves = inodes + 2 * (int64_t)(n - 1);
    two_phase<kKind, kGroup, kCta>(sm, active, (int)(g - o), n, o, (int64_t)blockIdx.x * kCta + g0, g0, t,
                                   codes + o, perm + o, (uint32_t)o, prims, inodes, leaves,
                                   store + (active ? store_start[b] : 0), flags);
}

template <int kKind, bool kAcqRel>
__global__ void __launch_bounds__(kThreads)
    construct_kernel(const uint64_t *__restrict__ codes, const uint32_t *__restrict__ perm,
                     const float *__restrict__ prims, int n, float4 *inodes, float4 *leaves,
                     unsigned long long *store, uint32_t *flags) {
    const int i = blockIdx.x * kThreads + threadIdx.x;
    if (i >= n) return;
    if (__ldcg(flags) & (kFlagTimeout | kFlagCorrupt)) return;  // the sort failed: leave store untouched
    construct_leaf<kKind, kAcqRel>(i, n, codes, perm, 0u, prims, inodes, leaves, store, flags);
}

// Many trees at once: global sorted position g belongs to the instance b with
// off[b] <= g < off[b+1]; its tree's records start at node_start[b] (float4
// units) and its store words at store_start[b].
template <int kKind>
__global__ void __launch_bounds__(kThreads)
    batch_construct_kernel(const uint64_t *__restrict__ codes, const uint32_t *__restrict__ perm,
                           const float *__restrict__ prims, const int64_t *__restrict__ off,
                           const int64_t *__restrict__ node_start, const int64_t *__restrict__ store_start,
                           int count, int64_t total, float4 *nodes, unsigned long long *store,
                           uint32_t *flags) {
    const int64_t g = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (g >= total) return;
    if (__ldcg(flags) & (kFlagTimeout | kFlagCorrupt)) return;  // the sort failed: leave store untouched
    const int b = instance_of(off, count, g);
    const int64_t o = off[b];
    const int n = (int)(off[b + 1] - o);
    float4 *inodes = nodes + node_start[b];
    float4 *leaves = inodes + 2 * (int64_t)(n - 1);
    construct_leaf<kKind, true>((int)(g - o), n, codes + o, perm + o, (uint32_t)o, prims, inodes, leaves,
                                store + store_start[b], flags);
}

}  // namespace

void launch_batch_construct(const uint64_t *sorted_codes, const uint32_t *perm, const float *prims,
                            const BatchTables &bt, int kind, float4 *nodes, unsigned long long *store,
                            uint32_t *flags, cudaStream_t s) {
    if (bt.total_prims <= 0) return;
    // LBVH_CONSTRUCT_GLOBAL=1: every exchange at device scope (tuning)
    static const bool one_phase = getenv("LBVH_CONSTRUCT_GLOBAL") && atoi(getenv("LBVH_CONSTRUCT_GLOBAL"));
    const bool pts = kind == LBVH_PRIM_POINTS;
    if (one_phase) {
        const unsigned blocks = (unsigned)((bt.total_prims + kThreads - 1) / kThreads);
        auto k = pts ? batch_construct_kernel<LBVH_PRIM_POINTS> : batch_construct_kernel<LBVH_PRIM_BOXES>;
        k<<<blocks, kThreads, 0, s>>>(sorted_codes, perm, prims, bt.prim_off, bt.node_start, bt.store_start, bt.count,
                                      bt.total_prims, nodes, store, flags);
    } else {
        constexpr int kGroup = 128, kCta = GroupShape<kGroup>::kCta;
        const unsigned blocks = (unsigned)((bt.total_prims + kCta - 1) / kCta);
        auto k = pts ? batch_construct_block_kernel<LBVH_PRIM_POINTS, kGroup>
                     : batch_construct_block_kernel<LBVH_PRIM_BOXES, kGroup>;
        k<<<blocks, kCta, 0, s>>>(sorted_codes, perm, prims, bt.prim_off, bt.node_start, bt.store_start, bt.count,
                                  bt.total_prims, nodes, store, flags);
    }
    count_launches(1);
}

namespace {

template <int kGroup>
void launch_construct_block(const uint64_t *sorted_codes, const uint32_t *perm, const float *prims, int64_t n,
                            int kind, float4 *inodes, float4 *leaves, unsigned long long *store, uint32_t *flags,
                            cudaStream_t s) {
    constexpr int kCta = GroupShape<kGroup>::kCta;
    const unsigned blocks = (unsigned)((n + kCta - 1) / kCta);
    auto k = kind == LBVH_PRIM_POINTS ? construct_block_kernel<LBVH_PRIM_POINTS, kGroup>
                                      : construct_block_kernel<LBVH_PRIM_BOXES, kGroup>;
    k<<<blocks, kCta, 0, s>>>(sorted_codes, perm, prims, (int)n, inodes, leaves, store, flags);
}

}  // namespace

void launch_construct(const uint64_t *sorted_codes, const uint32_t *perm, const float *prims,
                      int64_t n, int kind, float4 *inodes, float4 *leaves,
                      unsigned long long *store, uint32_t *flags, cudaStream_t s) {
    if (n <= 0) return;
    // tuning: LBVH_CONSTRUCT_GROUP = leaves per phase-1 group of
    // construct_block_kernel (32, 64, 128 or 256); LBVH_CONSTRUCT_GLOBAL=1 runs
    // every exchange at device scope (construct_kernel), LBVH_CONSTRUCT_FENCES=1
    // that with the fence form
    static const int group = [] {
        const char *e = getenv("LBVH_CONSTRUCT_GROUP");
        const int g = e ? atoi(e) : 128;
        return (g == 32 || g == 64 || g == 256) ? g : 128;
    }();
    static const bool one_phase = getenv("LBVH_CONSTRUCT_GLOBAL") && atoi(getenv("LBVH_CONSTRUCT_GLOBAL"));
    static const bool fences = getenv("LBVH_CONSTRUCT_FENCES") && atoi(getenv("LBVH_CONSTRUCT_FENCES"));
    const bool pts = kind == LBVH_PRIM_POINTS;
    if (one_phase || fences) {
        const unsigned blocks = (unsigned)((n + kThreads - 1) / kThreads);
        auto k = fences ? (pts ? construct_kernel<LBVH_PRIM_POINTS, false> : construct_kernel<LBVH_PRIM_BOXES, false>)
                        : (pts ? construct_kernel<LBVH_PRIM_POINTS, true> : construct_kernel<LBVH_PRIM_BOXES, true>);
        k<<<blocks, kThreads, 0, s>>>(sorted_codes, perm, prims, (int)n, inodes, leaves, store, flags);
    } else if (group == 32) {
        launch_construct_block<32>(sorted_codes, perm, prims, n, kind, inodes, leaves, store, flags, s);
    } else if (group == 64) {
        launch_construct_block<64>(sorted_codes, perm, prims, n, kind, inodes, leaves, store, flags, s);
    } else if (group == 256) {
        launch_construct_block<256>(sorted_codes, perm, prims, n, kind, inodes, leaves, store, flags, s);
    } else {
        launch_construct_block<128>(sorted_codes, perm, prims, n, kind, inodes, leaves, store, flags, s);
    }
    count_launches(1);
}

}  // namespace lbvh

// ---------------------------------------------------------------- no-allocation variant
//
// lbvh_construct_static runs the same construct kernel as the tree builds,
// with Algorithm 4's `store` words in a file-scope device array instead of
// memory the library allocates. The array is as large as the biggest tree the
// entry point accepts, and every GPU that loads this library holds it until
// the process exits.
namespace {

constexpr int64_t kStaticMaxPrims = (int64_t(1) << 20) + 1;  // store words: n - 1 <= 2^20 (8 MiB)

__device__ __align__(256) unsigned long long g_static_store[kStaticMaxPrims - 1];
__device__ __align__(256) uint32_t g_static_flags[64];

// Device addresses of the two arrays, looked up once per device (with that
// device current) and kept; host code must not use the symbols themselves.
struct StaticScratch {
    unsigned long long *store = nullptr;
    uint32_t *flags = nullptr;
};
std::mutex g_static_mu;
constexpr int kMaxDevices = 64;
StaticScratch g_static[kMaxDevices];

lbvh_status static_scratch(StaticScratch *out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return LBVH_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_static_mu);
    StaticScratch &s = g_static[dev];
    if (!s.store) {
        void *store = nullptr, *flags = nullptr;
        if (cudaGetSymbolAddress(&store, g_static_store) != cudaSuccess) return LBVH_ERR_CUDA;
        if (cudaGetSymbolAddress(&flags, g_static_flags) != cudaSuccess) return LBVH_ERR_CUDA;
        s.store = static_cast<unsigned long long *>(store);
        s.flags = static_cast<uint32_t *>(flags);
    }
    *out = s;
    return LBVH_OK;
}

}  // namespace

extern "C" lbvh_status lbvh_construct_static(const uint64_t *d_sorted_codes, const uint32_t *d_perm,
                                             const float *d_prims, int64_t n, int kind, float *d_inodes,
                                             float *d_leaves, uint32_t *d_flags, lbvh_stream_t stream) {
    if (n < 1 || n > kStaticMaxPrims) return LBVH_ERR_INVALID;
    if (kind != LBVH_PRIM_POINTS && kind != LBVH_PRIM_BOXES) return LBVH_ERR_INVALID;
    if (!d_sorted_codes || !d_perm || !d_prims || !d_leaves || (n > 1 && !d_inodes)) return LBVH_ERR_INVALID;
    StaticScratch scratch;
    const lbvh_status st = static_scratch(&scratch);
    if (st != LBVH_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // every call shares the array: the store words must start empty (zero)
    if (n > 1 && cudaMemsetAsync(scratch.store, 0, (size_t)(n - 1) * sizeof(unsigned long long), s) != cudaSuccess)
        return LBVH_ERR_CUDA;
    uint32_t *flags = d_flags;
    if (!flags) {
        flags = scratch.flags;
        if (cudaMemsetAsync(flags, 0, sizeof(uint32_t), s) != cudaSuccess) return LBVH_ERR_CUDA;
    }
    lbvh::launch_construct(d_sorted_codes, d_perm, d_prims, n, kind, reinterpret_cast<float4 *>(d_inodes),
                           reinterpret_cast<float4 *>(d_leaves), scratch.store, flags, s);
    return cudaGetLastError() == cudaSuccess ? LBVH_OK : LBVH_ERR_CUDA;
}

