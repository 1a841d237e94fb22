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
//     lie inside one group of consecutive leaves (256) meet in
//     shared memory (block-scope exchange, sibling box from shared memory);
//     only the nodes spanning a group's edge meet in the device-scope
//     `store` words (sibling box through L2, ld.global.cg). Batches group
//     their global sorted positions the same way (a group may hold several
//     trees; a split only ever joins leaves of one).
#include <atomic>

#include <cuda/atomic>

#include "lbvh_internal.cuh"
#include "morton.cuh"

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
// and, for the second thread, makes the sibling's node visible (acquire), as
// one acq_rel atomic. Measured with every exchange at device scope at 2^25
// points: 2.29 ms, against 2.96 ms for a relaxed exchange between two
// __threadfence() and 2.76 ms for a release-only exchange with an acquire
// fence taken by the second thread alone.
__device__ __forceinline__ unsigned long long publish_exchange(unsigned long long *slot, unsigned long long v) {
    cuda::atomic_ref<unsigned long long, cuda::thread_scope_device> a(*slot);
    return a.exchange(v, cuda::memory_order_acq_rel);
}

// Test hook (lbvh_test_construct_jitter): with kJitter, a thread waits a
// pseudo-random time of up to max_ns before each exchange (its delay drawn
// by splitmix64 from the seed and a salt naming the thread's place and
// level; %globaltimer, with an iteration cap as a backstop), so that the
// two children of a node arrive in other orders than the hardware's usual
// one. The kernels of every other build are instantiated without it.
struct Jitter {
    unsigned long long seed = 0;
    unsigned max_ns = 0;
};

template <bool kJitter>
__device__ __forceinline__ void jitter_wait(const Jitter &j, unsigned long long salt) {
    if constexpr (kJitter) {
        unsigned long long x = j.seed + (salt + 1ull) * 0x9e3779b97f4a7c15ull;
        x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ull;
        x = (x ^ (x >> 27)) * 0x94d049bb133111ebull;
        x ^= x >> 31;
        const unsigned long long d = x % ((unsigned long long)j.max_ns + 1ull);
        unsigned long long t0, t;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
        for (unsigned k = 0; k < (1u << 16); ++k) {
            asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
            if (t - t0 >= d) break;
        }
    }
}

// A thread's finished node while it climbs: leaf range [l, r], delta*(l-1),
// delta*(r), delta*(r+1), and its box.
struct Climb {
    uint32_t l, r, d_left, d_right, d_next;
    float3 lo, hi;
};

// delta*(i-1), delta*(i), delta*(i+1) around leaf i (255 = +inf at -1 and n-1).
// Codes out of order (c0 > c1) latch kFlagCorrupt: the input is not sorted.
__device__ __forceinline__ void leaf_deltas(int i, int n, const uint64_t *__restrict__ codes, uint32_t &dl,
                                            uint32_t &dr, uint32_t &drn, uint32_t *flags) {
    const uint64_t c0 = codes[i];
    dl = i > 0 ? delta_star(codes[i - 1], c0, (uint32_t)(i - 1)) : kInf;
    dr = kInf;
    drn = kInf;
    if (i + 1 < n) {
        const uint64_t c1 = codes[i + 1];
        if (c0 > c1) atomicOr(flags, kFlagCorrupt);
        dr = delta_star(c0, c1, (uint32_t)i);
        if (i + 2 < n) drn = delta_star(c1, codes[i + 2], (uint32_t)(i + 1));
    }
}

// The primitive's box (a point's box is the point).
template <int kKind>
__device__ __forceinline__ void gather_box(const float *__restrict__ prims, uint32_t p_id, float3 &lo, float3 &hi) {
    if (kKind == LBVH_PRIM_POINTS) {
        lo = make_float3(prims[3 * (int64_t)p_id], prims[3 * (int64_t)p_id + 1], prims[3 * (int64_t)p_id + 2]);
        hi = lo;
    } else {
        const float *b = prims + 6 * (int64_t)p_id;
        lo = make_float3(b[0], b[1], b[2]);
        hi = make_float3(b[3], b[4], b[5]);
    }
}

// Algorithm 4's leaf step for leaf i of one tree of n leaves, given its
// delta* values and its primitive (own index p_own, box lo/hi): the leaf's
// skip and box are written out and the climb state is set.
template <int kKind>
__device__ __forceinline__ void leaf_write(int i, int n, uint32_t p_own, float3 lo, float3 hi, float4 *leaves,
                                           uint32_t dl, uint32_t dr, uint32_t drn, Climb &c) {
    const int ni = n - 1;
    const int leaf_skip = i == n - 1 ? kSentinel : (dr < drn ? ni + i + 1 : i + 1);
    // the leaf's skip is position i+1: one bit says I_{i+1} rather than L_{i+1}
    const uint32_t word = p_own | (leaf_skip >= 0 && leaf_skip < ni ? kLeafSkipInternal : 0u);
    if (kKind == LBVH_PRIM_POINTS) {
        leaves[i] = make_float4(lo.x, lo.y, lo.z, __uint_as_float(word));
    } else {
        leaves[2 * (int64_t)i] = make_float4(lo.x, lo.y, lo.z, __uint_as_float(word));
        leaves[2 * (int64_t)i + 1] = make_float4(hi.x, hi.y, hi.z, 0.0f);
    }
    c = Climb{(uint32_t)i, (uint32_t)i, dl, dr, drn, lo, hi};
}

// The leaf step from sorted codes and a permutation. perm holds primitive
// indices into `prims`, the tree's own indices being perm - perm_base. False
// (and kFlagCorrupt) if perm is not a permutation of this tree.
template <int kKind>
__device__ __forceinline__ bool leaf_step(int i, int n, const uint64_t *__restrict__ codes,
                                          const uint32_t *__restrict__ perm, uint32_t perm_base,
                                          const float *__restrict__ prims, float4 *leaves, uint32_t *flags,
                                          Climb &c) {
    uint32_t dl, dr, drn;
    leaf_deltas(i, n, codes, dl, dr, drn, flags);
    const uint32_t p_id = perm[i];
    const uint32_t p_own = p_id - perm_base;
    if (p_own >= (uint32_t)n) {  // not a permutation of this tree: the sort failed
        atomicOr(flags, kFlagCorrupt);
        return false;
    }
    float3 lo, hi;
    gather_box<kKind>(prims, p_id, lo, hi);
    leaf_write<kKind>(i, n, p_own, lo, hi, leaves, dl, dr, drn, c);
    return true;
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
template <int kKind, bool kJitter = false>
__device__ __forceinline__ void climb_global(Climb c, int n, float4 *inodes, const float4 *leaves,
                                             unsigned long long *store, uint32_t *flags,
                                             const Jitter &jt = Jitter{}) {
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
        jitter_wait<kJitter>(jt, (unsigned long long)p << 8 | (unsigned)level);
        const unsigned long long other = publish_exchange(store + p, mine);
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

// Algorithm 4 with the climb split in two phases. The leaves are cut into
// groups of kGroup consecutive leaves [a, a + kGroup), one per CTA. A node
// whose leaf range lies inside a group has both children there, so its split
// p has a <= p and p + 1 < a + kGroup; such splits meet in a shared-memory
// word with a block-scope exchange, and the sibling's box is read from shared
// memory. A thread stops phase 1 at a split on the group's edge, or as the
// first up at a word. After the group's barrier every node inside the group
// is finished; a word still holding its first thread's half has a sibling
// that spans the group's edge, and that thread, like one stopped at the edge,
// continues with the device-scope exchanges of climb_global. Each node is
// still written once, by the second thread up at its split, with the same
// fields: only where the two halves meet changes. Group size, with the
// climbs that leave a group handed to a second kernel (construct time at 2^25
// points, 63-bit codes): 64 leaves 1.83 ms (8 hand-off slots 1.67), 128
// 1.64, 256 1.56 (16 slots; 12: 1.57; 8: 1.55; 32: 1.67), 512 1.57.
constexpr int kGroup = 256;

struct GroupSmem {
    unsigned long long word[kGroup];    // split at global position a + j: word[j]
    float3 lo[2][kGroup], hi[2][kGroup];  // boxes: [0] leaf, [1] internal node, by global position / index
    uint64_t code[kGroup + 3];          // sorted codes a-1 .. a+kGroup+1 (construct_encode_kernel)
    int failed;
    int pending;                        // climbs handed to climb_pending_kernel
};

// Climbs that leave a group: the CTA hands up to kPendSlots of them to
// climb_pending_kernel through its own slots (16 bytes each: l, r, the three
// delta* values and a valid bit), so that no CTA waits on device-scope
// exchanges with most of its threads done. On uniform points a group of 128
// leaves has 7.3 such climbs on average and 13 at most (one more level of
// the tree per doubling of the group); more than kPendSlots climb in place.
constexpr int kPendSlots = 12;
constexpr uint32_t kPendValid = 1u << 31;

// Both phases for thread t, holding leaf i's climb state c (go: the leaf was
// written and the tree has internal nodes), of a tree of n leaves whose leaf
// 0 sits at global position o (0 for a single tree; trees of a batch follow
// each other), in the group whose first global position is a. A split joins
// two leaves of one tree, so groups may hold several trees. Every thread of
// the CTA must call this (it holds the group's barrier).
// pend (nullable): the CTA's kPendSlots slots.
template <int kKind, bool kJitter = false>
__device__ __forceinline__ void two_phase(GroupSmem &sm, bool go, Climb c, int n, int64_t o, int64_t a, int t,
                                          float4 *inodes, const float4 *leaves, unsigned long long *store,
                                          uint32_t *flags, uint4 *pend, const Jitter &jt = Jitter{}) {
    const int ni = n - 1;
    bool pending = false, in_word = false;
    int word_at = 0;
    if (go) {
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
            jitter_wait<kJitter>(jt, (unsigned long long)p << 8 | (unsigned)level);
            cuda::atomic_ref<unsigned long long, cuda::thread_scope_block> w(sm.word[at]);
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
            const int sat = (int)(o + (sibling < ni ? sibling : sibling - ni) - a);  // at or at + 1
            const int q = write_parent(c, p, n, sm.lo[k][sat], sm.hi[k][sat], inodes);
            if (q == 0) break;  // the root: the whole tree lies in this group
            const int qat = (int)(o + q - a);  // q is l or r, inside the group
            sm.lo[1][qat] = c.lo;
            sm.hi[1][qat] = c.hi;
        }
    }
    __syncthreads();
    if (!pending) return;
    if (in_word && sm.word[word_at] == 0ull) return;  // the sibling came and carried on
    if (pend) {
        const int slot = atomicAdd(&sm.pending, 1);
        if (slot < kPendSlots) {
            pend[slot] = make_uint4(c.l, c.r, kPendValid | c.d_left | c.d_right << 8 | c.d_next << 16, 0u);
            return;
        }
    }
    // this thread wrote its own node, so its device-scope release covers it
    climb_global<kKind, kJitter>(c, n, inodes, leaves, store, flags, jt);
}

// The climbs handed over by the groups, one thread per slot: the climber's
// node (range [l, r], written by the first kernel) is read back for its box
// and the climb goes on with device-scope exchanges. Every valid slot is
// cleared, so the slots are zero again for the next build.
template <int kKind, bool kJitter>
__global__ void __launch_bounds__(256)
    climb_pending_kernel(uint4 *pend, int64_t slots, int n, float4 *inodes, const float4 *leaves,
                         unsigned long long *store, uint32_t *flags, Jitter jt) {
    const int64_t k = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (k >= slots) return;
    const uint4 e = pend[k];
    if (!(e.z & kPendValid)) return;
    pend[k] = make_uint4(0u, 0u, 0u, 0u);
    if (__ldcg(flags) & (kFlagTimeout | kFlagCorrupt)) return;
    const int ni = n - 1;
    Climb c;
    c.l = e.x;
    c.r = e.y;
    c.d_left = e.z & 0xffu;
    c.d_right = (e.z >> 8) & 0xffu;
    c.d_next = (e.z >> 16) & 0xffu;
    if (c.l > c.r || c.r >= (uint32_t)n) {
        atomicOr(flags, kFlagCorrupt);
        return;
    }
    // the node of range [l, r]: leaf l, or internal node r or l (its Karras index)
    const int id = c.l == c.r ? ni + (int)c.l : (c.d_right < c.d_left ? (int)c.r : (int)c.l);
    load_node_box<kKind>(inodes, leaves, ni, id, c.lo, c.hi);
    climb_global<kKind, kJitter>(c, n, inodes, leaves, store, flags, jt);
}

// Clears the CTA's shared words and reads the build's error flags: true if
// an earlier stage failed, in which case the whole CTA returns and leaves
// `store` untouched.
__device__ __forceinline__ bool group_start(GroupSmem &sm, const uint32_t *flags) {
    sm.word[threadIdx.x] = 0ull;
    if (threadIdx.x == 0) {
        sm.failed = (__ldcg(flags) & (kFlagTimeout | kFlagCorrupt)) != 0;
        sm.pending = 0;
    }
    __syncthreads();
    return sm.failed != 0;
}

// Algorithm 4 from sorted codes and a permutation (lbvh_build_from_sorted,
// refit, the no-allocation entry point).
template <int kKind, bool kJitter>
__global__ void __launch_bounds__(kGroup, 2048 / kGroup)
    construct_block_kernel(const uint64_t *__restrict__ codes, const uint32_t *__restrict__ perm,
                           const float *__restrict__ prims, int n, float4 *inodes, float4 *leaves,
                           unsigned long long *store, uint32_t *flags, uint4 *pend, Jitter jt) {
    __shared__ GroupSmem sm;
    if (group_start(sm, flags)) return;
    const int t = threadIdx.x;
    const int i = blockIdx.x * kGroup + t;
    Climb c;
    const bool ok = i < n && leaf_step<kKind>(i, n, codes, perm, 0u, prims, leaves, flags, c);
    two_phase<kKind, kJitter>(sm, ok && n > 1, c, n, 0, (int64_t)blockIdx.x * kGroup, t, inodes, leaves, store,
                              flags, pend ? pend + (int64_t)blockIdx.x * kPendSlots : nullptr, jt);
}

// Algorithm 4 after a sort that kept only the permutation. Each thread
// gathers its leaf's primitive and derives its Morton code again with the
// encoder's function (the same bits); the codes of the CTA's leaves and of
// three neighbours (positions a-1, a+kGroup, a+kGroup+1, gathered by threads
// 0-2) meet in shared memory for the delta* values. The sorted codes are
// written to codes_out (the tree keeps them for export and refit).
template <int kKind, bool kJitter>
__global__ void __launch_bounds__(kGroup, 2048 / kGroup)
    construct_encode_kernel(const uint32_t *__restrict__ perm, const float *__restrict__ prims,
                            const float *__restrict__ bounds, int b, int n, uint64_t *__restrict__ codes_out,
                            float4 *inodes, float4 *leaves, unsigned long long *store, uint32_t *flags,
                            uint4 *pend, Jitter jt) {
    __shared__ GroupSmem sm;
    if (group_start(sm, flags)) return;
    const int t = threadIdx.x;
    const int64_t a = (int64_t)blockIdx.x * kGroup;
    const int i = (int)a + t;
    const Grid3 g = make_grid(bounds, b);
    bool ok = i < n;
    uint32_t p_id = 0;
    float3 lo = make_float3(0.f, 0.f, 0.f), hi = lo;
    if (ok) {
        p_id = __ldcs(perm + i);
        if (p_id >= (uint32_t)n) {  // not a permutation: the sort failed
            atomicOr(flags, kFlagCorrupt);
            ok = false;
        } else {
            gather_box<kKind>(prims, p_id, lo, hi);
        }
    }
    // the three neighbours outside the CTA's range
    int64_t hpos = -1;
    float3 hlo = lo, hhi = hi;
    if (t < 3) {
        hpos = t == 0 ? a - 1 : a + kGroup + t - 1;
        if (hpos >= 0 && hpos < n) {
            const uint32_t hp = perm[hpos];
            if (hp < (uint32_t)n) gather_box<kKind>(prims, hp, hlo, hhi);
            else hpos = -1;
        } else {
            hpos = -1;
        }
    }
    if (ok) {
        const uint64_t code = morton(__fmul_rn(__fadd_rn(lo.x, hi.x), 0.5f), __fmul_rn(__fadd_rn(lo.y, hi.y), 0.5f),
                                     __fmul_rn(__fadd_rn(lo.z, hi.z), 0.5f), g);
        sm.code[t + 1] = code;
        codes_out[i] = code;
    }
    if (hpos >= 0)
        sm.code[t == 0 ? 0 : kGroup + t] =
            morton(__fmul_rn(__fadd_rn(hlo.x, hhi.x), 0.5f), __fmul_rn(__fadd_rn(hlo.y, hhi.y), 0.5f),
                   __fmul_rn(__fadd_rn(hlo.z, hhi.z), 0.5f), g);
    __syncthreads();
    Climb c;
    if (ok) {
        const uint64_t c0 = sm.code[t + 1];
        const uint32_t dl = i > 0 ? delta_star(sm.code[t], c0, (uint32_t)(i - 1)) : kInf;
        uint32_t dr = kInf, drn = kInf;
        if (i + 1 < n) {
            const uint64_t c1 = sm.code[t + 2];
            dr = delta_star(c0, c1, (uint32_t)i);
            if (i + 2 < n) drn = delta_star(c1, sm.code[t + 3], (uint32_t)(i + 1));
        }
        leaf_write<kKind>(i, n, p_id, lo, hi, leaves, dl, dr, drn, c);
    }
    two_phase<kKind, kJitter>(sm, ok && n > 1, c, n, 0, a, t, inodes, leaves, store, flags,
                              pend ? pend + (int64_t)blockIdx.x * kPendSlots : nullptr, jt);
}

// Many trees at once, grouped by global sorted position: global position g
// belongs to the instance b with off[b] <= g < off[b+1]; its tree's records
// start at node_start[b] (float4 units) and its store words at store_start[b].
template <int kKind>
__global__ void __launch_bounds__(kGroup, 2048 / kGroup)
    batch_construct_block_kernel(const uint64_t *__restrict__ codes, const uint32_t *__restrict__ perm,
                                 const float *__restrict__ prims, const int64_t *__restrict__ off,
                                 const int64_t *__restrict__ node_start, const int64_t *__restrict__ store_start,
                                 int count, int64_t total, float4 *nodes, unsigned long long *store,
                                 uint32_t *flags) {
    __shared__ GroupSmem sm;
    if (group_start(sm, flags)) return;
    const int t = threadIdx.x;
    const int64_t g = (int64_t)blockIdx.x * kGroup + t;
    const bool active = g < total;
    const int b = active ? instance_of(off, count, g) : 0;
    const int64_t o = active ? off[b] : 0;
    const int n = active ? (int)(off[b + 1] - o) : 1;
    float4 *inodes = nodes + (active ? node_start[b] : 0);
    float4 *leaves = inodes + 2 * (int64_t)(n - 1);
    Climb c;
    const bool ok = active && leaf_step<kKind>((int)(g - o), n, codes + o, perm + o, (uint32_t)o, prims, leaves,
                                               flags, c);
    two_phase<kKind>(sm, ok && n > 1, c, n, o, (int64_t)blockIdx.x * kGroup, t, inodes, leaves,
                     store + (active ? store_start[b] : 0), flags, nullptr);
}

}  // namespace

void launch_batch_construct(const uint64_t *sorted_codes, const uint32_t *perm, const float *prims,
                            const BatchTables &bt, int kind, float4 *nodes, unsigned long long *store,
                            uint32_t *flags, cudaStream_t s) {
    if (bt.total_prims <= 0) return;
    const unsigned blocks = (unsigned)((bt.total_prims + kGroup - 1) / kGroup);
    auto k = kind == LBVH_PRIM_POINTS ? batch_construct_block_kernel<LBVH_PRIM_POINTS>
                                      : batch_construct_block_kernel<LBVH_PRIM_BOXES>;
    k<<<blocks, kGroup, 0, s>>>(sorted_codes, perm, prims, bt.prim_off, bt.node_start, bt.store_start, bt.count,
                                bt.total_prims, nodes, store, flags);
    count_launches(1);
}

size_t construct_pend_bytes(int64_t n) { return (size_t)((n + kGroup - 1) / kGroup) * kPendSlots * sizeof(uint4); }

namespace {

// lbvh_test_construct_jitter's setting (max_ns 0: off)
std::atomic<unsigned long long> g_jitter_seed{0};
std::atomic<unsigned> g_jitter_ns{0};

Jitter jitter_setting() {
    Jitter j;
    j.seed = g_jitter_seed.load(std::memory_order_relaxed);
    j.max_ns = g_jitter_ns.load(std::memory_order_relaxed);
    return j;
}

void launch_pending(int64_t n, int kind, float4 *inodes, float4 *leaves, unsigned long long *store,
                    uint32_t *flags, void *pend, const Jitter &jt, cudaStream_t s) {
    if (!pend || n < 2) return;
    const int64_t slots = (n + kGroup - 1) / kGroup * kPendSlots;
    const unsigned blocks = (unsigned)((slots + 255) / 256);
    const bool pts = kind == LBVH_PRIM_POINTS;
    auto k = jt.max_ns ? (pts ? climb_pending_kernel<LBVH_PRIM_POINTS, true> : climb_pending_kernel<LBVH_PRIM_BOXES, true>)
                       : (pts ? climb_pending_kernel<LBVH_PRIM_POINTS, false>
                              : climb_pending_kernel<LBVH_PRIM_BOXES, false>);
    k<<<blocks, 256, 0, s>>>(static_cast<uint4 *>(pend), slots, (int)n, inodes, leaves, store, flags, jt);
    count_launches(1);
}

}  // namespace

void launch_construct(const uint64_t *sorted_codes, const uint32_t *perm, const float *prims,
                      int64_t n, int kind, float4 *inodes, float4 *leaves,
                      unsigned long long *store, uint32_t *flags, void *pend, cudaStream_t s) {
    if (n <= 0) return;
    const unsigned blocks = (unsigned)((n + kGroup - 1) / kGroup);
    const Jitter jt = jitter_setting();
    const bool pts = kind == LBVH_PRIM_POINTS;
    auto k = jt.max_ns ? (pts ? construct_block_kernel<LBVH_PRIM_POINTS, true>
                              : construct_block_kernel<LBVH_PRIM_BOXES, true>)
                       : (pts ? construct_block_kernel<LBVH_PRIM_POINTS, false>
                              : construct_block_kernel<LBVH_PRIM_BOXES, false>);
    k<<<blocks, kGroup, 0, s>>>(sorted_codes, perm, prims, (int)n, inodes, leaves, store, flags,
                                static_cast<uint4 *>(pend), jt);
    count_launches(1);
    launch_pending(n, kind, inodes, leaves, store, flags, pend, jt, s);
}

void launch_construct_encode(const uint32_t *perm, const float *prims, const float *bounds, int bits, int64_t n,
                             int kind, uint64_t *codes_out, float4 *inodes, float4 *leaves,
                             unsigned long long *store, uint32_t *flags, void *pend, cudaStream_t s) {
    if (n <= 0) return;
    const unsigned blocks = (unsigned)((n + kGroup - 1) / kGroup);
    const Jitter jt = jitter_setting();
    const bool pts = kind == LBVH_PRIM_POINTS;
    auto k = jt.max_ns ? (pts ? construct_encode_kernel<LBVH_PRIM_POINTS, true>
                              : construct_encode_kernel<LBVH_PRIM_BOXES, true>)
                       : (pts ? construct_encode_kernel<LBVH_PRIM_POINTS, false>
                              : construct_encode_kernel<LBVH_PRIM_BOXES, false>);
    k<<<blocks, kGroup, 0, s>>>(perm, prims, bounds, bits / 3, (int)n, codes_out, inodes, leaves, store, flags,
                                static_cast<uint4 *>(pend), jt);
    count_launches(1);
    launch_pending(n, kind, inodes, leaves, store, flags, pend, jt, s);
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

// Device addresses of the two arrays for the current device. Host code must
// not use the symbols themselves (in host code they name host-side stand-ins).
// The lookup is repeated on every call: it is cheap, and an address kept from
// an earlier call would go stale if the caller reset the device (the module,
// and with it the arrays, is loaded again into the new context).
struct StaticScratch {
    unsigned long long *store = nullptr;
    uint32_t *flags = nullptr;
};

lbvh_status static_scratch(StaticScratch *out) {
    void *store = nullptr, *flags = nullptr;
    if (cudaGetSymbolAddress(&store, g_static_store) != cudaSuccess) return LBVH_ERR_CUDA;
    if (cudaGetSymbolAddress(&flags, g_static_flags) != cudaSuccess) return LBVH_ERR_CUDA;
    out->store = static_cast<unsigned long long *>(store);
    out->flags = static_cast<uint32_t *>(flags);
    return LBVH_OK;
}

}  // namespace

extern "C" lbvh_status lbvh_test_construct_jitter(unsigned long long seed, unsigned max_ns) {
    if (max_ns > 1000000u) return LBVH_ERR_INVALID;
    lbvh::g_jitter_seed.store(seed, std::memory_order_relaxed);
    lbvh::g_jitter_ns.store(max_ns, std::memory_order_relaxed);
    return LBVH_OK;
}

extern "C" lbvh_status lbvh_construct_static(const uint64_t *d_sorted_codes, const uint32_t *d_perm,
                                             const float *d_prims, int64_t n, int kind, float *d_inodes,
                                             float *d_leaves, uint32_t *d_flags, lbvh_stream_t stream) {
    if (n < 1 || n > kStaticMaxPrims) return LBVH_ERR_INVALID;
    if (kind != LBVH_PRIM_POINTS && kind != LBVH_PRIM_BOXES) return LBVH_ERR_INVALID;
    if (!d_sorted_codes || !d_perm || !d_prims || !d_leaves || (n > 1 && !d_inodes)) return LBVH_ERR_INVALID;
    (void)cudaGetLastError();  // an earlier, unrelated error must not be charged to this call
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
                           reinterpret_cast<float4 *>(d_leaves), scratch.store, flags, nullptr, s);
    return cudaGetLastError() == cudaSuccess ? LBVH_OK : LBVH_ERR_CUDA;
}

