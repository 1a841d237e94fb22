// variants.cu -- the two hierarchy builds the paper compares Algorithm 4 with
// (Sec. 3 and Sec. 5), written as GPU kernels so that the three builds can be
// timed against each other on the same sorted codes. Both end in the tree
// layout Algorithm 4 writes (Karras' ordering, left child, skip, box), so a
// tree built either way is queried and exported like any other.
//
// Karras (Sec. 3.1): one thread per internal node i finds the node's range
// (it starts or ends at i: direction towards the neighbour with the smaller
// delta*, then an exponential and a binary search for the far end, using
// delta(i, j) = highest differing bit of the augmented keys i and j), the split
// inside it by a second binary search, and writes the children (at split and
// split + 1), the skip (Algorithm 2) and the children's parent. Boxes need a
// second, bottom-up pass: one thread per leaf climbs through the parent links
// and the second thread to reach a node (an arrival counter) writes its box.
//
// Apetrei (Algorithm 3): one thread per leaf climbs; each thread writes its
// own side's child pointer into the parent before a compare-and-swap on the
// parent's store slot; the first arrival stops, the second receives the other
// range end, recomputes the outdated delta* from the codes, reads the other
// child pointer to find its sibling, and writes the parent's box and range.
// Nodes are in Apetrei's ordering (an internal node's index is its split) and
// carry no skips: that is what the paper's Algorithm 4 changes. A second pass
// converts every node to Karras' ordering (index r or l of its range) with
// its skip (Algorithm 2), and checks each child pointer of Algorithm 3
// against the ranges.
#include <cuda/atomic>

#include "lbvh_internal.cuh"

namespace lbvh {

namespace {

constexpr int kThreads = 256;
constexpr uint32_t kInf = 255;

// delta of two sorted positions: 64 + highest differing code bit, or the
// highest differing bit of the positions when the codes are equal.
__device__ __forceinline__ uint32_t delta_pair(uint64_t ci, uint64_t cj, uint32_t i, uint32_t j) {
    const uint64_t x = ci ^ cj;
    if (x) return 127u - (uint32_t)__clzll((long long)x);
    return 31u - (uint32_t)__clz((int)(i ^ j));
}

// delta*(k) = delta(k, k+1); +inf outside [0, n-2].
__device__ __forceinline__ uint32_t delta_gap(const uint64_t *__restrict__ codes, int n, int k) {
    if (k < 0 || k >= n - 1) return kInf;
    return delta_pair(codes[k], codes[k + 1], (uint32_t)k, (uint32_t)k + 1u);
}

__device__ __forceinline__ uint32_t delta_to(const uint64_t *__restrict__ codes, int n, int i, uint64_t ci,
                                             int j) {
    if (j < 0 || j >= n) return kInf;
    return delta_pair(ci, codes[j], (uint32_t)i, (uint32_t)j);
}

template <int kKind>
__device__ __forceinline__ void leaf_box(const float *__restrict__ prims, uint32_t p, float3 &lo, float3 &hi) {
    if (kKind == LBVH_PRIM_POINTS) {
        lo = make_float3(prims[3 * (int64_t)p], prims[3 * (int64_t)p + 1], prims[3 * (int64_t)p + 2]);
        hi = lo;
    } else {
        const float *b = prims + 6 * (int64_t)p;
        lo = make_float3(b[0], b[1], b[2]);
        hi = make_float3(b[3], b[4], b[5]);
    }
}

template <int kKind>
__device__ __forceinline__ void write_leaf(float4 *leaves, int k, float3 lo, float3 hi, uint32_t word) {
    if (kKind == LBVH_PRIM_POINTS) {
        leaves[k] = make_float4(lo.x, lo.y, lo.z, __uint_as_float(word));
    } else {
        leaves[2 * (int64_t)k] = make_float4(lo.x, lo.y, lo.z, __uint_as_float(word));
        leaves[2 * (int64_t)k + 1] = make_float4(hi.x, hi.y, hi.z, 0.0f);
    }
}

template <int kKind>
__device__ __forceinline__ void read_leaf_box(const float4 *leaves, int k, float3 &lo, float3 &hi) {
    if (kKind == LBVH_PRIM_POINTS) {
        const float4 a = __ldcg(leaves + k);
        lo = make_float3(a.x, a.y, a.z);
        hi = lo;
    } else {
        const float4 a = __ldcg(leaves + 2 * (int64_t)k), b = __ldcg(leaves + 2 * (int64_t)k + 1);
        lo = make_float3(a.x, a.y, a.z);
        hi = make_float3(b.x, b.y, b.z);
    }
}

// The same union with the ordered minimum and maximum written as comparisons
// (identical results for finite values). The Karras box pass runs at 2.83 ms
// with it against 5.17 ms with grow() (2^25 points; the climb's loads and
// its acq_rel counter are scheduled differently), while Algorithm 3's climb
// is faster with grow() (4.0 against 6.1 ms).
__device__ __forceinline__ float min_cmp(float a, float b) { return (a < b || (a == b && __float_as_int(a) < 0)) ? a : b; }
__device__ __forceinline__ float max_cmp(float a, float b) { return (a > b || (a == b && __float_as_int(a) >= 0)) ? a : b; }
__device__ __forceinline__ void grow_cmp(float3 &lo, float3 &hi, float3 slo, float3 shi) {
    lo = make_float3(min_cmp(lo.x, slo.x), min_cmp(lo.y, slo.y), min_cmp(lo.z, slo.z));
    hi = make_float3(max_cmp(hi.x, shi.x), max_cmp(hi.y, shi.y), max_cmp(hi.z, shi.z));
}

__device__ __forceinline__ void grow(float3 &lo, float3 &hi, float3 slo, float3 shi) {
    lo = make_float3(min_ordered(lo.x, slo.x), min_ordered(lo.y, slo.y), min_ordered(lo.z, slo.z));
    hi = make_float3(max_ordered(hi.x, shi.x), max_ordered(hi.y, shi.y), max_ordered(hi.z, shi.z));
}

// Leaf k's skip is position k+1: internal when delta*(k) >= delta*(k+1).
__device__ __forceinline__ uint32_t leaf_skip_bit(const uint64_t *__restrict__ codes, int n, int k) {
    if (k >= n - 1) return 0u;
    return delta_gap(codes, n, k) < delta_gap(codes, n, k + 1) ? 0u : kLeafSkipInternal;
}

// Algorithm 2: the skip of a node whose range ends at r.
__device__ __forceinline__ int node_skip(const uint64_t *__restrict__ codes, int n, int r) {
    if (r == n - 1) return kSentinel;
    return delta_gap(codes, n, r) < delta_gap(codes, n, r + 1) ? (n - 1) + r + 1 : r + 1;
}

// ---------------------------------------------------------------- Karras

__global__ void __launch_bounds__(kThreads)
    karras_nodes_kernel(const uint64_t *__restrict__ codes, int n, int32_t *__restrict__ left,
                        int32_t *__restrict__ right, int32_t *__restrict__ skip, int32_t *__restrict__ parent,
                        uint32_t *flags) {
    const int i = blockIdx.x * kThreads + threadIdx.x;
    const int ni = n - 1;
    if (i >= ni) return;
    if (__ldcg(flags) & (kFlagTimeout | kFlagCorrupt)) return;  // the sort failed
    const uint64_t ci = codes[i];
    const uint32_t dl = delta_to(codes, n, i, ci, i - 1);
    const uint32_t dr = delta_to(codes, n, i, ci, i + 1);
    const int d = dr < dl ? 1 : -1;
    const uint32_t limit = d == 1 ? dl : dr;  // every gap inside the range is below it
    // far end: exponential, then binary search (at most 32 doublings)
    int lmax = 2;
    while (lmax < (1 << 30) && delta_to(codes, n, i, ci, i + lmax * d) < limit) lmax <<= 1;
    int len = 0;
    for (int t = lmax >> 1; t >= 1; t >>= 1)
        if (delta_to(codes, n, i, ci, i + (len + t) * d) < limit) len += t;
    const int j = i + len * d;
    const uint32_t dnode = delta_to(codes, n, i, ci, j);
    // split: the last position (from i) still on i's side of the largest gap
    int s = 0, step = len;
    do {
        step = (step + 1) >> 1;
        const int x = s + step;
        if (x < len && delta_to(codes, n, i, ci, i + x * d) < dnode) s = x;
    } while (step > 1);
    const int g = i + s * d + (d < 0 ? -1 : 0);
    const int l = min(i, j), r = max(i, j);
    if (len < 1 || g < l || g >= r) {  // not a valid radix tree: unsorted codes
        atomicOr(flags, kFlagCorrupt);
        return;
    }
    const int lc = l == g ? ni + g : g;
    const int rc = r == g + 1 ? ni + g + 1 : g + 1;
    left[i] = lc;
    right[i] = rc;
    skip[i] = node_skip(codes, n, r);
    parent[lc] = i;
    parent[rc] = i;
    if (i == 0) parent[0] = -1;
}

template <int kKind>
__global__ void __launch_bounds__(kThreads)
    karras_boxes_kernel(const uint64_t *__restrict__ codes, const uint32_t *__restrict__ perm,
                        const float *__restrict__ prims, int n, const int32_t *__restrict__ left,
                        const int32_t *__restrict__ right, const int32_t *__restrict__ skip,
                        const int32_t *__restrict__ parent, float4 *inodes, float4 *leaves,
                        unsigned int *counters, uint32_t *flags) {
    const int k = blockIdx.x * kThreads + threadIdx.x;
    if (k >= n) return;
    if (__ldcg(flags) & (kFlagTimeout | kFlagCorrupt)) return;  // an earlier step failed: counters untouched
    const int ni = n - 1;
    const uint32_t p_id = perm[k];
    if (p_id >= (uint32_t)n) {
        atomicOr(flags, kFlagCorrupt);
        return;
    }
    float3 lo, hi;
    leaf_box<kKind>(prims, p_id, lo, hi);
    write_leaf<kKind>(leaves, k, lo, hi, p_id | leaf_skip_bit(codes, n, k));
    if (n == 1) return;
    int node = ni + k;
    for (int level = 0; level < 128; ++level) {
        const int p = parent[node];
        if (p < 0 || p >= ni) {
            atomicOr(flags, kFlagCorrupt);
            return;
        }
        cuda::atomic_ref<unsigned int, cuda::thread_scope_device> c(counters[2 * (int64_t)p]);
        if (c.fetch_add(1u, cuda::memory_order_acq_rel) == 0u) return;  // first arrival
        counters[2 * (int64_t)p] = 0u;                                    // leave the counter clean
        const int lc = left[p], rc = right[p];
        const int sib = lc == node ? rc : lc;
        float3 slo, shi;
        if (sib >= ni) {
            read_leaf_box<kKind>(leaves, sib - ni, slo, shi);
        } else {
            const float4 a = __ldcg(inodes + 2 * (int64_t)sib), b = __ldcg(inodes + 2 * (int64_t)sib + 1);
            slo = make_float3(a.x, a.y, a.z);
            shi = make_float3(b.x, b.y, b.z);
        }
        grow_cmp(lo, hi, slo, shi);
        inodes[2 * (int64_t)p] = make_float4(lo.x, lo.y, lo.z, __int_as_float(lc));
        inodes[2 * (int64_t)p + 1] = make_float4(hi.x, hi.y, hi.z, __int_as_float(skip[p]));
        if (p == 0) return;
        node = p;
    }
    atomicOr(flags, kFlagCorrupt);
}

// ---------------------------------------------------------------- Apetrei

// Node p of Algorithm 3 (Apetrei ordering): {lo, left child}, {hi, right
// child}, {range l, range r, -, -}; child ids: internal p' < n-1, leaf k as
// (n-1) + k.
constexpr int kApetreiRecord = 3;

template <int kKind>
__global__ void __launch_bounds__(kThreads)
    apetrei_kernel(const uint64_t *__restrict__ codes, const uint32_t *__restrict__ perm,
                   const float *__restrict__ prims, int n, float4 *rec, float4 *leaves,
                   unsigned long long *store, uint32_t *flags) {
    const int i = blockIdx.x * kThreads + threadIdx.x;
    if (i >= n) return;
    if (__ldcg(flags) & (kFlagTimeout | kFlagCorrupt)) return;  // the sort failed: store untouched
    const int ni = n - 1;
    const uint32_t p_id = perm[i];
    if (p_id >= (uint32_t)n) {
        atomicOr(flags, kFlagCorrupt);
        return;
    }
    float3 lo, hi;
    leaf_box<kKind>(prims, p_id, lo, hi);
    write_leaf<kKind>(leaves, i, lo, hi, p_id);  // skips come with the second pass
    if (n == 1) return;
    int l = i, r = i;
    uint32_t d_left = delta_gap(codes, n, l - 1), d_right = delta_gap(codes, n, r);
    int cur = ni + i;
    for (int level = 0; level < 128; ++level) {
        int p, sib;
        unsigned long long old;
        const bool is_left = d_right < d_left;
        p = is_left ? r : l - 1;
        if (p < 0 || p >= ni) {
            atomicOr(flags, kFlagCorrupt);
            return;
        }
        float4 *node = rec + kApetreiRecord * (int64_t)p;
        // this thread's side of the parent, then the compare-and-swap
        reinterpret_cast<int *>(node + (is_left ? 0 : 1))[3] = cur;
        cuda::atomic_ref<unsigned long long, cuda::thread_scope_device> slot(store[p]);
        old = 0ull;
        const unsigned long long mine = 1ull + (unsigned long long)(is_left ? l : r);
        if (slot.compare_exchange_strong(old, mine, cuda::memory_order_acq_rel, cuda::memory_order_acquire))
            return;  // first arrival: the slot was empty
        store[p] = 0ull;  // second arrival: leave the slot empty again
        const int other = (int)(old - 1ull);
        if (other < 0 || other >= n) {
            atomicOr(flags, kFlagCorrupt);
            return;
        }
        if (is_left) {
            r = other;
            d_right = delta_gap(codes, n, r);  // recompute the outdated value
            sib = reinterpret_cast<const volatile int *>(node + 1)[3];
        } else {
            l = other;
            d_left = delta_gap(codes, n, l - 1);
            sib = reinterpret_cast<const volatile int *>(node)[3];
        }
        float3 slo, shi;
        if (sib >= ni) {
            if (sib - ni >= n) {
                atomicOr(flags, kFlagCorrupt);
                return;
            }
            read_leaf_box<kKind>(leaves, sib - ni, slo, shi);
        } else {
            if (sib < 0) {
                atomicOr(flags, kFlagCorrupt);
                return;
            }
            const float4 *s = rec + kApetreiRecord * (int64_t)sib;
            const float4 a = __ldcg(s), b = __ldcg(s + 1);
            slo = make_float3(a.x, a.y, a.z);
            shi = make_float3(b.x, b.y, b.z);
        }
        grow(lo, hi, slo, shi);
        const int lc = is_left ? cur : sib, rc = is_left ? sib : cur;
        node[0] = make_float4(lo.x, lo.y, lo.z, __int_as_float(lc));
        node[1] = make_float4(hi.x, hi.y, hi.z, __int_as_float(rc));
        node[2] = make_float4(__int_as_float(l), __int_as_float(r), 0.0f, 0.0f);
        if (l == 0 && r == ni) return;  // the range covers every leaf: the root
        cur = p;
    }
    atomicOr(flags, kFlagCorrupt);
}

// Apetrei node p -> Karras node q (r if delta*(r) < delta*(l-1), else l) with
// left child (at split p) and skip (Algorithm 2); leaf k's skip bit. Each
// child pointer of Algorithm 3 must be the node that covers the matching
// half of the range.
template <int kKind>
__global__ void __launch_bounds__(kThreads)
    apetrei_to_karras_kernel(const uint64_t *__restrict__ codes, const uint32_t *__restrict__ perm, int n,
                             const float4 *__restrict__ rec, float4 *inodes, float4 *leaves, uint32_t *flags) {
    const int k = blockIdx.x * kThreads + threadIdx.x;
    const int ni = n - 1;
    if (k < n) {
        const uint32_t word = perm[k] | leaf_skip_bit(codes, n, k);
        float4 *a = leaves + (kKind == LBVH_PRIM_POINTS ? (int64_t)k : 2 * (int64_t)k);
        reinterpret_cast<uint32_t *>(a)[3] = word;
    }
    if (k >= ni) return;
    const float4 *node = rec + kApetreiRecord * (int64_t)k;
    const float4 a = node[0], b = node[1], c = node[2];
    const int l = __float_as_int(c.x), r = __float_as_int(c.y);
    const int lc = __float_as_int(a.w), rc = __float_as_int(b.w);
    bool ok = l >= 0 && r < n && l <= k && k < r;
    if (ok) {
        ok = lc == (l == k ? ni + k : lc) && rc == (r == k + 1 ? ni + k + 1 : rc);
        if (ok && l != k) {  // internal left child: must cover [l, k]
            ok = lc >= 0 && lc < ni && __float_as_int(rec[kApetreiRecord * (int64_t)lc + 2].x) == l &&
                 __float_as_int(rec[kApetreiRecord * (int64_t)lc + 2].y) == k;
        }
        if (ok && r != k + 1) {  // internal right child: must cover [k+1, r]
            ok = rc >= 0 && rc < ni && __float_as_int(rec[kApetreiRecord * (int64_t)rc + 2].x) == k + 1 &&
                 __float_as_int(rec[kApetreiRecord * (int64_t)rc + 2].y) == r;
        }
    }
    if (!ok) {
        atomicOr(flags, kFlagCorrupt);
        return;
    }
    const int q = delta_gap(codes, n, r) < delta_gap(codes, n, l - 1) ? r : l;
    const int left = l == k ? ni + k : k;
    inodes[2 * (int64_t)q] = make_float4(a.x, a.y, a.z, __int_as_float(left));
    inodes[2 * (int64_t)q + 1] = make_float4(b.x, b.y, b.z, __int_as_float(node_skip(codes, n, r)));
}

unsigned blocks_for(int64_t n) { return (unsigned)((n + kThreads - 1) / kThreads); }

}  // namespace

size_t variant_scratch_bytes(int64_t n, int algorithm) {
    const int64_t ni = n > 0 ? n - 1 : 0;
    if (algorithm == LBVH_BUILD_KARRAS) return (size_t)(3 * ni + 2 * n) * 4 + 16;
    if (algorithm == LBVH_BUILD_APETREI) return (size_t)ni * kApetreiRecord * 16 + 16;
    return 0;
}

void launch_variant_hierarchy(int algorithm, const uint64_t *codes, const uint32_t *perm, const float *prims,
                              int64_t n, int kind, float4 *inodes, float4 *leaves, void *scratch,
                              unsigned long long *store, uint32_t *flags, cudaStream_t s) {
    if (n <= 0) return;
    const int ni = (int)n - 1;
    if (algorithm == LBVH_BUILD_KARRAS) {
        if (n < 2) return;
        int32_t *left = static_cast<int32_t *>(scratch);
        karras_nodes_kernel<<<blocks_for(ni), kThreads, 0, s>>>(codes, (int)n, left, left + ni, left + 2 * ni,
                                                                 left + 3 * ni, flags);
    } else {
        float4 *rec = static_cast<float4 *>(scratch);
        if (kind == LBVH_PRIM_POINTS)
            apetrei_kernel<LBVH_PRIM_POINTS><<<blocks_for(n), kThreads, 0, s>>>(codes, perm, prims, (int)n, rec,
                                                                                leaves, store, flags);
        else
            apetrei_kernel<LBVH_PRIM_BOXES><<<blocks_for(n), kThreads, 0, s>>>(codes, perm, prims, (int)n, rec,
                                                                               leaves, store, flags);
    }
    (void)inodes;
    count_launches(1);
}

void launch_variant_second(int algorithm, const uint64_t *codes, const uint32_t *perm, const float *prims,
                           int64_t n, int kind, float4 *inodes, float4 *leaves, void *scratch,
                           unsigned long long *store, uint32_t *flags, cudaStream_t s) {
    if (n <= 0) return;
    const int ni = (int)n - 1;
    if (algorithm == LBVH_BUILD_KARRAS) {
        const int32_t *left = static_cast<const int32_t *>(scratch);
        unsigned int *counters = reinterpret_cast<unsigned int *>(store);
        if (kind == LBVH_PRIM_POINTS)
            karras_boxes_kernel<LBVH_PRIM_POINTS><<<blocks_for(n), kThreads, 0, s>>>(
                codes, perm, prims, (int)n, left, left + ni, left + 2 * ni, left + 3 * ni, inodes, leaves,
                counters, flags);
        else
            karras_boxes_kernel<LBVH_PRIM_BOXES><<<blocks_for(n), kThreads, 0, s>>>(
                codes, perm, prims, (int)n, left, left + ni, left + 2 * ni, left + 3 * ni, inodes, leaves,
                counters, flags);
    } else {
        const float4 *rec = static_cast<const float4 *>(scratch);
        if (kind == LBVH_PRIM_POINTS)
            apetrei_to_karras_kernel<LBVH_PRIM_POINTS><<<blocks_for(n), kThreads, 0, s>>>(codes, perm, (int)n,
                                                                                          rec, inodes, leaves, flags);
        else
            apetrei_to_karras_kernel<LBVH_PRIM_BOXES><<<blocks_for(n), kThreads, 0, s>>>(codes, perm, (int)n,
                                                                                         rec, inodes, leaves, flags);
    }
    count_launches(1);
}

}  // namespace lbvh
