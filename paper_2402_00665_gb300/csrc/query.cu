// query.cu -- stackless range queries (Algorithm 1) and CSR assembly.
//
// Each thread walks the tree for one query: start at the root (id 0); when
// the predicate holds on an internal node go to its left child, on a leaf
// report it and go to its skip; when it fails go to the skip; stop at the
// sentinel. Internal nodes are two float4 (box + left, box + skip), point
// leaves one float4 (xyz + skip), so every step is one or two 16-byte loads
// through the read-only path and a few FP32 operations.
//
// Predicates (closed, FP32, fixed operation order, no fused multiply-add):
//   sphere  e_a = max(lo_a - c_a, c_a - hi_a, 0); d2 = (ex*ex + ey*ey) + ez*ez;
//           hit iff d2 <= r*r. Rounding is monotone, so a node's d2 never
//           exceeds the d2 of a primitive inside it: the walk prunes nothing
//           a brute-force scan would report.
//   box     lo_q <= hi_b and lo_b <= hi_q on every axis.
//
// CSR in three steps: a counting walk, an exclusive scan of the counts, and a
// filling walk that sorts each query's primitive ids in registers (lists of up
// to kQueryBufferHits; longer lists are written in walk order and sorted by a
// fix-up kernel, one CTA per list, with a bitonic network).
#include "lbvh_internal.cuh"

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

__device__ __forceinline__ float gap(float lo, float c, float hi) {
    return fmaxf(fmaxf(__fsub_rn(lo, c), __fsub_rn(c, hi)), 0.0f);
}

__device__ __forceinline__ bool hits(const Sphere &s, float3 lo, float3 hi) {
    const float ex = gap(lo.x, s.c.x, hi.x);
    const float ey = gap(lo.y, s.c.y, hi.y);
    const float ez = gap(lo.z, s.c.z, hi.z);
    const float d2 = __fadd_rn(__fadd_rn(__fmul_rn(ex, ex), __fmul_rn(ey, ey)), __fmul_rn(ez, ez));
    return d2 <= s.r2;
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
        const float r = a.radii ? a.radii[q] : a.radius;
        return Sphere{make_float3(p[0], p[1], p[2]), __fmul_rn(r, r)};
    }
};
template <>
struct QueryOf<LBVH_Q_BOX> {
    using type = Box;
    static __device__ __forceinline__ Box load(const QueryArgs &a, int64_t q) {
        const float *p = a.queries + 6 * q;
        return Box{make_float3(p[0], p[1], p[2]), make_float3(p[3], p[4], p[5])};
    }
};

__device__ __forceinline__ float3 xyz(float4 v) { return make_float3(v.x, v.y, v.z); }

// Algorithm 1. on_leaf(k) is called for every leaf k that satisfies the
// predicate, in increasing k. Returns false if the walk ran past 2(2n-1)
// steps or met an id outside the tree (a corrupt tree).
template <int kP, typename Q, typename F>
__device__ __forceinline__ bool walk(const TreeView &t, const Q &q, F &&on_leaf) {
    const int ni = (int)t.n - 1;
    const uint32_t nodes = 2u * (uint32_t)t.n - 1u;
    const uint32_t max_steps = 2u * nodes;
    int node = 0;
    uint32_t steps = 0;
    while (node != kSentinel) {
        if ((uint32_t)node >= nodes || ++steps > max_steps) return false;
        if (node < ni) {
            const float4 a = __ldg(t.inodes + 2 * node);
            const float4 b = __ldg(t.inodes + 2 * node + 1);
            node = hits(q, xyz(a), xyz(b)) ? __float_as_int(a.w) : __float_as_int(b.w);
        } else {
            const int k = node - ni;
            float4 a, b;
            if (kP == LBVH_PRIM_POINTS) {
                a = __ldg(t.leaves + k);
                b = a;
            } else {
                a = __ldg(t.leaves + 2 * k);
                b = __ldg(t.leaves + 2 * k + 1);
            }
            if (hits(q, xyz(a), xyz(b))) on_leaf(k);
            node = __float_as_int(a.w);
        }
    }
    return true;
}

template <int kQ, int kP>
__global__ void __launch_bounds__(kThreads)
    count_kernel(TreeView t, QueryArgs qa, uint32_t *__restrict__ counts, Control *ctl) {
    const int64_t qi = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (qi >= qa.nq) return;
    uint32_t c = 0;
    if (t.n > 0 && ctl->build_flags == 0) {
        const auto q = QueryOf<kQ>::load(qa, qi);
        if (!walk<kP>(t, q, [&](int) { ++c; })) atomicOr(&ctl->query_flags, kFlagCorrupt);
    }
    counts[qi] = c;
}

// Keeps buf[0..K) ascending: x moves in from the front, the largest value
// falls off the end (a padding value while fewer than K hits were inserted).
template <int K>
__device__ __forceinline__ void insert_sorted(uint32_t (&buf)[K], uint32_t x) {
#pragma unroll
    for (int j = 0; j < K; ++j) {
        const uint32_t lo = min(buf[j], x);
        x = max(buf[j], x);
        buf[j] = lo;
    }
}

template <int kQ, int kP>
__global__ void __launch_bounds__(kThreads)
    fill_kernel(TreeView t, QueryArgs qa, const int64_t *__restrict__ offsets,
                uint32_t *__restrict__ hits_out, uint32_t *__restrict__ overflow_list,
                Control *ctl) {
    const int64_t qi = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (qi >= qa.nq) return;
    const int64_t base = offsets[qi];
    const int64_t count = offsets[qi + 1] - base;
    if (count == 0) return;
    const auto q = QueryOf<kQ>::load(qa, qi);
    uint32_t *out = hits_out + base;
    if (count <= kQueryBufferHits) {
        uint32_t buf[kQueryBufferHits];
#pragma unroll
        for (int j = 0; j < kQueryBufferHits; ++j) buf[j] = 0xffffffffu;
        walk<kP>(t, q, [&](int k) { insert_sorted(buf, __ldg(t.perm + k)); });
#pragma unroll
        for (int j = 0; j < kQueryBufferHits; ++j)
            if (j < count) out[j] = buf[j];
    } else {
        int64_t c = 0;
        walk<kP>(t, q, [&](int k) {
            if (c < count) out[c] = __ldg(t.perm + k);
            ++c;
        });
        const uint32_t slot = atomicAdd(&ctl->overflow_filled, 1u);
        overflow_list[slot] = (uint32_t)qi;
    }
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
    scan_reduce_kernel(const uint32_t *__restrict__ counts, int64_t nq, int64_t *tile_sums,
                       uint32_t *overflow_expected) {
    __shared__ int64_t s_warp[kScanThreads / 32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    int64_t sum = 0;
    uint32_t big = 0;
    for (int j = 0; j < kScanItems; ++j) {
        const int64_t i = base + j * kScanThreads + threadIdx.x;
        if (i < nq) {
            const uint32_t c = counts[i];
            sum += c;
            big += c > (uint32_t)kQueryBufferHits;
        }
    }
    int64_t total;
    block_scan_exclusive(sum, s_warp, total);
    for (int off = 16; off > 0; off >>= 1) big += __shfl_xor_sync(0xffffffffu, big, off);
    if ((threadIdx.x & 31) == 0 && big) atomicAdd(overflow_expected, big);
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

__global__ void __launch_bounds__(kScanThreads)
    scan_apply_kernel(const uint32_t *__restrict__ counts, int64_t nq,
                      const int64_t *__restrict__ tile_sums, int64_t *__restrict__ offsets) {
    __shared__ int64_t s_warp[kScanThreads / 32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    // thread t owns kScanItems consecutive counts
    uint32_t c[kScanItems];
    int64_t sum = 0;
    const int64_t first = base + (int64_t)threadIdx.x * kScanItems;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        const int64_t i = first + j;
        c[j] = i < nq ? counts[i] : 0u;
        sum += c[j];
    }
    int64_t total;
    int64_t run = tile_sums[blockIdx.x] + block_scan_exclusive(sum, s_warp, total);
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        const int64_t i = first + j;
        if (i < nq) offsets[i] = run;
        run += c[j];
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

__global__ void __launch_bounds__(kFixThreads)
    sort_lists_kernel(const int64_t *__restrict__ offsets, uint32_t *hits,
                      const uint32_t *__restrict__ list) {
    __shared__ uint32_t s[kFixSmem];
    const uint32_t q = list[blockIdx.x];
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
}

template <int kQ, int kP>
void launch_count_t(const TreeView &t, const QueryArgs &q, uint32_t *counts, Control *ctl,
                    cudaStream_t s) {
    const unsigned blocks = (unsigned)((q.nq + kThreads - 1) / kThreads);
    count_kernel<kQ, kP><<<blocks, kThreads, 0, s>>>(t, q, counts, ctl);
    count_launches(1);
}

template <int kQ, int kP>
void launch_fill_t(const TreeView &t, const QueryArgs &q, const int64_t *offsets,
                   uint32_t *hits, uint32_t *overflow_list, Control *ctl, cudaStream_t s) {
    const unsigned blocks = (unsigned)((q.nq + kThreads - 1) / kThreads);
    fill_kernel<kQ, kP><<<blocks, kThreads, 0, s>>>(t, q, offsets, hits, overflow_list, ctl);
    count_launches(1);
}

}  // namespace

void launch_query_count(const TreeView &t, const QueryArgs &q, uint32_t *counts, Control *ctl,
                        cudaStream_t s) {
    if (q.nq <= 0) return;
    if (q.qkind == LBVH_Q_SPHERE) {
        if (t.kind == LBVH_PRIM_POINTS)
            launch_count_t<LBVH_Q_SPHERE, LBVH_PRIM_POINTS>(t, q, counts, ctl, s);
        else
            launch_count_t<LBVH_Q_SPHERE, LBVH_PRIM_BOXES>(t, q, counts, ctl, s);
    } else {
        if (t.kind == LBVH_PRIM_POINTS)
            launch_count_t<LBVH_Q_BOX, LBVH_PRIM_POINTS>(t, q, counts, ctl, s);
        else
            launch_count_t<LBVH_Q_BOX, LBVH_PRIM_BOXES>(t, q, counts, ctl, s);
    }
}

void launch_query_fill(const TreeView &t, const QueryArgs &q, const int64_t *offsets,
                       uint32_t *hits, uint32_t *overflow_list, Control *ctl, cudaStream_t s) {
    if (q.nq <= 0) return;
    if (q.qkind == LBVH_Q_SPHERE) {
        if (t.kind == LBVH_PRIM_POINTS)
            launch_fill_t<LBVH_Q_SPHERE, LBVH_PRIM_POINTS>(t, q, offsets, hits, overflow_list, ctl, s);
        else
            launch_fill_t<LBVH_Q_SPHERE, LBVH_PRIM_BOXES>(t, q, offsets, hits, overflow_list, ctl, s);
    } else {
        if (t.kind == LBVH_PRIM_POINTS)
            launch_fill_t<LBVH_Q_BOX, LBVH_PRIM_POINTS>(t, q, offsets, hits, overflow_list, ctl, s);
        else
            launch_fill_t<LBVH_Q_BOX, LBVH_PRIM_BOXES>(t, q, offsets, hits, overflow_list, ctl, s);
    }
}

int64_t scan_tile_count(int64_t nq) { return (nq + kScanTile - 1) / kScanTile; }

void launch_exclusive_scan(const uint32_t *counts, int64_t nq, int64_t *offsets,
                           int64_t *tile_sums, Control *ctl, cudaStream_t s) {
    const int64_t tiles = scan_tile_count(nq);
    if (tiles > 0)
        scan_reduce_kernel<<<(unsigned)tiles, kScanThreads, 0, s>>>(counts, nq, tile_sums,
                                                                  &ctl->overflow_expected);
    scan_tiles_kernel<<<1, kScanThreads, 0, s>>>(tile_sums, tiles, offsets, nq, &ctl->total);
    if (tiles > 0)
        scan_apply_kernel<<<(unsigned)tiles, kScanThreads, 0, s>>>(counts, nq, tile_sums, offsets);
    count_launches(tiles > 0 ? 3 : 1);
}

void launch_sort_overflow(const int64_t *offsets, uint32_t *hits, const uint32_t *overflow_list,
                          uint32_t count, cudaStream_t s) {
    if (count == 0) return;
    sort_lists_kernel<<<count, kFixThreads, 0, s>>>(offsets, hits, overflow_list);
    count_launches(1);
}

}  // namespace lbvh
