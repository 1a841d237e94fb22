// sort.cu -- stable LSD radix sort of 64-bit keys with 32-bit payloads
// (Sec. 3.1, Karras step 2: sort the Morton codes; the payload is the
// primitive index, so equal codes keep index order).
//
// One kernel launch per 8-bit digit ("onesweep"): the global digit counts of
// a pass are known when it starts (pass 0's from the Morton encoder or from
// digit_histogram_kernel; pass p+1's counted by pass p as it reads the keys),
// so each pass reads and writes the data once.
// Per pass, each CTA takes a tile (256 threads x 8-16 keys) by ticket (so every tile it may
// wait on is already running), ranks the keys by digit inside the tile with
// warp match/ballot counting, publishes its per-digit counts, resolves the
// exclusive prefix of its digits over all earlier tiles by decoupled look-back
// with a bounded spin, stages the tile in shared memory in digit order and
// writes it out so that consecutive threads write consecutive addresses.
//
// The same kernel also sorts many independent segments at once (batches of
// trees): tiles then never straddle two segments, and each segment has its own
// digit counts and look-back chain, so keys carry no segment bits.
//
// Look-back words: bits 31:30 = state (0 none, 1 aggregate, 2 inclusive
// prefix), bits 29:0 = count. Two regions alternate between passes; every
// tile clears its word block in the other region for the next pass.
#include <atomic>
#include <cstdlib>

#include "lbvh_internal.cuh"

namespace lbvh {

namespace {

constexpr int kWarps = kSortThreads / 32;
constexpr uint32_t kStateAgg = 1u << 30;
constexpr uint32_t kStatePrefix = 2u << 30;
constexpr uint32_t kStateMask = 3u << 30;
constexpr uint32_t kCountMask = (1u << 30) - 1u;
// A look-back wait gives up after about one second (%globaltimer), or after
// 2^26 polls whatever the clock says.
constexpr uint64_t kWaitNs = 1000000000ull;
constexpr uint32_t kSpinLimit = 1u << 26;

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed(uint32_t *p, uint32_t v) {
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Exclusive scan of one value per thread over the 256 threads of the block.
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t *s_warp) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
    for (int off = 1; off < 32; off <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, off);
        if (lane >= off) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    uint32_t before = 0;
    for (int w = 0; w < warp; ++w) before += s_warp[w];
    __syncthreads();
    return before + x - v;
}

template <int kItems, typename K = uint64_t>
struct SortSmem {
    static constexpr int kTile = kSortThreads * kItems;
    uint32_t warp_hist[kWarps][kRadix];  // per-warp digit counts, then per-warp offsets
    int32_t out_base[kRadix];            // global position of the digit's first staged key, minus its tile start
    uint32_t tile_start[kRadix];         // first staged slot of each digit
    uint32_t scan[kWarps];
    uint32_t tile;
    int32_t seg;                         // segment of the tile (segmented sorts)
    uint32_t next_hist[kRadix];          // digit counts of the next pass
    K keys[kTile];
    uint32_t vals[kTile];
};

// Lanes of the warp whose digit equals d: match.any, or eight ballots (one
// per digit bit).
template <bool kBallot>
__device__ __forceinline__ uint32_t digit_peers(uint32_t d) {
    if (!kBallot) return __match_any_sync(0xffffffffu, d);
    uint32_t peers = 0xffffffffu;
#pragma unroll
    for (int b = 0; b < kRadixBits; ++b) {
        const uint32_t bit = (d >> b) & 1u;
        const uint32_t vote = __ballot_sync(0xffffffffu, bit);
        peers &= bit ? vote : ~vote;
    }
    return peers;
}

struct SegArgs {
    const int64_t *off, *tile_first;
    int count;
};

// kSeg: segments are sorted independently. A tile then lies inside one
// segment; its keys start at off[seg] + (tile - tile_first[seg]) * kTile, its
// digit counts come from and go to the segment's rows of the histograms, and
// its look-back chain ends at the segment's first tile.
template <bool kIota, int kItems, int kMinBlocks, bool kBallot, bool kSeg, typename K = uint64_t>
__global__ void __launch_bounds__(kSortThreads, kMinBlocks)
    onesweep_kernel(const K *__restrict__ keys_in, const uint32_t *__restrict__ vals_in,
                    K *__restrict__ keys_out, uint32_t *__restrict__ vals_out, int64_t n,
                    int shift, const uint32_t *__restrict__ pass_hist, uint32_t *lookback,
                    uint32_t *lookback_next, uint32_t *ticket, int64_t tiles,
                    uint32_t *flags, uint32_t *next_hist, SegArgs seg, int64_t hold_tile,
                    int64_t prefetch_ahead) {
    using Smem = SortSmem<kItems, K>;
    constexpr int kTile = Smem::kTile;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem &sm = *reinterpret_cast<Smem *>(smem_raw);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    if (threadIdx.x == 0) {
        const uint32_t t = atomicAdd(ticket, 1u);
        if (t == tiles - 1) *ticket = 0;  // last ticket handed out: reset for the next pass
        sm.tile = t;
        if (kSeg) sm.seg = instance_of(seg.tile_first, seg.count, t);
    }
    for (int k = threadIdx.x; k < kWarps * kRadix; k += kSortThreads) (&sm.warp_hist[0][0])[k] = 0;
    sm.next_hist[threadIdx.x] = 0;
    __syncthreads();
    const int64_t tile = sm.tile;
    int64_t first_tile = 0, seg_begin = 0, seg_end = n, tile_base = tile * kTile;
    if (kSeg) {
        const int sg = sm.seg;
        first_tile = seg.tile_first[sg];
        seg_begin = seg.off[sg];
        seg_end = seg.off[sg + 1];
        tile_base = seg_begin + (tile - first_tile) * kTile;
        pass_hist += (int64_t)sg * kRadix;
        if (next_hist) next_hist += (int64_t)sg * kRadix;
    }
    const int64_t valid = min((int64_t)kTile, seg_end - tile_base);
    // warm L2 with the tile a CTA will take about one wave from now (its
    // keys and payloads are contiguous: one bulk prefetch each)
    if (!kSeg && threadIdx.x == 0 && prefetch_ahead > 0) {
        const int64_t ft = tile + prefetch_ahead;
        if (ft < tiles) {
            const int64_t fb = ft * kTile;
            const int64_t fcnt = min((int64_t)kTile, n - fb);
            const uint32_t kbytes = (uint32_t)((fcnt * (int64_t)sizeof(K)) & ~15ll);  // rounded down: stays inside
            if (kbytes) asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(keys_in + fb), "r"(kbytes) : "memory");
            if (!kIota) {
                const uint32_t vbytes = (uint32_t)((fcnt * 4) & ~15ll);
                if (vbytes) asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(vals_in + fb), "r"(vbytes)
                             : "memory");
            }
        }
    }

    // ---- load: warp w owns keys [w*32*kItems, (w+1)*32*kItems) of the tile,
    // round j lane l holds key w*32*kItems + 32*j + l
    K key[kItems];
    uint32_t val[kItems];
    uint32_t rank[kItems];
#pragma unroll
    for (int j = 0; j < kItems; ++j) {
        const int local = warp * (kItems * 32) + j * 32 + lane;
        const int64_t g = tile_base + local;
        if (local < valid) {
            key[j] = keys_in[g];
            val[j] = kIota ? (uint32_t)g : vals_in[g];
        } else {
            key[j] = ~K(0);  // ranks after every real key of digit 0xff
            val[j] = 0;
        }
    }

    // ---- digit counts for the next pass (its global histogram)
    if (next_hist) {
#pragma unroll
        for (int j = 0; j < kItems; ++j) {
            const int local = warp * (kItems * 32) + j * 32 + lane;
            if (local < valid)
                atomicAdd(&sm.next_hist[(uint32_t)(key[j] >> (shift + kRadixBits)) & (kRadix - 1)], 1u);
        }
    }

    // ---- rank inside the warp: peers with the same digit, in (round, lane) order
    const uint32_t below = lanemask_lt();
#pragma unroll
    for (int j = 0; j < kItems; ++j) {
        const uint32_t d = (uint32_t)(key[j] >> shift) & (kRadix - 1);
        const uint32_t peers = digit_peers<kBallot>(d);
        const uint32_t before = __popc(peers & below);
        const uint32_t base = sm.warp_hist[warp][d];
        __syncwarp();
        if (before == 0) sm.warp_hist[warp][d] = base + __popc(peers);
        __syncwarp();
        rank[j] = base + before;
    }
    __syncthreads();

    // ---- per digit: counts over warps, per-warp offsets, tile count
    const int d = threadIdx.x;  // kSortThreads == kRadix
    uint32_t count = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
        const uint32_t c = sm.warp_hist[w][d];
        sm.warp_hist[w][d] = count;
        count += c;
    }
    uint32_t *my_word = lookback + tile * kRadix + d;
    const bool publish = tile != hold_tile;  // a test hook: this tile's successors must time out
    if (publish) st_relaxed(my_word, (tile == first_tile ? kStatePrefix : kStateAgg) | count);

    const uint32_t global_base = (uint32_t)seg_begin + block_exclusive_scan(pass_hist[d], sm.scan);
    const uint32_t start = block_exclusive_scan(count, sm.scan);
    sm.tile_start[d] = start;

    // ---- decoupled look-back over earlier tiles for digit d
    uint32_t exclusive = 0;
    if (tile > first_tile) {
        int64_t t = tile - 1;
        while (true) {
            const uint32_t *w = lookback + t * kRadix + d;
            uint32_t v = ld_relaxed(w);
            if ((v & kStateMask) == 0) {
                const uint64_t t0 = global_ns();
                uint32_t spins = 0;
                while ((v & kStateMask) == 0) {
                    ++spins;
                    if (spins > kSpinLimit || ((spins & 1023u) == 0 && global_ns() - t0 > kWaitNs)) {
                        atomicOr(flags, kFlagTimeout);
                        v = kStatePrefix;  // give up: results are flagged invalid
                        break;
                    }
                    v = ld_relaxed(w);
                }
            }
            exclusive += v & kCountMask;
            if ((v & kStateMask) == kStatePrefix || t == first_tile) break;
            --t;
        }
        if (publish) st_relaxed(my_word, kStatePrefix | (exclusive + count));
    }
    lookback_next[tile * kRadix + d] = 0;  // the next pass's region
    sm.out_base[d] = (int32_t)(global_base + exclusive) - (int32_t)start;
    __syncthreads();

    if (next_hist) {
        const uint32_t c = sm.next_hist[threadIdx.x];
        if (c) atomicAdd(next_hist + threadIdx.x, c);
    }

    // ---- stage in digit order
#pragma unroll
    for (int j = 0; j < kItems; ++j) {
        const uint32_t dj = (uint32_t)(key[j] >> shift) & (kRadix - 1);
        const uint32_t slot = sm.tile_start[dj] + sm.warp_hist[warp][dj] + rank[j];
        sm.keys[slot] = key[j];
        sm.vals[slot] = val[j];
    }
    __syncthreads();

    // ---- write out: slot s goes to out_base[digit] + s
#pragma unroll
    for (int j = 0; j < kItems; ++j) {
        const int s = j * kSortThreads + threadIdx.x;
        if (s < valid) {
            const K k = sm.keys[s];
            const uint32_t dj = (uint32_t)(k >> shift) & (kRadix - 1);
            const int64_t pos = (int64_t)sm.out_base[dj] + s;
            if (pos < seg_begin || pos >= seg_end) {  // only after a timed-out look-back
                atomicOr(flags, kFlagCorrupt);
                continue;
            }
            keys_out[pos] = k;
            vals_out[pos] = sm.vals[s];
        }
    }
}

template <typename K>
using PassKernelT = void (*)(const K *, const uint32_t *, K *, uint32_t *, int64_t, int, const uint32_t *,
                             uint32_t *, uint32_t *, uint32_t *, int64_t, uint32_t *, uint32_t *, SegArgs,
                             int64_t, int64_t);
using PassKernel = PassKernelT<uint64_t>;

template <typename K = uint64_t>
struct VariantT {
    int items, min_blocks;
    bool ballot;
    PassKernelT<K> first, rest;          // payload = index / payload read
    PassKernelT<K> seg_first, seg_rest;  // the same, segmented
    size_t smem;
};
using Variant = VariantT<uint64_t>;

template <int kItems, int kMinBlocks, bool kBallot, typename K = uint64_t>
VariantT<K> make_variant() {
    return VariantT<K>{kItems,
                       kMinBlocks,
                       kBallot,
                       onesweep_kernel<true, kItems, kMinBlocks, kBallot, false, K>,
                       onesweep_kernel<false, kItems, kMinBlocks, kBallot, false, K>,
                       onesweep_kernel<true, kItems, kMinBlocks, kBallot, true, K>,
                       onesweep_kernel<false, kItems, kMinBlocks, kBallot, true, K>,
                       sizeof(SortSmem<kItems, K>)};
}

// Tile shapes the library is compiled with. The first entry is the default;
// LBVH_SORT_VARIANT=<index> selects another process-wide (tuning sweeps), and
// run_onesweep can be given one explicitly (the batch autotuner).
const Variant *variant_table(int *count) {
    static const Variant table[] = {
        make_variant<12, 4, true>(), make_variant<16, 3, true>(),  make_variant<8, 4, true>(),
        make_variant<16, 2, true>(), make_variant<12, 3, true>(),  make_variant<8, 6, true>(),
        make_variant<16, 2, false>(),
    };
    // kernel attributes set once, thread-safely (function-local static initialisation)
    static const bool configured = [] {
        for (const Variant &v : table) {
            for (PassKernel k : {v.first, v.rest, v.seg_first, v.seg_rest}) {
                cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)v.smem);
                cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
            }
        }
        return true;
    }();
    (void)configured;
    *count = (int)(sizeof table / sizeof table[0]);
    return table;
}

// 32-bit keys (query orders of up to 30 bits): the default tile shape only;
// its tiles hold as many keys as variant 0's, so segment tables made for
// variant 0 serve it.
const VariantT<uint32_t> &variant32() {
    static const VariantT<uint32_t> v = [] {
        const VariantT<uint32_t> w = make_variant<12, 4, true, uint32_t>();
        for (PassKernelT<uint32_t> k : {w.first, w.rest, w.seg_first, w.seg_rest}) {
            cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)w.smem);
            cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        }
        return w;
    }();
    return v;
}

const Variant &variant(int idx = -1) {
    int count = 0;
    const Variant *table = variant_table(&count);
    static const int pick = [&] {
        const char *env = getenv("LBVH_SORT_VARIANT");
        const int want = env ? atoi(env) : 0;
        return (want >= 0 && want < count) ? want : 0;
    }();
    return table[(idx >= 0 && idx < count) ? idx : pick];
}

__global__ void __launch_bounds__(256)
    digit_histogram_kernel(const uint64_t *__restrict__ keys, int64_t n, int passes,
                           uint32_t *__restrict__ hist) {
    __shared__ uint32_t s_hist[kMaxPasses * kRadix];
    for (int k = threadIdx.x; k < passes * kRadix; k += blockDim.x) s_hist[k] = 0;
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const uint64_t c = keys[i];
        for (int p = 0; p < passes; ++p)
            atomicAdd(&s_hist[p * kRadix + (uint32_t)((c >> (kRadixBits * p)) & (kRadix - 1))], 1u);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < passes * kRadix; k += blockDim.x) {
        const uint32_t v = s_hist[k];
        if (v) atomicAdd(&hist[k], v);
    }
}

}  // namespace

void launch_digit_histogram(const uint64_t *keys, int64_t n, int passes, uint32_t *hist,
                            cudaStream_t s) {
    if (n <= 0) return;
    int64_t blocks = (n + 255) / 256;
    const int64_t cap = (int64_t)device_sm_count() * 8;
    if (blocks > cap) blocks = cap;
    digit_histogram_kernel<<<(int)blocks, 256, 0, s>>>(keys, n, passes, hist);
    count_launches(1);
}

std::atomic<int64_t> g_hold_tile{-1};

void sort_set_hold_tile(int64_t tile) { g_hold_tile.store(tile, std::memory_order_relaxed); }

int64_t sort_variant_tile_keys(int idx) { return (int64_t)kSortThreads * variant(idx).items; }

int sort_variant_count() {
    int count = 0;
    variant_table(&count);
    return count;
}

int64_t sort_tile_keys_min() {
    int count = 0;
    const Variant *t = variant_table(&count);
    int items = t[0].items;
    for (int k = 1; k < count; ++k) items = t[k].items < items ? t[k].items : items;
    return (int64_t)kSortThreads * items;
}

// Tiles between a tile and the one its CTA prefetches into L2: two per SM
// (a sweep of 76..1216 at 2^25 keys: 0.313 ms per pass from 152 to 456,
// 0.327 ms without prefetch). LBVH_SORT_PREFETCH=0 turns it off, any other
// value sets the distance (tuning sweeps).
static int64_t prefetch_tiles() {
    static const int64_t env = [] {
        const char *e = getenv("LBVH_SORT_PREFETCH");
        return e ? (int64_t)atoll(e) : -1;
    }();
    if (env >= 0) return env;
    return (int64_t)device_sm_count() * 2;
}

template <typename K>
static bool run_passes(const VariantT<K> &v, K *keys_a, uint32_t *vals_a, bool iota, K *keys_b, uint32_t *vals_b,
                       int64_t n, int passes, const SortScratch &scratch, Control *ctl, cudaStream_t s,
                       cudaEvent_t (*pass_events)[2], const SortSegments *seg) {
    if (n <= 0 || passes <= 0) return false;
    const int64_t tiles = seg ? seg->tiles
                              : (n + (int64_t)kSortThreads * v.items - 1) / ((int64_t)kSortThreads * v.items);
    if (tiles <= 0) return false;
    const SegArgs sa{seg ? seg->off : nullptr, seg ? seg->tile_first : nullptr, seg ? seg->count : 0};
    const int64_t hist_stride = (int64_t)kRadix * (seg ? seg->count : 1);
    cudaMemsetAsync(scratch.lookback, 0, (size_t)tiles * kRadix * sizeof(uint32_t), s);
    K *kin = keys_a, *kout = keys_b;
    uint32_t *vin = vals_a, *vout = vals_b;
    for (int p = 0; p < passes; ++p) {
        uint32_t *cur = scratch.lookback + (p & 1) * scratch.lookback_words;
        uint32_t *nxt = scratch.lookback + ((p + 1) & 1) * scratch.lookback_words;
        const uint32_t *hist = scratch.hist + p * hist_stride;
        if (pass_events) cudaEventRecord(pass_events[p][0], s);
        PassKernelT<K> k =
            seg ? ((p == 0 && iota) ? v.seg_first : v.seg_rest) : ((p == 0 && iota) ? v.first : v.rest);
        uint32_t *next_hist = p + 1 < passes ? scratch.hist + (p + 1) * hist_stride : nullptr;
        const int64_t hold = p == 0 ? g_hold_tile.load(std::memory_order_relaxed) : -1;
        k<<<(unsigned)tiles, kSortThreads, v.smem, s>>>(kin, vin, kout, vout, n, kRadixBits * p, hist, cur,
                                                         nxt, &ctl->sort_ticket[p], tiles, &ctl->build_flags,
                                                         next_hist, sa, hold, prefetch_tiles());
        if (pass_events) cudaEventRecord(pass_events[p][1], s);
        count_launches(1);
        K *tk = kin;
        kin = kout;
        kout = tk;
        uint32_t *tv = vin;
        vin = vout;
        vout = tv;
    }
    return (passes & 1) != 0;
}

bool run_onesweep(uint64_t *keys_a, uint32_t *vals_a, bool iota, uint64_t *keys_b,
                  uint32_t *vals_b, int64_t n, int passes, const SortScratch &scratch,
                  Control *ctl, cudaStream_t s, cudaEvent_t (*pass_events)[2], int variant_idx,
                  const SortSegments *seg) {
    return run_passes(variant(variant_idx), keys_a, vals_a, iota, keys_b, vals_b, n, passes, scratch, ctl, s,
                      pass_events, seg);
}

bool run_onesweep32(uint32_t *keys_a, uint32_t *vals_a, bool iota, uint32_t *keys_b, uint32_t *vals_b,
                    int64_t n, int passes, const SortScratch &scratch, Control *ctl, cudaStream_t s,
                    const SortSegments *seg) {
    if (passes > 4) passes = 4;  // four 8-bit digits cover a 32-bit key
    return run_passes(variant32(), keys_a, vals_a, iota, keys_b, vals_b, n, passes, scratch, ctl, s, nullptr,
                      seg);
}

}  // namespace lbvh
