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
// warp ballots, publishes its per-digit counts, resolves the
// exclusive prefix of its digits over all earlier tiles by decoupled look-back
// with a bounded spin, stages the tile in shared memory in digit order and
// writes it out so that consecutive threads write consecutive addresses.
//
// Layouts of a pass. A digit is byte `db` of the 64-bit key (passes sort
// bytes db0, db0 + 1, ... in turn).
//   key + payload  uint64 keys[] and uint32 vals[] (or vals = the index)
//   packed         one uint64 word per element holding key bits above the
//                  payload: code << 32 | index for codes of at most 32 bits,
//                  or a wider code's top bits above the index (runs.cu)
// A packed pass moves 8 bytes per element each way instead of 12; the last
// pass of a packed sort may write the payloads alone (the sorted
// permutation), which is all a tree build needs (it derives each leaf's code
// again from the primitive it gathers).
//
// Two ways to launch a pass: one CTA per tile (onesweep_kernel), or a fixed
// grid of CTAs that take tiles until a count read on the device runs out
// (onesweep_counted_kernel), for a sort whose size a kernel decided.
//
// The same kernel also sorts many independent segments at once (batches of
// trees): tiles then never straddle two segments, and each segment has its own
// digit counts and look-back chain, so keys carry no segment bits.
//
// Look-back words: bits 31:30 = state (0 none, 1 aggregate, 2 inclusive
// prefix), bits 29:0 = count. Two regions alternate between passes; every
// tile clears its word block in the other region for the next pass.
#include <atomic>

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

// Input and output layouts of one pass.
enum : int { kInIota = 0, kInKV = 1, kInPacked = 2 };
enum : int { kOutKV = 0, kOutPacked = 1, kOutLow = 2 };

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

// Byte (sel & 3) of the key's low (kHi false) or high half: one byte permute.
template <bool kHi>
__device__ __forceinline__ uint32_t digit_of(uint64_t k, uint32_t sel) {
    return __byte_perm(kHi ? (uint32_t)(k >> 32) : (uint32_t)k, 0u, sel);
}

// Exclusive scans of two values per thread over the 256 threads of the
// block at once (one pair of barriers for both).
__device__ __forceinline__ void block_exclusive_scan2(uint32_t v0, uint32_t v1, uint2 *s_warp, uint32_t &e0,
                                                      uint32_t &e1) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x0 = v0, x1 = v1;
    for (int off = 1; off < 32; off <<= 1) {
        const uint32_t y0 = __shfl_up_sync(0xffffffffu, x0, off);
        const uint32_t y1 = __shfl_up_sync(0xffffffffu, x1, off);
        if (lane >= off) {
            x0 += y0;
            x1 += y1;
        }
    }
    if (lane == 31) s_warp[warp] = make_uint2(x0, x1);
    __syncthreads();
    uint32_t b0 = 0, b1 = 0;
    for (int w = 0; w < warp; ++w) {
        const uint2 s = s_warp[w];
        b0 += s.x;
        b1 += s.y;
    }
    __syncthreads();
    e0 = b0 + x0 - v0;
    e1 = b1 + x1 - v1;
}

template <int kItems, bool kVals, bool kTable>
struct SortSmem {
    static constexpr int kTile = kSortThreads * kItems;
    uint32_t warp_hist[kWarps][kRadix];  // per-warp digit counts, then per-warp offsets
    uint32_t peer_mask[kTable ? kWarps : 1][kRadix];  // table ranking: lanes of the round holding each digit (zero between rounds)
    int32_t out_base[kRadix];            // global position of the digit's first staged key, minus its tile start
    uint32_t tile_start[kRadix];         // first staged slot of each digit
    uint2 scan[kWarps];
    uint32_t tile;
    int32_t seg;                         // segment of the tile (segmented sorts)
    uint32_t next_hist[kRadix];          // digit counts of the next pass
    uint64_t keys[kTile];
    uint32_t vals[kVals ? kTile : 1];
};

// Lanes of the warp whose digit equals d: eight ballots, one per digit bit
// (faster than match.any on GB300).
__device__ __forceinline__ uint32_t digit_peers(uint32_t d) {
    uint32_t peers = 0xffffffffu;
#pragma unroll
    for (int b = 0; b < kRadixBits; ++b) {
        const uint32_t vote = __ballot_sync(0xffffffffu, (d >> b) & 1u);
        peers &= ((d >> b) & 1u) ? vote : ~vote;
    }
    return peers;
}

struct SegArgs {
    const int64_t *off, *tile_first;
    int count;
};

struct PassArgs {
    const uint64_t *keys_in;
    const uint32_t *vals_in;
    uint64_t *keys_out;
    uint32_t *vals_out;
    int64_t n;
    int db;  // digit byte
    const uint32_t *pass_hist;
    uint32_t *lookback, *lookback_next, *ticket;
    int64_t tiles;
    uint32_t *flags, *next_hist;
    SegArgs seg;
    int64_t hold_tile, prefetch_ahead;
    const uint32_t *count;  // persistent passes: the number of keys, on the device
};

// kIn / kOut: the layouts above; kHi: the digit byte lies in the key's high
// half (always for packed input). kTable: the lanes of a round that share a
// digit are found through a per-warp table in shared memory (each lane ORs
// its bit into its digit's word and reads the word back) instead of eight
// ballots. kSeg: segments are sorted independently. A
// tile then lies inside one segment; its keys start at off[seg] + (tile -
// tile_first[seg]) * kTile, its digit counts come from and go to the
// segment's rows of the histograms, and its look-back chain ends at the
// segment's first tile.
template <int kIn, int kOut, bool kHi, int kItems, int kMinBlocks, bool kTable, bool kSeg>
__device__ __forceinline__ void sweep_tile(const PassArgs &a, SortSmem<kItems, kIn != kInPacked, kTable> &sm,
                                           const int64_t tile, const int64_t n, const int64_t tiles) {
    constexpr bool kVals = kIn != kInPacked;  // a payload travels beside the key
    constexpr int kTile = SortSmem<kItems, kVals, kTable>::kTile;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t sel = 0x4440u | (uint32_t)(a.db & 3);
    const int nb = a.db + 1;  // the next pass's digit byte
    const uint32_t nsel = 0x4440u | (uint32_t)(nb & 3);
    uint32_t *next_hist = a.next_hist;
    const uint32_t *pass_hist = a.pass_hist;
    int64_t first_tile = 0, seg_begin = 0, seg_end = n, tile_base = tile * kTile;
    if (kSeg) {
        const int sg = sm.seg;
        first_tile = a.seg.tile_first[sg];
        seg_begin = a.seg.off[sg];
        seg_end = a.seg.off[sg + 1];
        tile_base = seg_begin + (tile - first_tile) * kTile;
        pass_hist += (int64_t)sg * kRadix;
        if (next_hist) next_hist += (int64_t)sg * kRadix;
    }
    const int valid = (int)min((int64_t)kTile, seg_end - tile_base);
    // warm L2 with the tile a CTA will take about one wave from now (its
    // keys and payloads are contiguous: one bulk prefetch each)
    if (!kSeg && threadIdx.x == 0 && a.prefetch_ahead > 0) {
        const int64_t ft = tile + a.prefetch_ahead;
        if (ft < tiles) {
            const int64_t fb = ft * kTile;
            const int64_t fcnt = min((int64_t)kTile, n - fb);
            const uint32_t kbytes = (uint32_t)((fcnt * 8) & ~15ll);  // rounded down: stays inside
            if (kbytes)
                asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a.keys_in + fb), "r"(kbytes)
                             : "memory");
            if (kIn == kInKV) {
                const uint32_t vbytes = (uint32_t)((fcnt * 4) & ~15ll);
                if (vbytes)
                    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a.vals_in + fb), "r"(vbytes)
                                 : "memory");
            }
        }
    }

    // ---- load: warp w owns keys [w*32*kItems, (w+1)*32*kItems) of the tile,
    // round j lane l holds key w*32*kItems + 32*j + l
    uint64_t key[kItems];
    uint32_t val[kVals ? kItems : 1];
    uint32_t rank[kItems];
    {
        const int wbase = warp * (kItems * 32) + lane;
        const uint64_t *kp = a.keys_in + tile_base + wbase;
        const uint32_t *vp = a.vals_in + tile_base + wbase;
#pragma unroll
        for (int j = 0; j < kItems; ++j) {
            const int local = wbase + j * 32;
            if (local < valid) {
                key[j] = kp[j * 32];
                if (kIn == kInKV) val[j] = vp[j * 32];
                if (kIn == kInIota) val[j] = (uint32_t)(tile_base + local);
            } else {
                key[j] = ~0ull;  // ranks after every real key of digit 0xff
                if (kVals) val[j] = 0;
            }
        }
    }

    // ---- digit counts for the next pass (its global histogram)
    if (next_hist) {
        const bool nhi = nb >= 4;
#pragma unroll
        for (int j = 0; j < kItems; ++j) {
            const int local = warp * (kItems * 32) + j * 32 + lane;
            if (local < valid) {
                const uint32_t w = nhi ? (uint32_t)(key[j] >> 32) : (uint32_t)key[j];
                atomicAdd(&sm.next_hist[__byte_perm(w, 0u, nsel)], 1u);
            }
        }
    }

    // ---- rank inside the warp: peers with the same digit, in (round, lane) order
    const uint32_t below = lanemask_lt();
#pragma unroll
    for (int j = 0; j < kItems; ++j) {
        const uint32_t d = digit_of<kHi>(key[j], sel);
        uint32_t peers;
        if (kTable) {
            atomicOr(&sm.peer_mask[warp][d], 1u << lane);
            __syncwarp();
            peers = sm.peer_mask[warp][d];
        } else {
            peers = digit_peers(d);
        }
        const uint32_t before = __popc(peers & below);
        const uint32_t base = sm.warp_hist[warp][d];
        __syncwarp();
        if (before == 0) {
            sm.warp_hist[warp][d] = base + __popc(peers);
            if (kTable) sm.peer_mask[warp][d] = 0;
        }
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
    uint32_t *my_word = a.lookback + tile * kRadix + d;
    const bool publish = tile != a.hold_tile;  // a test hook: this tile's successors must time out
    if (publish) st_relaxed(my_word, (tile == first_tile ? kStatePrefix : kStateAgg) | count);

    uint32_t hist_before, start;
    block_exclusive_scan2(pass_hist[d], count, sm.scan, hist_before, start);
    const uint32_t global_base = (uint32_t)seg_begin + hist_before;
    sm.tile_start[d] = start;

    // ---- decoupled look-back over earlier tiles for digit d
    uint32_t exclusive = 0;
    if (tile > first_tile) {
        int64_t t = tile - 1;
        while (true) {
            const uint32_t *w = a.lookback + t * kRadix + d;
            uint32_t v = ld_relaxed(w);
            if ((v & kStateMask) == 0) {
                const uint64_t t0 = global_ns();
                uint32_t spins = 0;
                while ((v & kStateMask) == 0) {
                    ++spins;
                    if (spins > kSpinLimit || ((spins & 1023u) == 0 && global_ns() - t0 > kWaitNs)) {
                        atomicOr(a.flags, kFlagTimeout);
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
    a.lookback_next[tile * kRadix + d] = 0;  // the next pass's region
    sm.out_base[d] = (int32_t)(global_base + exclusive) - (int32_t)start;
    __syncthreads();

    if (next_hist) {
        const uint32_t c = sm.next_hist[threadIdx.x];
        if (c) atomicAdd(next_hist + threadIdx.x, c);
    }

    // ---- stage in digit order
#pragma unroll
    for (int j = 0; j < kItems; ++j) {
        const uint32_t dj = digit_of<kHi>(key[j], sel);
        const uint32_t slot = sm.tile_start[dj] + sm.warp_hist[warp][dj] + rank[j];
        sm.keys[slot] = key[j];
        if (kVals) sm.vals[slot] = val[j];
    }
    __syncthreads();

    // ---- write out: slot s goes to out_base[digit] + s
    const uint32_t lo = (uint32_t)seg_begin, span = (uint32_t)(seg_end - seg_begin);
#pragma unroll
    for (int j = 0; j < kItems; ++j) {
        const int s = j * kSortThreads + threadIdx.x;
        if (s < valid) {
            const uint64_t k = sm.keys[s];
            const int32_t pos = sm.out_base[digit_of<kHi>(k, sel)] + s;
            if ((uint32_t)pos - lo >= span) {  // only after a timed-out look-back
                atomicOr(a.flags, kFlagCorrupt);
                continue;
            }
            if (kOut == kOutKV) {
                a.keys_out[pos] = k;
                a.vals_out[pos] = sm.vals[s];
            } else if (kOut == kOutPacked) {
                a.keys_out[pos] = k;
            } else if (kIn == kInPacked) {
                a.vals_out[pos] = (uint32_t)k;
            } else {
                a.vals_out[pos] = sm.vals[s];
            }
        }
    }
}

// One CTA per tile, taken by ticket (so every tile it may wait on is
// already running).
template <int kIn, int kOut, bool kHi, int kItems, int kMinBlocks, bool kTable, bool kSeg>
__global__ void __launch_bounds__(kSortThreads, kMinBlocks) onesweep_kernel(const PassArgs a) {
    using Smem = SortSmem<kItems, kIn != kInPacked, kTable>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem &sm = *reinterpret_cast<Smem *>(smem_raw);
    if (threadIdx.x == 0) {
        const uint32_t t = atomicAdd(a.ticket, 1u);
        if (t == a.tiles - 1) *a.ticket = 0;  // last ticket handed out: reset for the next pass
        sm.tile = t;
        if (kSeg) sm.seg = instance_of(a.seg.tile_first, a.seg.count, t);
    }
    for (int k = threadIdx.x; k < kWarps * kRadix; k += kSortThreads) {
        (&sm.warp_hist[0][0])[k] = 0;
        if (kTable) (&sm.peer_mask[0][0])[k] = 0;
    }
    sm.next_hist[threadIdx.x] = 0;
    __syncthreads();
    sweep_tile<kIn, kOut, kHi, kItems, kMinBlocks, kTable, kSeg>(a, sm, sm.tile, a.n, a.tiles);
}

// A fixed grid of CTAs taking tiles by ticket until the keys run out; the
// number of keys is read from the device (*a.count), so a pass can follow a
// kernel that decided it, with no host round trip. A CTA takes its next
// ticket only when it is ready to work on that tile, so every tile a CTA
// waits on is being worked on. Each CTA takes exactly one ticket past the
// last tile (and leaves), so the ticket handed out last is number
// tiles + gridDim.x - 1, whose holder resets the counter.
template <int kIn, int kOut, bool kHi, int kItems, int kMinBlocks, bool kTable>
__global__ void __launch_bounds__(kSortThreads, kMinBlocks) onesweep_counted_kernel(const PassArgs a) {
    using Smem = SortSmem<kItems, kIn != kInPacked, kTable>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem &sm = *reinterpret_cast<Smem *>(smem_raw);
    const int64_t n = min((int64_t)*a.count, a.n);  // a.n: the most the buffers hold
    const int64_t tiles = (n + Smem::kTile - 1) / Smem::kTile;
    while (true) {
        if (threadIdx.x == 0) {
            const uint32_t t = atomicAdd(a.ticket, 1u);
            if ((int64_t)t == tiles + gridDim.x - 1) *a.ticket = 0;
            sm.tile = t;
        }
        for (int k = threadIdx.x; k < kWarps * kRadix; k += kSortThreads) {
            (&sm.warp_hist[0][0])[k] = 0;
            if (kTable) (&sm.peer_mask[0][0])[k] = 0;
        }
        sm.next_hist[threadIdx.x] = 0;
        __syncthreads();
        const int64_t tile = sm.tile;
        if (tile >= tiles) return;
        sweep_tile<kIn, kOut, kHi, kItems, kMinBlocks, kTable, false>(a, sm, tile, n, tiles);
        __syncthreads();  // the tile's shared state is read before the next one clears it
    }
}

using PassKernel = void (*)(PassArgs);

// The (input, output, digit half) combinations the library runs.
enum PassKind : int {
    kIotaKV,        // pass 0 of a pair sort: payload = index
    kKVKVLo,        // key + payload in and out, digit in the low half
    kKVKVHi,        // the same, digit in the high half
    kPackedPacked,  // packed in and out
    kPackedLow,     // packed in, payloads out (the last pass)
    kPackedPackedLo,  // packed in and out, digit in the low half (words key << ib | index, ib < 32)
    kPassKinds
};

struct Variant {
    int items, min_blocks;
    bool table;
    PassKernel k[2][kPassKinds];  // [segmented][kind]
    size_t smem_kv, smem_packed;
};

template <int kItems, int kMinBlocks, bool kTable, bool kSeg>
void fill_kinds(PassKernel (&k)[kPassKinds]) {
    k[kIotaKV] = onesweep_kernel<kInIota, kOutKV, false, kItems, kMinBlocks, kTable, kSeg>;
    k[kKVKVLo] = onesweep_kernel<kInKV, kOutKV, false, kItems, kMinBlocks, kTable, kSeg>;
    k[kKVKVHi] = onesweep_kernel<kInKV, kOutKV, true, kItems, kMinBlocks, kTable, kSeg>;
    k[kPackedPacked] = onesweep_kernel<kInPacked, kOutPacked, true, kItems, kMinBlocks, kTable, kSeg>;
    k[kPackedLow] = onesweep_kernel<kInPacked, kOutLow, true, kItems, kMinBlocks, kTable, kSeg>;
    k[kPackedPackedLo] = kSeg ? nullptr : onesweep_kernel<kInPacked, kOutPacked, false, kItems, kMinBlocks, kTable, false>;
}

template <int kItems, int kMinBlocks, bool kTable>
Variant make_variant() {
    Variant v{};
    v.items = kItems;
    v.min_blocks = kMinBlocks;
    v.table = kTable;
    fill_kinds<kItems, kMinBlocks, kTable, false>(v.k[0]);
    fill_kinds<kItems, kMinBlocks, kTable, true>(v.k[1]);
    v.smem_kv = sizeof(SortSmem<kItems, true, kTable>);
    v.smem_packed = sizeof(SortSmem<kItems, false, kTable>);
    return v;
}

size_t pass_smem(const Variant &v, int kind) {
    return (kind == kPackedPacked || kind == kPackedLow || kind == kPackedPackedLo) ? v.smem_packed : v.smem_kv;
}

// Tile shapes the library is compiled with (keys per thread, CTAs per SM,
// digit peers by table or ballots). The first entry is the default; the
// autotuner may pick another.
const Variant *variant_table(int *count) {
    // Sort passes at 2^25 (ms for the 8 passes of 63-bit uniform points /
    // mixture boxes at 63 bits / the 4 passes at 30 bits; keys per thread x
    // CTAs per SM, digit peers by table or ballots): 24 x 2 table 2.10 /
    // 2.14 / 1.00; 28 x 2 table 2.11 / 2.15 / 0.98; 20 x 2 table 2.17 / 2.21
    // / 1.05; 16 x 3 table 2.17 / 2.21 / 1.03; 12 x 4 table 2.25 / 2.28 /
    // 1.07; 32 x 2 table 2.37 / 2.42 / 1.00; 10 x 5 table 2.38 / 2.41 /
    // 1.09; 12 x 4 ballots 2.39 / 2.34 / 1.08; 16 x 3 ballots 2.42 / 2.37 /
    // 1.06; 8 x 6 ballots 2.50 / 2.46 / 1.15; 8 x 6 table 2.50 / 2.53 /
    // 1.16. Larger tiles mean fewer tiles, look-back chains and barriers per
    // key; past 28 keys the key + payload passes spill.
    static const Variant table[] = {
        make_variant<24, 2, true>(),
        make_variant<28, 2, true>(),
        make_variant<16, 3, true>(),
        make_variant<12, 4, true>(),
        make_variant<12, 4, false>(),
        make_variant<16, 3, false>(),
    };
    // kernel attributes set once, thread-safely (function-local static initialisation)
    static const bool configured = [] {
        for (const Variant &v : table)
            for (int sg = 0; sg < 2; ++sg)
                for (int kind = 0; kind < kPassKinds; ++kind) {
                    if (!v.k[sg][kind]) continue;
                    cudaFuncSetAttribute(v.k[sg][kind], cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)pass_smem(v, kind));
                    cudaFuncSetAttribute(v.k[sg][kind], cudaFuncAttributePreferredSharedMemoryCarveout, 100);
                }
        return true;
    }();
    (void)configured;
    *count = (int)(sizeof table / sizeof table[0]);
    return table;
}

const Variant &variant(int idx = -1) {
    int count = 0;
    const Variant *table = variant_table(&count);
    return table[(idx >= 0 && idx < count) ? idx : 0];
}

// count (nullable): only the first *count keys (read on the device) are counted.
__global__ void __launch_bounds__(256)
    digit_histogram_kernel(const uint64_t *__restrict__ keys, int64_t n, int passes,
                           uint32_t *__restrict__ hist, const uint32_t *count) {
    if (count) n = min(n, (int64_t)*count);
    if (n == 0) return;
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
    digit_histogram_kernel<<<(int)blocks, 256, 0, s>>>(keys, n, passes, hist, nullptr);
    count_launches(1);
}

void launch_digit_histogram_counted(const uint64_t *keys, int64_t n_max, const uint32_t *count, uint32_t *hist,
                                    cudaStream_t s) {
    if (n_max <= 0) return;
    int64_t blocks = (n_max + 255) / 256;
    const int64_t cap = (int64_t)device_sm_count() * 8;
    if (blocks > cap) blocks = cap;
    digit_histogram_kernel<<<(int)blocks, 256, 0, s>>>(keys, n_max, 1, hist, count);
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
// 0.327 ms without prefetch).
static int64_t prefetch_tiles() { return (int64_t)device_sm_count() * 2; }

namespace {

// One pass: kind, digit byte, buffers.
struct Pass {
    int kind, db;
    const uint64_t *kin;
    const uint32_t *vin;
    uint64_t *kout;
    uint32_t *vout;
};

void run_pass_list(const Variant &v, const Pass *ps, int passes, int64_t n, const SortScratch &scratch,
                   Control *ctl, cudaStream_t s, cudaEvent_t (*pass_events)[2], const SortSegments *seg) {
    const int64_t tiles = seg ? seg->tiles : (n + (int64_t)kSortThreads * v.items - 1) / ((int64_t)kSortThreads * v.items);
    if (tiles <= 0) return;
    const SegArgs sa{seg ? seg->off : nullptr, seg ? seg->tile_first : nullptr, seg ? seg->count : 0};
    const int64_t hist_stride = (int64_t)kRadix * (seg ? seg->count : 1);
    cudaMemsetAsync(scratch.lookback, 0, (size_t)tiles * kRadix * sizeof(uint32_t), s);
    for (int p = 0; p < passes; ++p) {
        const Pass &q = ps[p];
        PassArgs a{};
        a.keys_in = q.kin;
        a.vals_in = q.vin;
        a.keys_out = q.kout;
        a.vals_out = q.vout;
        a.n = n;
        a.db = q.db;
        a.pass_hist = scratch.hist + p * hist_stride;
        a.lookback = scratch.lookback + (p & 1) * scratch.lookback_words;
        a.lookback_next = scratch.lookback + ((p + 1) & 1) * scratch.lookback_words;
        a.ticket = &ctl->sort_ticket[p];
        a.tiles = tiles;
        a.flags = &ctl->build_flags;
        a.next_hist = p + 1 < passes ? scratch.hist + (p + 1) * hist_stride : nullptr;
        a.seg = sa;
        a.hold_tile = p == 0 ? g_hold_tile.load(std::memory_order_relaxed) : -1;
        a.prefetch_ahead = prefetch_tiles();
        if (pass_events) cudaEventRecord(pass_events[p][0], s);
        v.k[seg ? 1 : 0][q.kind]<<<(unsigned)tiles, kSortThreads, pass_smem(v, q.kind), s>>>(a);
        if (pass_events) cudaEventRecord(pass_events[p][1], s);
        count_launches(1);
    }
}

}  // namespace

bool run_onesweep(uint64_t *keys_a, uint32_t *vals_a, bool iota, uint64_t *keys_b,
                  uint32_t *vals_b, int64_t n, int passes, const SortScratch &scratch,
                  Control *ctl, cudaStream_t s, cudaEvent_t (*pass_events)[2], int variant_idx,
                  const SortSegments *seg) {
    if (n <= 0 || passes <= 0) return false;
    Pass ps[kMaxPasses];
    uint64_t *kb[2] = {keys_a, keys_b};
    uint32_t *vb[2] = {vals_a, vals_b};
    for (int p = 0; p < passes; ++p) {
        const int in = p & 1, out = in ^ 1;
        ps[p] = Pass{(p == 0 && iota) ? kIotaKV : (p >= 4 ? kKVKVHi : kKVKVLo), p, kb[in], vb[in], kb[out], vb[out]};
    }
    run_pass_list(variant(variant_idx), ps, passes, n, scratch, ctl, s, pass_events, seg);
    return (passes & 1) != 0;
}

uint32_t *run_index_sort(uint64_t *keys_a, uint64_t *keys_b, uint32_t *vals_out, int64_t n, int key_bits,
                         const SortScratch &scratch, Control *ctl, cudaStream_t s, cudaEvent_t (*pass_events)[2],
                         int variant_idx) {
    if (n <= 0) return vals_out;
    const int passes = sort_passes(key_bits);
    Pass ps[kMaxPasses];
    uint64_t *kb[2] = {keys_a, keys_b};
    // bytes 4 .. 4 + passes - 1 of words code << 32 | index
    for (int p = 0; p < passes; ++p) {
        const int in = p & 1, out = in ^ 1;
        const bool last = p == passes - 1;
        ps[p] = Pass{last ? kPackedLow : kPackedPacked, 4 + p, kb[in], nullptr, kb[out], last ? vals_out : nullptr};
    }
    run_pass_list(variant(variant_idx), ps, passes, n, scratch, ctl, s, pass_events, nullptr);
    return vals_out;
}

uint64_t *run_top_sort(uint64_t *keys_a, uint64_t *keys_b, int64_t n, int index_bits, int skip,
                       const SortScratch &scratch, Control *ctl, cudaStream_t s, cudaEvent_t (*pass_events)[2],
                       int variant_idx) {
    if (n <= 0) return keys_a;
    const int first = top_first_byte(index_bits, skip);
    const int passes = kMaxPasses - first;
    Pass ps[kMaxPasses];
    uint64_t *kb[2] = {keys_a, keys_b};
    for (int p = 0; p < passes; ++p) {
        const int in = p & 1, out = in ^ 1;
        const int db = first + p;
        ps[p] = Pass{db < 4 ? kPackedPackedLo : kPackedPacked, db, kb[in], nullptr, kb[out], nullptr};
    }
    run_pass_list(variant(variant_idx), ps, passes, n, scratch, ctl, s, pass_events, nullptr);
    return kb[passes & 1];
}

namespace {

// The counted passes use the default tile shape (24 keys x 2 CTAs per SM,
// shared-memory table).
constexpr int kCountedItems = 24, kCountedBlocks = 2;

struct CountedKernels {
    PassKernel lo, hi;  // key + payload, digit in the low / high half
    size_t smem;
};

const CountedKernels &counted_kernels() {
    static const CountedKernels c = [] {
        CountedKernels k{};
        k.lo = onesweep_counted_kernel<kInKV, kOutKV, false, kCountedItems, kCountedBlocks, true>;
        k.hi = onesweep_counted_kernel<kInKV, kOutKV, true, kCountedItems, kCountedBlocks, true>;
        k.smem = sizeof(SortSmem<kCountedItems, true, true>);
        for (PassKernel f : {k.lo, k.hi}) {
            cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)k.smem);
            cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        }
        return k;
    }();
    return c;
}

}  // namespace

bool run_counted_sort(uint64_t *keys_a, uint32_t *vals_a, uint64_t *keys_b, uint32_t *vals_b,
                      const uint32_t *count, int64_t n_max, int key_bits, const SortScratch &scratch, Control *ctl,
                      cudaStream_t s) {
    if (n_max <= 0) return false;
    const CountedKernels &k = counted_kernels();
    const int passes = sort_passes(key_bits);
    const int64_t tile = (int64_t)kSortThreads * kCountedItems;
    const int64_t tiles_max = (n_max + tile - 1) / tile;
    int64_t grid = (int64_t)device_sm_count() * kCountedBlocks;
    if (grid > tiles_max) grid = tiles_max;
    cudaMemsetAsync(scratch.lookback, 0, (size_t)tiles_max * kRadix * sizeof(uint32_t), s);
    uint64_t *kb[2] = {keys_a, keys_b};
    uint32_t *vb[2] = {vals_a, vals_b};
    for (int p = 0; p < passes; ++p) {
        const int in = p & 1, out = in ^ 1;
        PassArgs a{};
        a.keys_in = kb[in];
        a.vals_in = vb[in];
        a.keys_out = kb[out];
        a.vals_out = vb[out];
        a.n = n_max;
        a.db = p;
        a.pass_hist = scratch.hist + p * kRadix;
        a.lookback = scratch.lookback + (p & 1) * scratch.lookback_words;
        a.lookback_next = scratch.lookback + ((p + 1) & 1) * scratch.lookback_words;
        a.ticket = &ctl->sort_ticket[p];
        a.tiles = tiles_max;
        a.flags = &ctl->build_flags;
        a.next_hist = p + 1 < passes ? scratch.hist + (p + 1) * kRadix : nullptr;
        a.hold_tile = -1;
        a.prefetch_ahead = 0;
        a.count = count;
        (p < 4 ? k.lo : k.hi)<<<(unsigned)grid, kSortThreads, k.smem, s>>>(a);
        count_launches(1);
    }
    return (passes & 1) != 0;
}

}  // namespace lbvh
