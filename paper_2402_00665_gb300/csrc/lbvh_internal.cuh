// lbvh_internal.cuh -- declarations shared by the CUDA translation units of
// the library (kernels + C ABI). Not part of the public interface.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "lbvh.h"

namespace lbvh {

// ---------------------------------------------------------------- status bits
// Latched on the device during a build or query; read back with the control
// block and mapped to an lbvh_status on the host.
enum : uint32_t {
    kFlagNonfinite = 1u << 0,
    kFlagTimeout = 1u << 1,
    kFlagCorrupt = 1u << 2,
    kFlagCapacity = 1u << 3,
};

// One small device-resident block per tree: status flags, the query's hit
// total, and the ticket counters of the sort passes and the bounds reduction.
// Ticket counters are reset by the block that takes the last ticket, so they
// only need zeroing once, when the block is allocated. build_flags is cleared
// at the start of every build, the query fields at the start of every query.
struct Control {
    uint32_t build_flags;          // kFlag* latched by the last build
    uint32_t bounds_ticket;        // last-block detection of the bounds reduction
    uint32_t sort_ticket[16];      // tile tickets of each sort pass
    uint32_t query_flags;          // kFlag* latched by the last query
    uint32_t overflow_filled;      // entries of the overflow list
    unsigned long long total;      // total hits of the last query
    uint32_t overflow_big;         // overflow lists too long for one warp's sort
    uint32_t spill_used;           // spill chunks handed out by the walk
    uint32_t run_long;             // run_code_sort: runs listed for a CTA each,
    uint32_t run_fallback;         //   a run too long for one CTA was met,
    uint32_t run_sort_count;       //   elements of the fallback sort,
    uint32_t run_heads;            //   runs listed for short_runs_kernel (in this order)
    uint32_t pad[2];
};
constexpr int kQueryBufferHits = 64;  // hits kept per query by the walk

// ---------------------------------------------------------------- min / max
// FP32 min / max that order -0.0 below +0.0, so the scene bounds and the
// boxes do not depend on the order in which values are combined. Inputs are
// finite (a build with a NaN or infinity is rejected).
// On GB300 fminf / fmaxf (PTX min.f32 / max.f32) already order -0.0 below
// +0.0, whichever argument comes first (checked on the device, and pinned by
// the signed-zero parity tests against the oracle's explicit ordering), so
// each is one instruction (the explicit comparison form cost the construct
// 0.30 ms at 2^25 points: 2.12 against 1.82 ms).
__device__ __forceinline__ float min_ordered(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ float max_ordered(float a, float b) { return fmaxf(a, b); }

// ---------------------------------------------------------------- node layout
// Canonical ids: internal k -> k, leaf k -> (n-1)+k, sentinel -> -1.
// Internal node k: one 32-byte record (two float4) in `inodes`:
//   inodes[2k]      {lo.x, lo.y, lo.z, left}
//   inodes[2k + 1]  {hi.x, hi.y, hi.z, skip}
// Leaf k: the skip of a leaf is always position k+1 (Algorithm 2): L_{k+1}
// or I_{k+1}, or the sentinel for k = n-1, so it needs one bit. One word
// carries the primitive index and that bit:
//   word = perm[k] | (skip is I_{k+1} ? kLeafSkipInternal : 0)
//   points: leaves[k]      {x, y, z, word}                 (16 bytes)
//   boxes:  leaves[2k]     {lo.xyz, word}, leaves[2k+1] {hi.xyz, 0}
// left/skip/word are stored as int bits. The tree keeps both arrays in one
// allocation, leaves right after the 2(n-1) float4 of the internal nodes, so
// a node's record starts at float4 unit 2*id (internal, box leaf) or id+(n-1)
// (point leaf) of that allocation. In ids, a leaf's skip is id + 1 (L_{k+1})
// or id + 1 - (n-1) (I_{k+1}); for the last leaf id + 1 = 2n-1, one past the
// last node, which ends a walk like the sentinel.
constexpr int kSentinel = -1;
constexpr uint32_t kLeafSkipInternal = 1u << 31;
constexpr uint32_t kLeafIndexMask = kLeafSkipInternal - 1u;

inline size_t leaf_float4s(int64_t n, int kind) { return (size_t)n * (kind == LBVH_PRIM_POINTS ? 1 : 2); }

// Skip id of leaf k from its word.
__host__ __device__ __forceinline__ int leaf_skip_id(uint32_t word, int k, int n) {
    if (k == n - 1) return kSentinel;
    return (word & kLeafSkipInternal) ? k + 1 : (n - 1) + k + 1;
}

// ---------------------------------------------------------------- radix sort
constexpr int kRadixBits = 8;
constexpr int kRadix = 1 << kRadixBits;
constexpr int kSortThreads = 256;
constexpr int kMaxPasses = 8;

// 8-bit digit passes for keys of key_bits bits.
inline int sort_passes(int key_bits) { return (key_bits + kRadixBits - 1) / kRadixBits; }

struct SortScratch {
    uint32_t *hist;          // kMaxPasses * kRadix global digit counts
    uint32_t *lookback;      // 2 regions of tiles * kRadix words
    int64_t lookback_words;  // words per region
};

// Global digit histograms of the first `passes` passes (the stand-alone sort
// asks for pass 0 only; the build's encoder counts pass 0 itself). `hist`
// must be zero.
void launch_digit_histogram(const uint64_t *keys, int64_t n, int passes, uint32_t *hist,
                            cudaStream_t s);
// The first pass's digit counts of the first *count keys (count on the
// device, at most n_max).
void launch_digit_histogram_counted(const uint64_t *keys, int64_t n_max, const uint32_t *count, uint32_t *hist,
                                    cudaStream_t s);

// Independent segments sorted in one pass sequence: segment b is keys
// [off[b], off[b+1]) and is sorted on its own (tiles never straddle two
// segments, digit counts and look-back chains are per segment), so the keys
// need no segment bits. Segment b's tiles are [tile_first[b], tile_first[b+1])
// for the tile shape the sort runs with (see sort_variant_tile_keys).
// hist then holds, per pass, `count` rows of kRadix counts.
struct SortSegments {
    const int64_t *off;         // count + 1, device
    const int64_t *tile_first;  // count + 1, device
    int count;
    int64_t tiles;              // tile_first[count]
};

// Sorts (keys, vals) by the low `passes * 8` bits. keys_a/vals_a hold the
// input (with `iota` the payload is the index and vals_a's contents are
// ignored; it is still used as a ping-pong buffer); keys_b/vals_b are the
// second buffers. Returns true if the result ended in the *_b buffers.
// hist[0..256) must hold pass 0's global digit counts and the rest of hist
// must be zero (pass p counts pass p+1's digits). Region 0 of the look-back
// is cleared here with a memset.
// pass_events (nullable): an event pair per pass, recorded around its kernel.
// variant_idx: tile shape (< sort_variant_count()), or -1 for the default.
// The look-back regions must hold sort_tiles_max(n) * kRadix words each
// (seg->tiles * kRadix with segments).
// seg (nullable): sort each segment on its own; its tile table must be the
// one for variant_idx's tile shape.
bool run_onesweep(uint64_t *keys_a, uint32_t *vals_a, bool iota, uint64_t *keys_b,
                  uint32_t *vals_b, int64_t n, int passes, const SortScratch &scratch,
                  Control *ctl, cudaStream_t s, cudaEvent_t (*pass_events)[2] = nullptr,
                  int variant_idx = -1, const SortSegments *seg = nullptr);
// The sort of codes of at most 32 bits when only the permutation is needed
// (a 30-bit build, the query order): keys_a holds words code << 32 | index;
// passes sort bytes 4, 5, ... in packed 8-byte words, and the last one
// writes the indices alone to vals_out, which is returned. keys_a and keys_b
// are free again afterwards. hist and the look-back are used as by
// run_onesweep.
uint32_t *run_index_sort(uint64_t *keys_a, uint64_t *keys_b, uint32_t *vals_out, int64_t n, int key_bits,
                         const SortScratch &scratch, Control *ctl, cudaStream_t s,
                         cudaEvent_t (*pass_events)[2] = nullptr, int variant_idx = -1);
// The sort of a build's codes of more than 32 bits, first step: keys_a
// holds words (code >> (index_bits - 1)) << index_bits | index (the code's
// top 64 - index_bits bits above the index, n <= 2^index_bits), sorted on
// bytes top_first_byte(index_bits, skip) .. 7: with skip 0 from the byte
// holding the code's lowest bit in the word (the index bits inside it only
// follow the index order the words are already in), with skip 1 one byte
// (one pass) fewer. The words come out ordered by their bits from
// top_run_shift(index_bits, skip) up, and in index order where those are
// equal. Returns the buffer holding the sorted words; the other one is free.
// hist[0..256) must hold the first pass's digit counts and the rest of hist
// must be zero.
uint64_t *run_top_sort(uint64_t *keys_a, uint64_t *keys_b, int64_t n, int index_bits, int skip,
                       const SortScratch &scratch, Control *ctl, cudaStream_t s,
                       cudaEvent_t (*pass_events)[2] = nullptr, int variant_idx = -1);
// The whole sort of a build's codes of more than 32 bits (runs.cu): keys_a
// holds the encoder's kCodeTop words (index bits top_index_bits(n)); their
// top bits are sorted by run_top_sort (skip: as there), then the runs of
// equal sorted bits are put in code order (their codes derived again from
// prims with the scene bounds and bits / 3 bits per axis). Returns vals_a, which then holds the
// permutation; keys_a, keys_b, vals_b and scratch (2n words) are used on the
// way. The hist, look-back and control words as for the other sorts.
// scratch: code_sort_scratch_words(n) words.
// runs_events (nullable): an event pair around the second step.
int64_t code_sort_scratch_words(int64_t n);
uint32_t *run_code_sort(const float *prims, int kind, int bits, const float *bounds, int64_t n, uint64_t *keys_a,
                        uint64_t *keys_b, uint32_t *vals_a, uint32_t *vals_b, uint32_t *scratch,
                        const SortScratch &sc, Control *ctl, cudaStream_t s, cudaEvent_t (*pass_events)[2],
                        cudaEvent_t *runs_events, int variant_idx, int skip);
// A key + payload sort of the first *count (device) pairs, at most n_max,
// over the low key_bits bits: a fixed grid of CTAs per pass takes tiles by
// ticket up to the count it reads on the device. hist and the look-back as
// for run_onesweep (the look-back regions hold sort_tiles_max(n_max) * kRadix
// words). Returns true if the result ended in the *_b buffers.
bool run_counted_sort(uint64_t *keys_a, uint32_t *vals_a, uint64_t *keys_b, uint32_t *vals_b,
                      const uint32_t *count, int64_t n_max, int key_bits, const SortScratch &scratch, Control *ctl,
                      cudaStream_t s);
int sort_variant_count();
// A tree build's sort choice c (the tuner's index, lbvh_tree_set_tuning):
// tile shape c % sort_variant_count() and, for codes wider than 30 bits,
// skip = c / sort_variant_count() (run_top_sort sorts one byte fewer when 1).
inline int build_sort_choices() { return 2 * sort_variant_count(); }
inline int sort_choice_tile(int c) { return c < 0 ? -1 : c % sort_variant_count(); }
inline int sort_choice_skip(int c) { return c < 0 ? 0 : c / sort_variant_count(); }
// Test hook (lbvh_test_hold_sort_tile): tile `tile` of every sort's first pass
// publishes nothing, so later tiles' bounded look-back waits run out; -1: off.
void sort_set_hold_tile(int64_t tile);
// Keys per tile of variant idx (-1: the default variant).
int64_t sort_variant_tile_keys(int idx);
int64_t sort_tile_keys_min();
inline int64_t sort_tiles_max(int64_t n) { return (n + sort_tile_keys_min() - 1) / sort_tile_keys_min(); }

// ---------------------------------------------------------------- Morton
// bounds: float[6] out; partials: float[blocks * 8]; codes: uint64[n];
// hist: kMaxPasses * kRadix (accumulated; must be zero beforehand).
int bounds_blocks(int64_t n);
void launch_bounds(const float *prims, int64_t n, int kind, float *partials, float *bounds,
                   Control *ctl, cudaStream_t s);
// What the encoder writes per primitive i: the code; code << 32 | i (codes
// of at most 32 bits, run_index_sort's packed mode); or the top bits
// (code >> (ib - 1)) << ib | i for run_top_sort, ib = index_bits with
// n <= 2^ib (index_bits is read for kCodeTop only).
enum CodeLayout : int { kCodePlain = 0, kCodeLow = 1, kCodeTop = 2 };
// Index bits of the top layout for n primitives: ceil(log2 n), at least 1.
inline int top_index_bits(int64_t n) {
    int ib = 1;
    while (ib < 62 && (int64_t(1) << ib) < n) ++ib;
    return ib;
}
// The first byte run_top_sort sorts, and the run shift: the sorted words are
// ordered by their bits from the run shift up (the code's bits from
// shift - 1 up; below the shift, index order). skip 1 starts one byte
// higher, which is taken only while the in-run keys (the code's low
// shift - 1 bits above the index_bits-bit index) fit 64 bits.
__host__ __device__ inline int top_first_byte(int index_bits, int skip) {
    const int first = index_bits / kRadixBits;
    const bool ok = skip > 0 && first + 1 < kMaxPasses && kRadixBits * (first + 1) - 1 + index_bits <= 64;
    return ok ? first + 1 : first;
}
__host__ __device__ inline int top_run_shift(int index_bits, int skip) {
    const int first = top_first_byte(index_bits, skip);
    return first == index_bits / kRadixBits ? index_bits : kRadixBits * first;
}
// skip (kCodeTop): the histogram counts byte top_first_byte(index_bits, skip).
void launch_encode(const float *prims, int64_t n, int kind, int bits, const float *bounds,
                   uint64_t *codes, uint32_t *hist, int hist_passes, int layout, int index_bits, cudaStream_t s,
                   int skip = 0);
// codes[i] = the Morton code of primitive perm[i].
void launch_sorted_codes(const float *prims, const uint32_t *perm, int64_t n, int kind, int bits,
                         const float *bounds, uint64_t *codes, cudaStream_t s);

// ---------------------------------------------------------------- construct
// Algorithm 4 with boxes: writes inodes and leaves (layout above), and uses
// `store` (n-1 words, all zero on entry; left all zero on exit).
// flags: kFlagCorrupt is latched if a perm entry is out of range, adjacent
// codes are out of order, or a climb leaves the tree.
// The Karras and Apetrei hierarchy builds (variants.cu): scratch bytes, the
// hierarchy kernel, and the second pass (Karras: boxes; Apetrei: ordering and
// skips). `store` is the tree's zeroed Algorithm 4 scratch (left zeroed).
size_t variant_scratch_bytes(int64_t n, int algorithm);
void launch_variant_hierarchy(int algorithm, const uint64_t *codes, const uint32_t *perm, const float *prims,
                              int64_t n, int kind, float4 *inodes, float4 *leaves, void *scratch,
                              unsigned long long *store, uint32_t *flags, cudaStream_t s);
void launch_variant_second(int algorithm, const uint64_t *codes, const uint32_t *perm, const float *prims,
                           int64_t n, int kind, float4 *inodes, float4 *leaves, void *scratch,
                           unsigned long long *store, uint32_t *flags, cudaStream_t s);
// pend (nullable): construct_pend_bytes(n) of zeroed scratch, left zeroed.
// With it, the climbs that leave a CTA's group of leaves run in a second
// kernel with full warps instead of holding their CTA; without it (the
// no-allocation entry point) they run in place.
size_t construct_pend_bytes(int64_t n);
void launch_construct(const uint64_t *sorted_codes, const uint32_t *perm, const float *prims,
                      int64_t n, int kind, float4 *inodes, float4 *leaves,
                      unsigned long long *store, uint32_t *flags, void *pend, cudaStream_t s);
// The same pass after run_index_sort: each leaf's code is derived again from
// its gathered primitive (bounds: the build's scene bounds; bits: code bits)
// and the sorted codes are written to codes_out.
void launch_construct_encode(const uint32_t *perm, const float *prims, const float *bounds, int bits, int64_t n,
                             int kind, uint64_t *codes_out, float4 *inodes, float4 *leaves,
                             unsigned long long *store, uint32_t *flags, void *pend, cudaStream_t s);

// ---------------------------------------------------------------- query
struct TreeView {
    const float4 *inodes;
    const float4 *leaves;
    int64_t n;
    int kind;
};
struct QueryArgs {
    const float *queries;
    int64_t nq;
    int qkind;
    const float *radii;  // null: `radius` for every query
    float radius;
    const uint32_t *order;  // null: thread i walks query i; else query order[i]
    int walk = 0;           // kWalk*: how the collecting walk runs
};
// The collecting walk: one thread per query (CTAs of 256 threads, or of 512),
// or groups of 8, 16 or 32 lanes walking together (walk_group in query.cu).
enum : int {
    kWalkThread = 0,
    kWalkGroup8 = 1,
    kWalkGroup16 = 2,
    kWalkGroup32 = 3,
    kWalkThread512 = 4,
    kWalkKinds = 5
};
// A tree's walk choice c (the tuner's index, lbvh_tree_set_tuning): walk kind
// c % kWalkKinds, and the Morton bits of the query order: 30 (4 sort passes)
// for c < kWalkKinds, 24 (3 passes) above.
constexpr int kWalkChoices = 2 * kWalkKinds;
inline int walk_choice_kind(int c) { return c < 0 ? kWalkThread : c % kWalkKinds; }
inline int walk_choice_order_bits(int c) { return c >= kWalkKinds ? 24 : 30; }
// Hits past a walk's slot go to chunks of kSpillChunkWords words taken from a
// shared pool (word 0 links to the next chunk of the same walk, the rest
// hold hits). When the pool runs out, the query walks a second time instead.
constexpr int kSpillChunkWords = 64;
constexpr uint32_t kSpilledTag = 1u << 31;  // overflow-list entry whose hits are all in slot + chunks
inline uint32_t spill_chunks_for(int64_t nq) {
    const int64_t c = nq / 16;
    return (uint32_t)(c < 1024 ? 1024 : (c > (1 << 26) ? (1 << 26) : c));
}

struct QueryScratch {
    uint32_t *counts;         // nq: hits of query q
    uint32_t *slots;          // nq * kQueryBufferHits: first hits of query q, in walk order
    uint32_t *overflow_list;  // nq: queries with more hits than a slot (kSpilledTag: no second walk)
    uint32_t *spill_head;     // nq: first spill chunk of query q
    uint32_t *spill;          // spill_chunks * kSpillChunkWords
    uint32_t spill_chunks;
};
// The collecting walk (counts, short sorted lists, overflow list).
void launch_query_collect(const TreeView &t, const QueryArgs &q, const QueryScratch &qs, Control *ctl,
                          cudaStream_t s);
// k nearest neighbours of the query points q.queries (float[nq][3], q.order
// the walk order) into rows of out_idx / out_d2 (uint32 / float [nq][k]);
// codes: the tree's sorted codes (null: no seeding), bounds and bits of its
// Morton grid. k <= kKnnMaxK.
constexpr int kKnnMaxK = 256;
// Node visits of Algorithm 1 for every query (counts[0] += leaves,
// counts[1] += internal nodes; counts zeroed by the caller).
void launch_visits(const TreeView &t, const QueryArgs &q, unsigned long long *counts, Control *ctl, cudaStream_t s);
void launch_knn(const TreeView &t, const uint64_t *codes, const float *bounds, int bits, const QueryArgs &q, int k,
                uint32_t *out_idx, float *out_d2, Control *ctl, cudaStream_t s);
// offsets[0..nq] = exclusive scan of counts (offsets[nq] = total =
// ctl->total).
int64_t scan_tile_count(int64_t nq);
// offsets[0..n) += base (a chunk's CSR offsets moved to its place in the whole)
void launch_offsets_add(int64_t *offsets, int64_t n, int64_t base, cudaStream_t s);
void launch_exclusive_scan(const uint32_t *counts, int64_t nq, int64_t *offsets,
                           int64_t *tile_sums, Control *ctl, cudaStream_t s);
// Short lists from the scratch buffer to their CSR positions.
void launch_query_copy(const QueryArgs &q, const QueryScratch &qs, const int64_t *offsets,
                       uint32_t *hits, Control *ctl, cudaStream_t s);
// Second walk + sort for the `count` queries of the overflow list.
// ctl: the query's control block (overflow counts on the device).
void launch_query_overflow(const TreeView &t, const QueryArgs &q, const QueryScratch &qs,
                           uint32_t count, const int64_t *offsets, uint32_t *hits, Control *ctl,
                           cudaStream_t s);

// ---------------------------------------------------------------- batches
// Many independent trees in one pass. Instance b owns primitives
// [prim_off[b], prim_off[b+1]) of one concatenated array and queries
// [query_off[b], query_off[b+1]); its tree's records start at node_start[b]
// (float4 units of one shared node buffer, laid out as a single tree) and its
// Algorithm 4 store words at store_start[b]. Chunks split every instance into
// pieces of at most kBatchChunk primitives for the per-instance reductions.
constexpr int kBatchChunk = 8192;
struct BatchChunk {
    int64_t begin, end;
    int inst, pad;
};
struct BatchTables {
    const int64_t *prim_off;     // count + 1
    const int64_t *query_off;    // count + 1
    const int64_t *node_start;   // count
    const int64_t *store_start;  // count
    const BatchChunk *chunks;    // nchunks (primitives)
    const int64_t *chunk_first;  // count + 1: instance b's chunks are [chunk_first[b], chunk_first[b+1])
    const BatchChunk *qchunks;   // nqchunks (queries, for their Morton order)
    int count;
    int64_t total_prims, total_queries, nchunks, nqchunks;
};

// Largest b in [0, count) with off[b] <= g (the instance of element g).
__device__ __forceinline__ int instance_of(const int64_t *__restrict__ off, int count, int64_t g) {
    int lo = 0, hi = count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(off + mid) <= g) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Per-instance bounds: partials (nchunks * 8 floats), then bounds (count * 6).
void launch_batch_bounds(const float *prims, int kind, const BatchTables &bt, float *partials,
                         float *bounds, Control *ctl, cudaStream_t s);
// Morton codes of primitives (or of query centres, with `queries` = true:
// qchunks and qkind decide the layout), each in its own instance's grid, plus
// pass 0's digit histogram of every instance (hist row inst * kRadix).
void launch_batch_encode(const float *data, int kind, bool queries, const BatchTables &bt, int bits,
                         const float *bounds, uint64_t *keys, uint32_t *hist, cudaStream_t s);
void launch_batch_construct(const uint64_t *sorted_codes, const uint32_t *perm, const float *prims,
                            const BatchTables &bt, int kind, float4 *nodes, unsigned long long *store,
                            uint32_t *flags, cudaStream_t s);
// The collecting walk over all instances' queries (instance of a query found
// from query_off), and the overflow walk + list sort with device-side counts.
void launch_batch_collect(const float4 *nodes, int kind, const BatchTables &bt, const QueryArgs &q,
                          const QueryScratch &qs, Control *ctl, cudaStream_t s);
void launch_batch_overflow(const float4 *nodes, int kind, const BatchTables &bt, const QueryArgs &q,
                           const QueryScratch &qs, Control *ctl, const int64_t *offsets, uint32_t *hits,
                           unsigned long long capacity, cudaStream_t s);
// Copy with the capacity check on the device (no host round trip): lists are
// written only if ctl->total <= capacity; otherwise kFlagCapacity is latched.
void launch_query_copy_checked(const QueryArgs &q, const QueryScratch &qs, const int64_t *offsets,
                               uint32_t *hits, unsigned long long capacity, Control *ctl, cudaStream_t s);

// Used by the request server (server.cu): run a batch without graph capture;
// copy one instance of a finished batch into a tree of its own (nodes and
// bounds only: it can be queried, not exported); free a tree's query scratch
// (stream-ordered on s, after the queries that used it).
void batch_set_graphs(lbvh_batch_t b, bool on);
lbvh_status tree_from_batch(lbvh_batch_t b, int64_t instance, lbvh_tree_t t, cudaStream_t s);
void tree_release_query_scratch(lbvh_tree_t t, cudaStream_t s);

int device_sm_count();

// ---------------------------------------------------------------- autotuner (tune.cu)
// A configuration: GPU, ceil(log2 n), Morton bits, primitive kind, query kind
// (-1: the sort of a build), trees built together.
struct TuneKey {
    std::string gpu;
    int n_log2, bits, kind, qkind;
    int64_t instances;
    bool operator<(const TuneKey &o) const;
};
// sort: variant of sort.cu's table; walk: kWalk*; -1: not measured.
struct TuneChoice {
    int sort = -1, walk = -1;
    float sort_ms = 0.0f, walk_ms = 0.0f;
};
int ceil_log2(int64_t x);
std::string current_gpu_name();
TuneKey tune_key(int64_t n, int bits, int kind, int qkind, int64_t instances);
bool tune_find(const TuneKey &k, TuneChoice *out);
// Stores the fields of c that are set (>= 0), keeping the others.
void tune_put(const TuneKey &k, const TuneChoice &c);
// The cached choices for a configuration: the sort variant (-1: the default)
// and the walk (kWalkThread when nothing is cached).
int tune_sort_choice(int64_t n, int bits, int kind, int64_t instances);
int tune_walk_choice(int64_t n, int bits, int kind, int qkind, int64_t instances);

// Device memory of the library: one stream-ordered pool per device, owned by
// the library, that keeps freed blocks for reuse (its release threshold is
// never reached), so buffers that are freed and allocated again do not map
// and unmap memory at every synchronisation. lbvh_release_cached_memory
// hands the unused part back.
cudaError_t pool_alloc(void **p, size_t bytes, cudaStream_t s);
void pool_free(void *p, cudaStream_t s);
// Grows the current device's pool by `bytes` of reusable memory now (one
// allocation, freed again at once and kept by the pool).
cudaError_t pool_reserve(size_t bytes, cudaStream_t s);

// Adds k to the process-wide count of kernels launched by this library.
void count_launches(int k);

}  // namespace lbvh
