// runs.cu -- the sort of a build's Morton codes wider than 32 bits
// (Sec. 3.1, Karras step 2), in two steps.
//
// 1. run_top_sort (sort.cu) sorts words top << ib | index, where
//    ib = ceil(log2 n) and top = code >> (ib - 1) holds all of the code but
//    its low ib - 1 bits: 64 - ib key bits travel in one 8-byte word with the
//    index, so every pass moves 8 bytes each way, and the passes cover the
//    key bits only (5 passes at n = 2^25 and 63-bit codes, against 8 passes
//    over the whole code; 4 when the tuner has the passes start one byte
//    higher). The words come out ordered by their bits from the run shift
//    rs up (rs = ib, or the first sorted bit when a byte is skipped), and in
//    index order where those are equal.
// 2. Words whose sorted bits are shared with a neighbour ("members": the runs
//    of equal word >> rs, each over consecutive positions) are not yet in
//    code order. Runs are disjoint, so each is put in order on its own: the
//    full codes of its elements are derived again from their primitives, and
//    inside a run the order by (code, index) is the order of the 64-bit keys
//    (code's low rs - 1 bits) << ib | index, all distinct.
//
// Uniform points at n = 2^25 with 63-bit codes have about 2,000 members in
// runs of 2 or 3 (rs = ib = 25), or 0.8% of the points (rs = 32); the
// Gaussian-mixture boxes 16% in runs of 2 to 7; equal codes make long runs.
//
//   runs_kernel       one pass over the sorted words: perm[j] = the index in
//                     word j for every position outside a run, and the list
//                     of the runs' first positions.
//   short_runs_kernel a thread per listed run: a run of at most kShortRun
//                     elements sorted in place, a longer one listed.
//   long_runs_kernel  a CTA per listed long run: up to kLongRun elements
//                     sorted in shared memory; a longer run raises the
//                     fallback.
//   fallback          only after a run longer than kLongRun (all kernels read
//                     the decision on the device and leave at once
//                     otherwise): the full codes of all elements with their
//                     indices, a stable key + payload sort of them
//                     (run_counted_sort), and the permutation copied out.
#include "lbvh_internal.cuh"
#include "morton.cuh"

namespace lbvh {

namespace {

constexpr int kThreads = 256;
constexpr int kPer = 8;          // consecutive positions per thread
constexpr int kShortRun = 16;    // runs sorted by one thread
constexpr int kLongRun = 4096;   // runs sorted by one CTA in shared memory

template <int kKind>
__device__ __forceinline__ uint64_t code_of(const float *prims, uint32_t i, const Grid3 &g) {
    float x, y, z;
    if (kKind == LBVH_PRIM_POINTS) {
        x = prims[3 * (int64_t)i];
        y = prims[3 * (int64_t)i + 1];
        z = prims[3 * (int64_t)i + 2];
    } else {
        box_centroid(prims + 6 * (int64_t)i, x, y, z);
    }
    return morton(x, y, z, g);
}

// The in-run key of the primitive with index idx: the code bits below the
// sorted ones (its low rs - 1 bits, rs the run shift) above the index.
template <int kKind>
__device__ __forceinline__ uint64_t run_key(const float *prims, uint32_t idx, const Grid3 &g, int ib, int rs) {
    const uint64_t low = code_of<kKind>(prims, idx, g) & ((1ull << (rs - 1)) - 1ull);
    return low << ib | idx;
}

// A CTA covers kThreads * kPer consecutive positions, each thread kPer of
// them: it writes the permutation at every position outside a run and lists
// the first position of every run it holds (warp-aggregated appends). The
// runs are ordered by short_runs_kernel, so that this pass, which every
// element goes through, keeps no gathers or barriers waiting on them (with
// runs in 0.8% of the positions, nearly every CTA holds one).
__global__ void __launch_bounds__(kThreads)
    runs_kernel(const uint64_t *__restrict__ words, int64_t n, int ib, int rs, uint32_t *__restrict__ perm,
                uint32_t *__restrict__ run_list, uint32_t *run_count, int64_t run_cap, uint32_t *flags) {
    constexpr int kSpan = kThreads * kPer;
    // the CTA's words, loaded across the CTA (position p at p + p / kPer: one
    // padding word per thread's row keeps a thread's reads of its own row
    // free of bank conflicts)
    __shared__ uint64_t s_word[kSpan + kThreads];
    const int64_t cta0 = (int64_t)blockIdx.x * kSpan;
    const int64_t p0 = cta0 + (int64_t)threadIdx.x * kPer;
    const uint32_t imask = (uint32_t)((1ull << ib) - 1ull);
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
        const int p = j * kThreads + threadIdx.x;
        s_word[p + p / kPer] = cta0 + p < n ? words[cta0 + p] : 0ull;
    }
    __syncthreads();
    uint64_t w[kPer];
#pragma unroll
    for (int k = 0; k < kPer; ++k) w[k] = s_word[threadIdx.x * (kPer + 1) + k];
    uint32_t member = 0, head = 0;  // bit k: position p0 + k is in a run / starts one
    if (p0 < n) {
        // the last word of the previous thread's row (its padding word follows it)
        const uint64_t left = threadIdx.x > 0 ? s_word[threadIdx.x * (kPer + 1) - 2] : (p0 > 0 ? words[p0 - 1] : 0ull);
        const uint64_t right = threadIdx.x + 1 < kThreads ? s_word[(threadIdx.x + 1) * (kPer + 1)]
                                                          : (p0 + kPer < n ? words[p0 + kPer] : 0ull);
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            const int64_t p = p0 + k;
            const uint64_t top = w[k] >> rs;
            const bool eq_prev = p > 0 && ((k > 0 ? w[k - 1] : left) >> rs) == top;
            const bool eq_next = p + 1 < n && ((k + 1 < kPer ? w[k + 1] : right) >> rs) == top;
            if (p < n && (eq_prev || eq_next)) member |= 1u << k;
            if (p < n && !eq_prev && eq_next) head |= 1u << k;
        }
        // positions outside runs: the index as it stands
        if (member == 0 && p0 + kPer <= n) {
            uint4 *o = reinterpret_cast<uint4 *>(perm + p0);
#pragma unroll
            for (int k = 0; k < kPer / 4; ++k)
                o[k] = make_uint4((uint32_t)w[4 * k] & imask, (uint32_t)w[4 * k + 1] & imask,
                                  (uint32_t)w[4 * k + 2] & imask, (uint32_t)w[4 * k + 3] & imask);
        } else {
#pragma unroll
            for (int k = 0; k < kPer; ++k)
                if (p0 + k < n && !(member & (1u << k))) perm[p0 + k] = (uint32_t)w[k] & imask;
        }
    }
    // list the run heads: one atomic per warp that holds any
    const int lane = threadIdx.x & 31;
    const uint32_t mine = (uint32_t)__popc(head);
    uint32_t incl = mine;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += y;
    }
    const uint32_t warp_total = __shfl_sync(0xffffffffu, incl, 31);
    if (warp_total == 0) return;
    uint32_t base = 0;
    if (lane == 31) base = atomicAdd(run_count, warp_total);
    base = __shfl_sync(0xffffffffu, base, 31) + incl - mine;
    for (int k = 0; k < kPer; ++k) {
        if (!(head & (1u << k))) continue;
        if ((int64_t)base < run_cap) run_list[base] = (uint32_t)(p0 + k);
        else atomicOr(flags, kFlagCorrupt);  // more runs than positions allow
        ++base;
    }
}

// One thread per listed run (a fixed grid strides over the list, whose
// length is known on the device): the run's length from the sorted words,
// then a run of at most kShortRun elements is put in code order in place:
// the in-run keys of its elements (their primitives gathered, the codes
// derived again) sorted by insertion; a longer run is listed for
// long_runs_kernel.
template <int kKind>
__global__ void __launch_bounds__(kThreads)
    short_runs_kernel(const uint64_t *__restrict__ words, int64_t n, int ib, int rs, const float *__restrict__ prims,
                      const float *__restrict__ bounds, int b, uint32_t *__restrict__ perm,
                      const uint32_t *__restrict__ run_list, const uint32_t *run_count, int64_t run_cap,
                      uint32_t *__restrict__ long_list, uint32_t *long_count, uint32_t *flags) {
    const int64_t count = min((int64_t)*run_count, run_cap);
    const uint32_t imask = (uint32_t)((1ull << ib) - 1ull);
    const Grid3 g = make_grid(bounds, b);
    for (int64_t r = (int64_t)blockIdx.x * kThreads + threadIdx.x; r < count; r += (int64_t)gridDim.x * kThreads) {
        const int64_t s = run_list[r];
        if (s >= n) {  // a corrupt list entry
            atomicOr(flags, kFlagCorrupt);
            continue;
        }
        const uint64_t top = words[s] >> rs;
        int len = 1;
        while (len <= kShortRun && s + len < n && (words[s + len] >> rs) == top) ++len;
        if (len > kShortRun) {
            const uint32_t slot = atomicAdd(long_count, 1u);
            if ((int64_t)slot < n / (kShortRun + 1) + 1) long_list[slot] = (uint32_t)s;
            else atomicOr(flags, kFlagCorrupt);  // more long runs than positions allow
            continue;
        }
        uint64_t key[kShortRun];
        for (int i = 0; i < len; ++i) {
            const uint32_t idx = (uint32_t)words[s + i] & imask;
            key[i] = 0ull;
            if ((int64_t)idx < n) key[i] = run_key<kKind>(prims, idx, g, ib, rs);
            else atomicOr(flags, kFlagCorrupt);  // only after a timed-out pass
        }
        for (int i = 1; i < len; ++i) {  // insertion sort: runs are short
            const uint64_t v = key[i];
            int j = i - 1;
            while (j >= 0 && key[j] > v) {
                key[j + 1] = key[j];
                --j;
            }
            key[j + 1] = v;
        }
        for (int i = 0; i < len; ++i) perm[s + i] = (uint32_t)key[i] & imask;
    }
}

// A CTA per listed run (grid-stride over the list): the run's length, then
// its keys sorted in shared memory by a bitonic network over the next power
// of two (padded with all-ones keys, which sort last). A run longer than
// kLongRun raises *fallback instead.
template <int kKind>
__global__ void __launch_bounds__(kThreads)
    long_runs_kernel(const uint64_t *__restrict__ words, int64_t n, int ib, int rs, const float *__restrict__ prims,
                     const float *__restrict__ bounds, int b, uint32_t *__restrict__ perm,
                     const uint32_t *__restrict__ long_list, const uint32_t *long_count, uint32_t *fallback,
                     uint32_t *flags) {
    __shared__ uint64_t key[kLongRun];
    __shared__ int s_len;
    const int64_t count = min((int64_t)*long_count, n / (kShortRun + 1) + 1);
    const uint32_t imask = (uint32_t)((1ull << ib) - 1ull);
    const Grid3 g = make_grid(bounds, b);
    for (int64_t r = blockIdx.x; r < count; r += gridDim.x) {
        const int64_t s = long_list[r];
        if (s >= n) {  // a corrupt list entry
            if (threadIdx.x == 0) atomicOr(flags, kFlagCorrupt);
            continue;
        }
        const uint64_t top = words[s] >> rs;
        if (threadIdx.x == 0) s_len = kLongRun + 1;
        __syncthreads();
        // the run's end: the first position after s whose top differs
        for (int off = 1; off <= kLongRun; off += kThreads) {
            const int o = off + (int)threadIdx.x;
            const bool end = o <= kLongRun && (s + o >= n || (words[s + o] >> rs) != top);
            if (end) atomicMin(&s_len, o);
            if (__syncthreads_or(end)) break;
        }
        const int len = s_len;
        if (len > kLongRun) {
            if (threadIdx.x == 0) atomicOr(fallback, 1u);
            __syncthreads();  // s_len is rewritten for the next run
            continue;
        }
        int pow2 = 1;
        while (pow2 < len) pow2 <<= 1;
        for (int i = threadIdx.x; i < pow2; i += kThreads) {
            uint64_t k = ~0ull;
            if (i < len) {
                const uint32_t idx = (uint32_t)words[s + i] & imask;
                if ((int64_t)idx < n) k = run_key<kKind>(prims, idx, g, ib, rs);
                else atomicOr(flags, kFlagCorrupt);  // only after a timed-out pass
            }
            key[i] = k;
        }
        __syncthreads();
        for (int size = 2; size <= pow2; size <<= 1)
            for (int stride = size >> 1; stride > 0; stride >>= 1) {
                for (int i = threadIdx.x; i < pow2; i += kThreads) {
                    const int j = i ^ stride;
                    if (j > i) {
                        const uint64_t a = key[i], c = key[j];
                        const bool ascending = (i & size) == 0;
                        if ((a > c) == ascending) {
                            key[i] = c;
                            key[j] = a;
                        }
                    }
                }
                __syncthreads();
            }
        for (int i = threadIdx.x; i < len; i += kThreads) perm[s + i] = (uint32_t)key[i] & imask;
        __syncthreads();  // key and s_len are rewritten for the next run
    }
}

// Fallback, first step: every element's full code and index (the words'
// order is (top, index), so a stable sort by code leaves equal codes in
// index order), and the count the sort reads.
template <int kKind>
__global__ void __launch_bounds__(kThreads)
    fallback_keys_kernel(const uint64_t *__restrict__ words, int64_t n, int ib, const float *__restrict__ prims,
                         const float *__restrict__ bounds, int b, uint64_t *__restrict__ codes,
                         uint32_t *__restrict__ index, const uint32_t *fallback, uint32_t *count, uint32_t *flags) {
    if (*fallback == 0) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) *count = (uint32_t)n;
    const uint32_t imask = (uint32_t)((1ull << ib) - 1ull);
    const Grid3 g = make_grid(bounds, b);
    for (int64_t j = (int64_t)blockIdx.x * kThreads + threadIdx.x; j < n; j += (int64_t)gridDim.x * kThreads) {
        uint32_t idx = (uint32_t)words[j] & imask;
        if ((int64_t)idx >= n) {  // only after a timed-out pass
            atomicOr(flags, kFlagCorrupt);
            idx = 0;
        }
        codes[j] = code_of<kKind>(prims, idx, g);
        index[j] = idx;
    }
}

// Fallback, last step: the sorted indices are the permutation.
__global__ void __launch_bounds__(kThreads)
    fallback_copy_kernel(const uint32_t *__restrict__ index, int64_t n, uint32_t *__restrict__ perm,
                         const uint32_t *fallback) {
    if (*fallback == 0) return;
    for (int64_t j = (int64_t)blockIdx.x * kThreads + threadIdx.x; j < n; j += (int64_t)gridDim.x * kThreads)
        perm[j] = index[j];
}

}  // namespace

int64_t code_sort_scratch_words(int64_t n) { return n + (n / (kShortRun + 1) + 1) + (n / 2 + 1); }

uint32_t *run_code_sort(const float *prims, int kind, int bits, const float *bounds, int64_t n, uint64_t *keys_a,
                        uint64_t *keys_b, uint32_t *vals_a, uint32_t *vals_b, uint32_t *scratch,
                        const SortScratch &sc, Control *ctl, cudaStream_t s, cudaEvent_t (*pass_events)[2],
                        cudaEvent_t *runs_events, int variant_idx, int skip) {
    if (n <= 0) return vals_a;
    const int ib = top_index_bits(n);
    const int rs = top_run_shift(ib, skip);
    uint64_t *words = run_top_sort(keys_a, keys_b, n, ib, skip, sc, ctl, s, pass_events, variant_idx);
    uint64_t *codes = words == keys_a ? keys_b : keys_a;
    uint32_t *perm = vals_a, *index_alt = scratch, *long_list = scratch + n;
    uint32_t *run_list = long_list + (n / (kShortRun + 1) + 1);  // each run has two elements or more
    const int64_t run_cap = n / 2 + 1;
    if (runs_events) cudaEventRecord(runs_events[0], s);
    const bool points = kind == LBVH_PRIM_POINTS;
    const int b = bits / 3;
    // long-run count, fallback flag, fallback sort count, run count
    cudaMemsetAsync(&ctl->run_long, 0, 4 * sizeof(uint32_t), s);
    const int64_t blocks = (n + (int64_t)kThreads * kPer - 1) / ((int64_t)kThreads * kPer);
    runs_kernel<<<(unsigned)blocks, kThreads, 0, s>>>(words, n, ib, rs, perm, run_list, &ctl->run_heads, run_cap,
                                                     &ctl->build_flags);
    const int sms = device_sm_count();
    (points ? short_runs_kernel<LBVH_PRIM_POINTS> : short_runs_kernel<LBVH_PRIM_BOXES>)<<<sms * 8, kThreads, 0, s>>>(
        words, n, ib, rs, prims, bounds, b, perm, run_list, &ctl->run_heads, run_cap, long_list, &ctl->run_long,
        &ctl->build_flags);
    (points ? long_runs_kernel<LBVH_PRIM_POINTS> : long_runs_kernel<LBVH_PRIM_BOXES>)<<<sms * 2, kThreads, 0, s>>>(
        words, n, ib, rs, prims, bounds, b, perm, long_list, &ctl->run_long, &ctl->run_fallback,
        &ctl->build_flags);
    // the fallback (each kernel leaves at once unless a run was too long)
    (points ? fallback_keys_kernel<LBVH_PRIM_POINTS> : fallback_keys_kernel<LBVH_PRIM_BOXES>)<<<sms * 4, kThreads, 0,
                                                                                               s>>>(
        words, n, ib, prims, bounds, b, codes, vals_b, &ctl->run_fallback, &ctl->run_sort_count, &ctl->build_flags);
    count_launches(4);
    cudaMemsetAsync(sc.hist, 0, (size_t)kMaxPasses * kRadix * sizeof(uint32_t), s);
    launch_digit_histogram_counted(codes, n, &ctl->run_sort_count, sc.hist, s);
    const bool in_b = run_counted_sort(codes, vals_b, words, index_alt, &ctl->run_sort_count, n, bits, sc, ctl, s);
    fallback_copy_kernel<<<sms * 4, kThreads, 0, s>>>(in_b ? index_alt : vals_b, n, perm, &ctl->run_fallback);
    count_launches(1);
    if (runs_events) cudaEventRecord(runs_events[1], s);
    return perm;
}

}  // namespace lbvh
