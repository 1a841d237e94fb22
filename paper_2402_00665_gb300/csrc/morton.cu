// morton.cu -- scene bounds and Morton codes (Sec. 3.1, Karras step 1). The
// encoding itself (centroid, quantisation, interleave) is in morton.cuh.
//
// Both kernels stream the primitives once. Points are read as float4 (three
// float4 = four points per thread step) when the array is 16-byte aligned.
// The encoder also accumulates the global digit histograms of every radix-sort
// pass (shared-memory counters, flushed once per block), which saves the sort
// a separate read of the codes.
#include <cfloat>

#include "lbvh_internal.cuh"
#include "morton.cuh"

namespace lbvh {

namespace {

constexpr int kThreads = 256;

struct MinMax {
    float lo[3], hi[3];
    bool ok;
    __device__ void init() {
        for (int a = 0; a < 3; ++a) {
            lo[a] = FLT_MAX;
            hi[a] = -FLT_MAX;
        }
        ok = true;
    }
    __device__ __forceinline__ void add(float x, float y, float z) {
        ok = ok && finite3(x, y, z);
        lo[0] = min_ordered(lo[0], x);
        lo[1] = min_ordered(lo[1], y);
        lo[2] = min_ordered(lo[2], z);
        hi[0] = max_ordered(hi[0], x);
        hi[1] = max_ordered(hi[1], y);
        hi[2] = max_ordered(hi[2], z);
    }
};

// Visits the centroid of every primitive: f(i, x, y, z). Points go through
// float4 loads when `prims` is 16-byte aligned (4 points per step).
template <int kKind, typename F>
__device__ __forceinline__ void for_each_centroid(const float *prims, int64_t n, F &&f) {
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    if (kKind == LBVH_PRIM_POINTS) {
        const bool vec = (reinterpret_cast<uintptr_t>(prims) & 15u) == 0;
        int64_t head = 0;
        if (vec) {
            const float4 *p4 = reinterpret_cast<const float4 *>(prims);
            const int64_t groups = n / 4;
            for (int64_t g = tid; g < groups; g += stride) {
                const float4 a = p4[3 * g], b = p4[3 * g + 1], c = p4[3 * g + 2];
                f(4 * g + 0, a.x, a.y, a.z);
                f(4 * g + 1, a.w, b.x, b.y);
                f(4 * g + 2, b.z, b.w, c.x);
                f(4 * g + 3, c.y, c.z, c.w);
            }
            head = groups * 4;
        }
        for (int64_t i = head + tid; i < n; i += stride)
            f(i, prims[3 * i], prims[3 * i + 1], prims[3 * i + 2]);
    } else {
        for (int64_t i = tid; i < n; i += stride) {
            float x, y, z;
            box_centroid(prims + 6 * i, x, y, z);
            f(i, x, y, z);
        }
    }
}

template <int kKind>
__global__ void __launch_bounds__(kThreads)
    bounds_kernel(const float *__restrict__ prims, int64_t n, float *__restrict__ partials,
                  float *__restrict__ bounds, Control *__restrict__ ctl) {
    MinMax m;
    m.init();
    for_each_centroid<kKind>(prims, n, [&](int64_t, float x, float y, float z) { m.add(x, y, z); });

    // warp, then block reduction of 6 extrema and the finite flag
    __shared__ float s_v[kThreads / 32][6];
    __shared__ int s_ok[kThreads / 32];
    __shared__ bool s_last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int ok = m.ok;
    for (int off = 16; off > 0; off >>= 1) {
        for (int a = 0; a < 3; ++a) {
            m.lo[a] = min_ordered(m.lo[a], __shfl_xor_sync(0xffffffffu, m.lo[a], off));
            m.hi[a] = max_ordered(m.hi[a], __shfl_xor_sync(0xffffffffu, m.hi[a], off));
        }
        ok &= __shfl_xor_sync(0xffffffffu, ok, off);
    }
    if (lane == 0) {
        for (int a = 0; a < 3; ++a) {
            s_v[warp][a] = m.lo[a];
            s_v[warp][3 + a] = m.hi[a];
        }
        s_ok[warp] = ok;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float v[6];
        int all = 1;
        for (int k = 0; k < 6; ++k) v[k] = s_v[0][k];
        for (int w = 0; w < kThreads / 32; ++w) {
            for (int a = 0; a < 3; ++a) {
                v[a] = min_ordered(v[a], s_v[w][a]);
                v[3 + a] = max_ordered(v[3 + a], s_v[w][3 + a]);
            }
            all &= s_ok[w];
        }
        float *out = partials + 8 * (int64_t)blockIdx.x;
        for (int k = 0; k < 6; ++k) out[k] = v[k];
        out[6] = all ? 1.0f : 0.0f;
        __threadfence();
        const uint32_t ticket = atomicAdd(&ctl->bounds_ticket, 1u);
        s_last = ticket == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    // the last block folds the per-block partials, all threads in parallel
    __threadfence();
    MinMax f;
    f.init();
    int all = 1;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += kThreads) {
        const float *p = partials + 8 * (int64_t)b;
        for (int a = 0; a < 3; ++a) {
            f.lo[a] = min_ordered(f.lo[a], __ldcg(p + a));
            f.hi[a] = max_ordered(f.hi[a], __ldcg(p + 3 + a));
        }
        all &= __ldcg(p + 6) != 0.0f;
    }
    for (int off = 16; off > 0; off >>= 1) {
        for (int a = 0; a < 3; ++a) {
            f.lo[a] = min_ordered(f.lo[a], __shfl_xor_sync(0xffffffffu, f.lo[a], off));
            f.hi[a] = max_ordered(f.hi[a], __shfl_xor_sync(0xffffffffu, f.hi[a], off));
        }
        all &= __shfl_xor_sync(0xffffffffu, all, off);
    }
    __syncthreads();  // s_v / s_ok are reused
    if (lane == 0) {
        for (int a = 0; a < 3; ++a) {
            s_v[warp][a] = f.lo[a];
            s_v[warp][3 + a] = f.hi[a];
        }
        s_ok[warp] = all;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float v[6];
        int ok_all = 1;
        for (int k = 0; k < 6; ++k) v[k] = s_v[0][k];
        for (int w = 1; w < kThreads / 32; ++w) {
            for (int a = 0; a < 3; ++a) {
                v[a] = min_ordered(v[a], s_v[w][a]);
                v[3 + a] = max_ordered(v[3 + a], s_v[w][3 + a]);
            }
            ok_all &= s_ok[w];
        }
        ok_all &= s_ok[0];
        for (int k = 0; k < 6; ++k) bounds[k] = v[k];
        if (!ok_all) atomicOr(&ctl->build_flags, kFlagNonfinite);
        ctl->bounds_ticket = 0;  // ready for the next reduction
    }
}

// kLayout (CodeLayout): kCodePlain writes the code alone; kCodeLow the word
// code << 32 | index (codes of at most 32 bits, for a sort that carries the
// index in the key's low half); kCodeTop the word (code >> (ib - 1)) << ib |
// index (the code's top 64 - ib bits above the index, n <= 2^ib). The
// histograms count the bytes of the code (plain, low) or of the word from
// byte top_first_byte(ib, skip) on (top): the bytes the sort's passes take
// in turn.
template <int kKind, int kLayout>
__global__ void __launch_bounds__(kThreads)
    encode_kernel(const float *__restrict__ prims, int64_t n, int b, const float *__restrict__ bounds,
                  uint64_t *__restrict__ codes, uint32_t *__restrict__ hist, int passes, int ib, int skip) {
    __shared__ uint32_t s_hist[kMaxPasses * kRadix];
    for (int k = threadIdx.x; k < passes * kRadix; k += kThreads) s_hist[k] = 0;
    const Grid3 g = make_grid(bounds, b);
    const int hist_shift = kLayout == kCodeTop ? kRadixBits * top_first_byte(ib, skip) : 0;
    __syncthreads();
    for_each_centroid<kKind>(prims, n, [&](int64_t i, float x, float y, float z) {
        const uint64_t c = morton(x, y, z, g);
        const uint64_t w = kLayout == kCodeTop   ? ((c >> (ib - 1)) << ib) | (uint64_t)(uint32_t)i
                           : kLayout == kCodeLow ? (c << 32) | (uint64_t)(uint32_t)i
                                                 : c;
        codes[i] = w;
        const uint64_t h = kLayout == kCodeTop ? w >> hist_shift : c;
        for (int p = 0; p < passes; ++p)
            atomicAdd(&s_hist[p * kRadix + (uint32_t)((h >> (kRadixBits * p)) & (kRadix - 1))], 1u);
    });
    __syncthreads();
    for (int k = threadIdx.x; k < passes * kRadix; k += kThreads) {
        const uint32_t v = s_hist[k];
        if (v) atomicAdd(&hist[k], v);
    }
}

// The codes of the primitives in sorted order: codes[i] = the code of
// primitive perm[i] (a gather through the permutation and the same encoding).
template <int kKind>
__global__ void __launch_bounds__(kThreads)
    sorted_codes_kernel(const float *__restrict__ prims, const uint32_t *__restrict__ perm, int64_t n, int b,
                        const float *__restrict__ bounds, uint64_t *__restrict__ codes) {
    const Grid3 g = make_grid(bounds, b);
    for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads) {
        const int64_t p = perm[i];
        float x, y, z;
        if (kKind == LBVH_PRIM_POINTS) {
            x = prims[3 * p];
            y = prims[3 * p + 1];
            z = prims[3 * p + 2];
        } else {
            box_centroid(prims + 6 * p, x, y, z);
        }
        codes[i] = morton(x, y, z, g);
    }
}

// ---- batches: one CTA per chunk of one instance

template <int kKind>
__device__ __forceinline__ void centroid_at(const float *prims, int64_t i, float &x, float &y, float &z) {
    if (kKind == LBVH_PRIM_POINTS) {
        x = prims[3 * i];
        y = prims[3 * i + 1];
        z = prims[3 * i + 2];
    } else {
        box_centroid(prims + 6 * i, x, y, z);
    }
}

template <int kKind>
__global__ void __launch_bounds__(kThreads)
    batch_bounds_kernel(const float *__restrict__ prims, const BatchChunk *__restrict__ chunks,
                        float *__restrict__ partials) {
    const BatchChunk c = chunks[blockIdx.x];
    MinMax m;
    m.init();
    for (int64_t i = c.begin + threadIdx.x; i < c.end; i += kThreads) {
        float x, y, z;
        centroid_at<kKind>(prims, i, x, y, z);
        m.add(x, y, z);
    }
    __shared__ float s_v[kThreads / 32][6];
    __shared__ int s_ok[kThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int ok = m.ok;
    for (int off = 16; off > 0; off >>= 1) {
        for (int a = 0; a < 3; ++a) {
            m.lo[a] = min_ordered(m.lo[a], __shfl_xor_sync(0xffffffffu, m.lo[a], off));
            m.hi[a] = max_ordered(m.hi[a], __shfl_xor_sync(0xffffffffu, m.hi[a], off));
        }
        ok &= __shfl_xor_sync(0xffffffffu, ok, off);
    }
    if (lane == 0) {
        for (int a = 0; a < 3; ++a) {
            s_v[warp][a] = m.lo[a];
            s_v[warp][3 + a] = m.hi[a];
        }
        s_ok[warp] = ok;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float v[6];
        int all = 1;
        for (int k = 0; k < 6; ++k) v[k] = s_v[0][k];
        for (int w = 0; w < kThreads / 32; ++w) {
            for (int a = 0; a < 3; ++a) {
                v[a] = min_ordered(v[a], s_v[w][a]);
                v[3 + a] = max_ordered(v[3 + a], s_v[w][3 + a]);
            }
            all &= s_ok[w];
        }
        float *out = partials + 8 * (int64_t)blockIdx.x;
        for (int k = 0; k < 6; ++k) out[k] = v[k];
        out[6] = all ? 1.0f : 0.0f;
    }
}

__global__ void __launch_bounds__(kThreads)
    batch_bounds_fold_kernel(const float *__restrict__ partials, const int64_t *__restrict__ chunk_first,
                             int count, float *__restrict__ bounds, Control *ctl) {
    const int b = blockIdx.x * kThreads + threadIdx.x;
    if (b >= count) return;
    float v[6] = {FLT_MAX, FLT_MAX, FLT_MAX, -FLT_MAX, -FLT_MAX, -FLT_MAX};
    int all = 1;
    for (int64_t c = chunk_first[b]; c < chunk_first[b + 1]; ++c) {
        const float *p = partials + 8 * c;
        for (int a = 0; a < 3; ++a) {
            v[a] = min_ordered(v[a], p[a]);
            v[3 + a] = max_ordered(v[3 + a], p[3 + a]);
        }
        all &= p[6] != 0.0f;
    }
    for (int k = 0; k < 6; ++k) bounds[6 * (int64_t)b + k] = v[k];
    if (!all) atomicOr(&ctl->build_flags, kFlagNonfinite);
}

template <int kKind>
__global__ void __launch_bounds__(kThreads)
    batch_encode_kernel(const float *__restrict__ data, const BatchChunk *__restrict__ chunks, int b,
                        const float *__restrict__ bounds, uint64_t *__restrict__ keys,
                        uint32_t *__restrict__ hist) {
    __shared__ uint32_t s_hist[kRadix];
    s_hist[threadIdx.x] = 0;  // kThreads == kRadix
    const BatchChunk c = chunks[blockIdx.x];
    const Grid3 g = make_grid(bounds + 6 * (int64_t)c.inst, b);
    __syncthreads();
    for (int64_t i = c.begin + threadIdx.x; i < c.end; i += kThreads) {
        float x, y, z;
        centroid_at<kKind>(data, i, x, y, z);
        const uint64_t key = morton(x, y, z, g);
        keys[i] = key;
        atomicAdd(&s_hist[(uint32_t)key & (kRadix - 1)], 1u);
    }
    __syncthreads();
    const uint32_t v = s_hist[threadIdx.x];
    if (v) atomicAdd(&hist[(int64_t)c.inst * kRadix + threadIdx.x], v);
}

}  // namespace

void launch_batch_bounds(const float *prims, int kind, const BatchTables &bt, float *partials,
                         float *bounds, Control *ctl, cudaStream_t s) {
    if (bt.nchunks <= 0) return;
    if (kind == LBVH_PRIM_POINTS)
        batch_bounds_kernel<LBVH_PRIM_POINTS><<<(unsigned)bt.nchunks, kThreads, 0, s>>>(prims, bt.chunks, partials);
    else
        batch_bounds_kernel<LBVH_PRIM_BOXES><<<(unsigned)bt.nchunks, kThreads, 0, s>>>(prims, bt.chunks, partials);
    batch_bounds_fold_kernel<<<(unsigned)((bt.count + kThreads - 1) / kThreads), kThreads, 0, s>>>(
        partials, bt.chunk_first, bt.count, bounds, ctl);
    count_launches(2);
}

void launch_batch_encode(const float *data, int kind, bool queries, const BatchTables &bt, int bits,
                         const float *bounds, uint64_t *keys, uint32_t *hist, cudaStream_t s) {
    const int64_t nchunks = queries ? bt.nqchunks : bt.nchunks;
    const BatchChunk *chunks = queries ? bt.qchunks : bt.chunks;
    if (nchunks <= 0) return;
    const int b = bits / 3;
    if (kind == LBVH_PRIM_POINTS)
        batch_encode_kernel<LBVH_PRIM_POINTS><<<(unsigned)nchunks, kThreads, 0, s>>>(data, chunks, b, bounds,
                                                                                     keys, hist);
    else
        batch_encode_kernel<LBVH_PRIM_BOXES><<<(unsigned)nchunks, kThreads, 0, s>>>(data, chunks, b, bounds,
                                                                                    keys, hist);
    count_launches(1);
}

int bounds_blocks(int64_t n) {
    const int64_t want = (n / 4 + kThreads - 1) / kThreads;
    const int64_t cap = (int64_t)device_sm_count() * 8;
    return (int)(want < 1 ? 1 : (want > cap ? cap : want));
}

void launch_bounds(const float *prims, int64_t n, int kind, float *partials, float *bounds,
                   Control *ctl, cudaStream_t s) {
    const int blocks = bounds_blocks(n);
    if (kind == LBVH_PRIM_POINTS)
        bounds_kernel<LBVH_PRIM_POINTS><<<blocks, kThreads, 0, s>>>(prims, n, partials, bounds, ctl);
    else
        bounds_kernel<LBVH_PRIM_BOXES><<<blocks, kThreads, 0, s>>>(prims, n, partials, bounds, ctl);
    count_launches(1);
}

void launch_encode(const float *prims, int64_t n, int kind, int bits, const float *bounds,
                   uint64_t *codes, uint32_t *hist, int hist_passes, int layout, int index_bits, cudaStream_t s,
                   int skip) {
    const int blocks = bounds_blocks(n);
    const int b = bits / 3;
    using Kernel = void (*)(const float *, int64_t, int, const float *, uint64_t *, uint32_t *, int, int, int);
    static const Kernel table[2][3] = {
        {encode_kernel<LBVH_PRIM_POINTS, kCodePlain>, encode_kernel<LBVH_PRIM_POINTS, kCodeLow>,
         encode_kernel<LBVH_PRIM_POINTS, kCodeTop>},
        {encode_kernel<LBVH_PRIM_BOXES, kCodePlain>, encode_kernel<LBVH_PRIM_BOXES, kCodeLow>,
         encode_kernel<LBVH_PRIM_BOXES, kCodeTop>}};
    table[kind == LBVH_PRIM_POINTS ? 0 : 1][layout]<<<blocks, kThreads, 0, s>>>(prims, n, b, bounds, codes, hist,
                                                                               hist_passes, index_bits, skip);
    count_launches(1);
}

void launch_sorted_codes(const float *prims, const uint32_t *perm, int64_t n, int kind, int bits,
                         const float *bounds, uint64_t *codes, cudaStream_t s) {
    if (n <= 0) return;
    int64_t blocks = (n + kThreads - 1) / kThreads;
    const int64_t cap = (int64_t)device_sm_count() * 16;
    if (blocks > cap) blocks = cap;
    if (kind == LBVH_PRIM_POINTS)
        sorted_codes_kernel<LBVH_PRIM_POINTS><<<(unsigned)blocks, kThreads, 0, s>>>(prims, perm, n, bits / 3,
                                                                                    bounds, codes);
    else
        sorted_codes_kernel<LBVH_PRIM_BOXES><<<(unsigned)blocks, kThreads, 0, s>>>(prims, perm, n, bits / 3,
                                                                                   bounds, codes);
    count_launches(1);
}

}  // namespace lbvh
