// morton.cu -- scene bounds and Morton codes (Sec. 3.1, Karras step 1).
//
// The paper leaves the encoding open. The one used here:
//   centroid    a point itself; a box (lo + hi) * 0.5 in FP32
//   bounds      per-axis min / max of the centroids (exact FP32 compares,
//               -0.0 ordered below +0.0)
//   quantise    t = (c - min) / (max - min), IEEE FP32 subtract and divide;
//               v = t * 2^b (exact); cell = 0 if !(v > 0), 2^b - 1 if
//               v >= 2^b - 1, else trunc(v); cell = 0 on an axis of zero extent
//   interleave  bit 3k+2 = x_k, 3k+1 = y_k, 3k = z_k
// Every float operation is an explicit round-to-nearest intrinsic so the
// compiler cannot contract or reassociate them.
//
// Both kernels stream the primitives once. Points are read as float4 (three
// float4 = four points per thread step) when the array is 16-byte aligned.
// The encoder also accumulates the global digit histograms of every radix-sort
// pass (shared-memory counters, flushed once per block), which saves the sort
// a separate read of the codes.
#include <cfloat>

#include "lbvh_internal.cuh"

namespace lbvh {

namespace {

constexpr int kThreads = 256;

// Mask of the bit positions that input bit k occupies after the spreading
// steps of levels >= L: bit k has moved up by 2 * (k with its low L bits
// cleared). At level 0 every bit k sits at 3k.
constexpr uint64_t spread_mask(int level) {
    uint64_t m = 0;
    for (int k = 0; k < 21; ++k) m |= 1ull << (k + 2 * (k & ~((1 << level) - 1)));
    return m;
}

// Moves bit k of a 21-bit value to bit 3k.
__device__ __forceinline__ uint64_t spread3(uint32_t v) {
    uint64_t x = v & 0x1fffffu;
    x = (x | (x << 32)) & spread_mask(4);
    x = (x | (x << 16)) & spread_mask(3);
    x = (x | (x << 8)) & spread_mask(2);
    x = (x | (x << 4)) & spread_mask(1);
    x = (x | (x << 2)) & spread_mask(0);
    return x;
}

struct Grid3 {
    float lo[3];
    float extent[3];
    float cells;  // 2^b
    float top;    // 2^b - 1
    uint32_t topi;
};

__device__ __forceinline__ uint32_t cell_of(float c, float lo, float extent, const Grid3 &g) {
    if (!(extent > 0.0f)) return 0u;
    const float t = __fdiv_rn(__fsub_rn(c, lo), extent);
    const float v = __fmul_rn(t, g.cells);
    if (!(v > 0.0f)) return 0u;
    if (v >= g.top) return g.topi;
    return __float2uint_rz(v);
}

__device__ __forceinline__ uint64_t morton(float x, float y, float z, const Grid3 &g) {
    const uint32_t qx = cell_of(x, g.lo[0], g.extent[0], g);
    const uint32_t qy = cell_of(y, g.lo[1], g.extent[1], g);
    const uint32_t qz = cell_of(z, g.lo[2], g.extent[2], g);
    return (spread3(qx) << 2) | (spread3(qy) << 1) | spread3(qz);
}

__device__ __forceinline__ bool finite3(float x, float y, float z) {
    return fabsf(x) <= FLT_MAX && fabsf(y) <= FLT_MAX && fabsf(z) <= FLT_MAX;
}

__device__ __forceinline__ void box_centroid(const float *b, float &x, float &y, float &z) {
    x = __fmul_rn(__fadd_rn(b[0], b[3]), 0.5f);
    y = __fmul_rn(__fadd_rn(b[1], b[4]), 0.5f);
    z = __fmul_rn(__fadd_rn(b[2], b[5]), 0.5f);
}

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

template <int kKind, typename K>
__global__ void __launch_bounds__(kThreads)
    encode_kernel(const float *__restrict__ prims, int64_t n, int b,
                  const float *__restrict__ bounds, K *__restrict__ codes,
                  uint32_t *__restrict__ hist, int passes) {
    __shared__ uint32_t s_hist[kMaxPasses * kRadix];
    for (int k = threadIdx.x; k < passes * kRadix; k += kThreads) s_hist[k] = 0;
    Grid3 g;
    for (int a = 0; a < 3; ++a) {
        g.lo[a] = bounds[a];
        g.extent[a] = __fsub_rn(bounds[3 + a], bounds[a]);
    }
    g.topi = (1u << b) - 1u;
    g.cells = (float)(1u << b);
    g.top = (float)g.topi;
    __syncthreads();
    for_each_centroid<kKind>(prims, n, [&](int64_t i, float x, float y, float z) {
        const uint64_t c = morton(x, y, z, g);
        codes[i] = (K)c;
        for (int p = 0; p < passes; ++p)
            atomicAdd(&s_hist[p * kRadix + (uint32_t)((c >> (kRadixBits * p)) & (kRadix - 1))], 1u);
    });
    __syncthreads();
    for (int k = threadIdx.x; k < passes * kRadix; k += kThreads) {
        const uint32_t v = s_hist[k];
        if (v) atomicAdd(&hist[k], v);
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
    Grid3 g;
    const float *bd = bounds + 6 * (int64_t)c.inst;
    for (int a = 0; a < 3; ++a) {
        g.lo[a] = bd[a];
        g.extent[a] = __fsub_rn(bd[3 + a], bd[a]);
    }
    g.topi = (1u << b) - 1u;
    g.cells = (float)(1u << b);
    g.top = (float)g.topi;
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

template <typename K>
static void encode_as(const float *prims, int64_t n, int kind, int bits, const float *bounds, K *codes,
                      uint32_t *hist, int hist_passes, cudaStream_t s) {
    const int blocks = bounds_blocks(n);
    const int b = bits / 3;
    if (kind == LBVH_PRIM_POINTS)
        encode_kernel<LBVH_PRIM_POINTS, K><<<blocks, kThreads, 0, s>>>(prims, n, b, bounds, codes, hist,
                                                                       hist_passes);
    else
        encode_kernel<LBVH_PRIM_BOXES, K><<<blocks, kThreads, 0, s>>>(prims, n, b, bounds, codes, hist,
                                                                      hist_passes);
    count_launches(1);
}

void launch_encode(const float *prims, int64_t n, int kind, int bits, const float *bounds,
                   uint64_t *codes, uint32_t *hist, int hist_passes, cudaStream_t s) {
    encode_as(prims, n, kind, bits, bounds, codes, hist, hist_passes, s);
}

void launch_encode(const float *prims, int64_t n, int kind, int bits, const float *bounds,
                   uint32_t *codes, uint32_t *hist, int hist_passes, cudaStream_t s) {
    encode_as(prims, n, kind, bits, bounds, codes, hist, hist_passes, s);
}

}  // namespace lbvh
