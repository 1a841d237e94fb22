// morton.cuh -- the Morton code of a centroid (Sec. 3.1, Karras step 1), as
// device functions shared by the encoder and by the construct, which derives
// each leaf's code again from the primitive it gathers. Both must compute the
// same bits, so both call these functions.
//
// The paper leaves the encoding open. The one used here:
//   centroid    a point itself; a box (lo + hi) * 0.5 in FP32
//   quantise    t = (c - min) / (max - min), IEEE FP32 subtract and divide;
//               v = t * 2^b (exact); cell = 0 if !(v > 0), 2^b - 1 if
//               v >= 2^b - 1, else trunc(v); cell = 0 on an axis of zero extent
//   interleave  bit 3k+2 = x_k, 3k+1 = y_k, 3k = z_k
// Every float operation is an explicit round-to-nearest intrinsic so the
// compiler cannot contract or reassociate them.
#pragma once

#include <cfloat>
#include <cstdint>

namespace lbvh {

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

// The quantisation grid: scene bounds and 2^b cells per axis.
struct Grid3 {
    float lo[3];
    float extent[3];
    float cells;  // 2^b
    float top;    // 2^b - 1
    uint32_t topi;
};

// bounds: float[6] {min.xyz, max.xyz}; b = code bits / 3.
__device__ __forceinline__ Grid3 make_grid(const float *bounds, int b) {
    Grid3 g;
    for (int a = 0; a < 3; ++a) {
        g.lo[a] = bounds[a];
        g.extent[a] = __fsub_rn(bounds[3 + a], bounds[a]);
    }
    g.topi = (1u << b) - 1u;
    g.cells = (float)(1u << b);
    g.top = (float)g.topi;
    return g;
}

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

}  // namespace lbvh
