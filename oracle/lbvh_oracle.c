/*
 * lbvh_oracle.c -- CPU oracle for the linear BVH with skip connections of
 * arXiv 2402.00665 (Prokopenko & Lebrun-Grandie).
 *
 * TEST INFRASTRUCTURE ONLY: the reference that the CUDA library is checked
 * against. Only tests, the smoke check and the benchmark's CPU-baseline leg
 * load it; the product path never does. It shares no code with the CUDA path.
 *
 * Build: plain C99, -O2 -ffp-contract=off, so that every float operation is
 * one IEEE-754 single-precision operation rounded to nearest exactly as
 * written below (fused multiply-add only where fmaf is called).
 *
 * The method's result is exact: for distinct augmented keys the binary radix
 * tree is unique (Sec. 3.1), and the stackless traversal reports exactly the
 * primitives whose box satisfies the predicate (Sec. 2, Algorithm 1). So this
 * file writes out the definitions rather than re-running Algorithm 4:
 *
 *   Morton code   Sec. 3.1 step 1. The paper does not fix the encoding; the
 *                 reading used here (also used by the CUDA library, which
 *                 restates it independently) is:
 *                   centroid   point itself; box (lo + hi) * 0.5f
 *                   bounds     per-axis min/max of the centroids
 *                   quantise   t = (c - min) / (max - min) in float,
 *                              v = t * 2^b, q = clamp(trunc(v), 0, 2^b - 1);
 *                              q = 0 on an axis of zero extent
 *                   interleave bit 3k+2 = x_k, 3k+1 = y_k, 3k = z_k
 *   Sort          Sec. 3.1 step 2; ties go to the lower primitive index.
 *   delta         Sec. 3.1 defines delta(i, j) on keys m_i, m_j for
 *                 0 <= i < j < n and +infinity otherwise; Sec. 3.2 replaces
 *                 the common-prefix length by the XOR of the keys and augments
 *                 equal keys with their index. Read with XOR semantics (larger
 *                 = the keys differ at a higher bit), the index being the
 *                 sorted position. delta is the position of the highest set
 *                 bit of the 96-bit XOR of (code:64 | position:32).
 *   Topology      Sec. 3.1: node over [i, j] splits at the gap g with
 *                 delta(g, g+1) = delta(i, j); children [i, g] and [g+1, j]
 *                 get ids g and g+1 (leaf when the range is one key). Root I_0.
 *   Skips         Sec. 2 and Fig. 1: the node that follows the subtree in
 *                 pre-order, the sentinel on the right-most path.
 *   Boxes         Sec. 3.1 step 4: union of the children's boxes. Min and
 *                 max (here and in the bounds) order -0.0 below +0.0.
 *   Queries       Algorithm 1. Sphere: closed ball; squared distance from the
 *                 centre to the box, axes x, y, z accumulated in that order,
 *                 ex*ex rounded, then each further term added with one fused
 *                 multiply-add; a NaN centre coordinate or radius hits
 *                 nothing. Box: closed overlap test.
 */
#include "lbvh_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_NOMEM 3
#define ORACLE_MAX_N (1LL << 30)

/* ------------------------------------------------------------------ */
/* Morton codes (Sec. 3.1, step 1)                                     */
/* ------------------------------------------------------------------ */

int oracle_centroids(const float *prims, int64_t n, int kind, float *out) {
    if (n < 0 || (kind != ORACLE_POINTS && kind != ORACLE_BOXES)) return ORACLE_INVALID;
    for (int64_t i = 0; i < n; ++i) {
        for (int a = 0; a < 3; ++a) {
            if (kind == ORACLE_POINTS) {
                out[3 * i + a] = prims[3 * i + a];
            } else {
                float lo = prims[6 * i + a];
                float hi = prims[6 * i + 3 + a];
                float s = lo + hi;
                out[3 * i + a] = s * 0.5f;
            }
        }
    }
    return ORACLE_OK;
}

/* a < b in the total order of finite floats that puts -0.0 below +0.0
 * (the paper is silent; this makes min and max independent of the order in
 * which values are combined) */
static int is_below(float a, float b) { return a < b || (a == b && signbit(a) && !signbit(b)); }

int oracle_scene_bounds(const float *c, int64_t n, float *out) {
    if (n <= 0) return ORACLE_INVALID;
    for (int a = 0; a < 3; ++a) {
        out[a] = c[a];
        out[3 + a] = c[a];
    }
    for (int64_t i = 0; i < n; ++i) {
        for (int a = 0; a < 3; ++a) {
            float v = c[3 * i + a];
            if (!isfinite(v)) return ORACLE_NONFINITE;
            if (is_below(v, out[a])) out[a] = v;
            if (is_below(out[3 + a], v)) out[3 + a] = v;
        }
    }
    return ORACLE_OK;
}

uint32_t oracle_quantize(float c, float lo, float hi, int b) {
    const uint32_t cells = 1u << b;
    const uint32_t top = cells - 1u;
    float extent = hi - lo;
    if (!(extent > 0.0f)) return 0u; /* zero extent on this axis */
    float t = (c - lo) / extent;
    float v = t * (float)cells; /* exact: scaling by a power of two */
    if (!(v > 0.0f)) return 0u;
    if (v >= (float)top) return top;
    return (uint32_t)v; /* truncation toward zero */
}

uint64_t oracle_interleave(uint32_t qx, uint32_t qy, uint32_t qz, int b) {
    uint64_t code = 0;
    for (int k = 0; k < b; ++k) {
        code |= (uint64_t)((qx >> k) & 1u) << (3 * k + 2);
        code |= (uint64_t)((qy >> k) & 1u) << (3 * k + 1);
        code |= (uint64_t)((qz >> k) & 1u) << (3 * k);
    }
    return code;
}

static int valid_bits(int bits) { return bits >= 3 && bits <= 63 && bits % 3 == 0; }

int oracle_morton_codes(const float *prims, int64_t n, int kind, int bits,
                        uint64_t *codes, float *bounds_out) {
    if (n < 0 || n > ORACLE_MAX_N || !valid_bits(bits)) return ORACLE_INVALID;
    if (kind != ORACLE_POINTS && kind != ORACLE_BOXES) return ORACLE_INVALID;
    if (n == 0) return ORACLE_OK;
    const int b = bits / 3;
    float *c = (float *)malloc((size_t)n * 3 * sizeof(float));
    if (!c) return ORACLE_NOMEM;
    oracle_centroids(prims, n, kind, c);
    float bounds[6];
    int st = oracle_scene_bounds(c, n, bounds);
    if (st != ORACLE_OK) {
        free(c);
        return st;
    }
    for (int64_t i = 0; i < n; ++i) {
        uint32_t qx = oracle_quantize(c[3 * i + 0], bounds[0], bounds[3], b);
        uint32_t qy = oracle_quantize(c[3 * i + 1], bounds[1], bounds[4], b);
        uint32_t qz = oracle_quantize(c[3 * i + 2], bounds[2], bounds[5], b);
        codes[i] = oracle_interleave(qx, qy, qz, b);
    }
    if (bounds_out) memcpy(bounds_out, bounds, sizeof bounds);
    free(c);
    return ORACLE_OK;
}

/* ------------------------------------------------------------------ */
/* Sort (Sec. 3.1, step 2)                                             */
/* ------------------------------------------------------------------ */

typedef struct {
    uint64_t code;
    uint32_t index;
} keyed;

static int cmp_keyed(const void *pa, const void *pb) {
    const keyed *a = (const keyed *)pa, *b = (const keyed *)pb;
    if (a->code != b->code) return a->code < b->code ? -1 : 1;
    if (a->index != b->index) return a->index < b->index ? -1 : 1;
    return 0;
}

int oracle_sort_codes(const uint64_t *codes, int64_t n, uint32_t *perm, uint64_t *sorted) {
    if (n < 0 || n > ORACLE_MAX_N) return ORACLE_INVALID;
    if (n == 0) return ORACLE_OK;
    keyed *tmp = (keyed *)malloc((size_t)n * sizeof(keyed));
    if (!tmp) return ORACLE_NOMEM;
    for (int64_t i = 0; i < n; ++i) {
        tmp[i].code = codes[i];
        tmp[i].index = (uint32_t)i;
    }
    qsort(tmp, (size_t)n, sizeof(keyed), cmp_keyed);
    for (int64_t i = 0; i < n; ++i) {
        if (perm) perm[i] = tmp[i].index;
        if (sorted) sorted[i] = tmp[i].code;
    }
    free(tmp);
    return ORACLE_OK;
}

/* ------------------------------------------------------------------ */
/* delta and the Karras topology (Sec. 3.1, 3.2)                       */
/* ------------------------------------------------------------------ */

static int highest_bit(uint64_t x) { return 63 - __builtin_clzll(x); } /* x != 0 */

int32_t oracle_delta(const uint64_t *sorted, int64_t n, int64_t i, int64_t j) {
    if (!(0 <= i && i < j && j < n)) return INT32_MAX;
    uint64_t x = sorted[i] ^ sorted[j];
    if (x != 0) return 32 + highest_bit(x);
    /* equal codes: the keys differ only in the appended 32-bit position */
    return highest_bit((uint64_t)((uint32_t)i ^ (uint32_t)j));
}

int oracle_topology(const uint64_t *sorted, int64_t n, int32_t *left, int32_t *right,
                    int32_t *range_l, int32_t *range_r, int32_t *split) {
    if (n < 0 || n > ORACLE_MAX_N) return ORACLE_INVALID;
    if (n < 2) return ORACLE_OK;
    const int32_t ni = (int32_t)(n - 1); /* number of internal nodes */
    int32_t *dstar = (int32_t *)malloc((size_t)(n - 1) * sizeof(int32_t));
    int32_t *stack = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    if (!dstar || !stack) {
        free(dstar);
        free(stack);
        return ORACLE_NOMEM;
    }
    for (int64_t g = 0; g + 1 < n; ++g) dstar[g] = oracle_delta(sorted, n, g, g + 1);

    int64_t sp = 0;
    range_l[0] = 0;
    range_r[0] = (int32_t)(n - 1);
    stack[sp++] = 0;
    int status = ORACLE_OK;
    while (sp > 0) {
        const int32_t k = stack[--sp];
        const int32_t l = range_l[k], r = range_r[k];
        const int32_t d = oracle_delta(sorted, n, l, r);
        int32_t g = -1;
        for (int32_t j = l; j < r; ++j) {
            if (dstar[j] == d) {
                g = j;
                break;
            }
        }
        if (g < 0) { /* cannot happen for sorted input */
            status = ORACLE_INVALID;
            break;
        }
        split[k] = g;
        if (g == l) {
            left[k] = ni + g; /* leaf L_g */
        } else {
            left[k] = g; /* internal I_g covering [l, g] */
            range_l[g] = l;
            range_r[g] = g;
            stack[sp++] = g;
        }
        if (g + 1 == r) {
            right[k] = ni + g + 1; /* leaf L_{g+1} */
        } else {
            right[k] = g + 1; /* internal I_{g+1} covering [g+1, r] */
            range_l[g + 1] = g + 1;
            range_r[g + 1] = r;
            stack[sp++] = g + 1;
        }
    }
    free(dstar);
    free(stack);
    return status;
}

/* ------------------------------------------------------------------ */
/* Skip connections (Sec. 2, Fig. 1)                                   */
/* ------------------------------------------------------------------ */

int oracle_skips(int64_t n, const int32_t *left, const int32_t *right,
                 int32_t *skip_internal, int32_t *skip_leaf, int32_t *preorder) {
    if (n < 0 || n > ORACLE_MAX_N) return ORACLE_INVALID;
    if (n == 0) return ORACLE_OK;
    const int64_t ni = n - 1;
    int32_t *stack = (int32_t *)malloc((size_t)(n + 1) * sizeof(int32_t));
    if (!stack) return ORACLE_NOMEM;
    int64_t sp = 0, pos = 0;
    stack[sp++] = 0; /* root: I_0, or L_0 (id 0) when n == 1 */
    while (sp > 0) {
        const int32_t id = stack[--sp];
        /* whatever waits on the stack is visited right after this subtree */
        const int32_t skip = sp > 0 ? stack[sp - 1] : -1;
        if (preorder) preorder[pos] = id;
        ++pos;
        if (id < ni) {
            skip_internal[id] = skip;
            stack[sp++] = right[id];
            stack[sp++] = left[id];
        } else {
            skip_leaf[id - ni] = skip;
        }
    }
    free(stack);
    return ORACLE_OK;
}

/* ------------------------------------------------------------------ */
/* Boxes (Sec. 3.1, step 4)                                            */
/* ------------------------------------------------------------------ */

int oracle_boxes(const float *prims, int64_t n, int kind, const uint32_t *perm,
                 const int32_t *left, const int32_t *right, float *leaf_box,
                 float *internal_box) {
    if (n < 0 || n > ORACLE_MAX_N) return ORACLE_INVALID;
    if (n == 0) return ORACLE_OK;
    const int64_t ni = n - 1;
    for (int64_t k = 0; k < n; ++k) {
        const int64_t p = perm[k];
        for (int a = 0; a < 3; ++a) {
            if (kind == ORACLE_POINTS) {
                leaf_box[6 * k + a] = prims[3 * p + a];
                leaf_box[6 * k + 3 + a] = prims[3 * p + a];
            } else {
                leaf_box[6 * k + a] = prims[6 * p + a];
                leaf_box[6 * k + 3 + a] = prims[6 * p + 3 + a];
            }
        }
    }
    if (n < 2) return ORACLE_OK;
    int32_t *order = (int32_t *)malloc((size_t)(2 * n - 1) * sizeof(int32_t));
    int32_t *si = (int32_t *)malloc((size_t)ni * sizeof(int32_t));
    int32_t *sl = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    if (!order || !si || !sl) {
        free(order);
        free(si);
        free(sl);
        return ORACLE_NOMEM;
    }
    oracle_skips(n, left, right, si, sl, order);
    /* children follow their parent in pre-order: walk it backwards */
    for (int64_t t = 2 * n - 2; t >= 0; --t) {
        const int32_t id = order[t];
        if (id >= ni) continue;
        const float *bl = left[id] < ni ? internal_box + 6 * (int64_t)left[id]
                                        : leaf_box + 6 * (int64_t)(left[id] - ni);
        const float *br = right[id] < ni ? internal_box + 6 * (int64_t)right[id]
                                         : leaf_box + 6 * (int64_t)(right[id] - ni);
        float *out = internal_box + 6 * (int64_t)id;
        for (int a = 0; a < 3; ++a) {
            out[a] = is_below(br[a], bl[a]) ? br[a] : bl[a];
            out[3 + a] = is_below(bl[3 + a], br[3 + a]) ? br[3 + a] : bl[3 + a];
        }
    }
    free(order);
    free(si);
    free(sl);
    return ORACLE_OK;
}

/* ------------------------------------------------------------------ */
/* Whole build                                                          */
/* ------------------------------------------------------------------ */

int oracle_build(const float *prims, int64_t n, int kind, int bits, uint64_t *codes_out,
                 float *bounds_out, uint32_t *perm_out, uint64_t *sorted_out,
                 int32_t *left_out, int32_t *right_out, int32_t *skip_internal_out,
                 int32_t *skip_leaf_out, int32_t *range_l_out, int32_t *range_r_out,
                 int32_t *split_out, float *leaf_box_out, float *internal_box_out) {
    if (n < 0 || n > ORACLE_MAX_N || !valid_bits(bits)) return ORACLE_INVALID;
    if (kind != ORACLE_POINTS && kind != ORACLE_BOXES) return ORACLE_INVALID;
    if (n == 0) return ORACLE_OK;
    const size_t un = (size_t)n, ui = (size_t)(n - 1);
    uint64_t *codes = codes_out ? codes_out : (uint64_t *)malloc(un * 8);
    uint32_t *perm = perm_out ? perm_out : (uint32_t *)malloc(un * 4);
    uint64_t *sorted = sorted_out ? sorted_out : (uint64_t *)malloc(un * 8);
    int32_t *left = left_out ? left_out : (int32_t *)malloc(ui * 4 + 4);
    int32_t *right = right_out ? right_out : (int32_t *)malloc(ui * 4 + 4);
    int32_t *rl = range_l_out ? range_l_out : (int32_t *)malloc(ui * 4 + 4);
    int32_t *rr = range_r_out ? range_r_out : (int32_t *)malloc(ui * 4 + 4);
    int32_t *sp = split_out ? split_out : (int32_t *)malloc(ui * 4 + 4);
    int32_t *si = skip_internal_out ? skip_internal_out : (int32_t *)malloc(ui * 4 + 4);
    int32_t *sl = skip_leaf_out ? skip_leaf_out : (int32_t *)malloc(un * 4);
    float *lb = leaf_box_out ? leaf_box_out : (float *)malloc(un * 24);
    float *ib = internal_box_out ? internal_box_out : (float *)malloc(ui * 24 + 24);
    int st = ORACLE_NOMEM;
    if (codes && perm && sorted && left && right && rl && rr && sp && si && sl && lb && ib) {
        st = oracle_morton_codes(prims, n, kind, bits, codes, bounds_out);
        if (st == ORACLE_OK) st = oracle_sort_codes(codes, n, perm, sorted);
        if (st == ORACLE_OK) st = oracle_topology(sorted, n, left, right, rl, rr, sp);
        if (st == ORACLE_OK) st = oracle_skips(n, left, right, si, sl, NULL);
        if (st == ORACLE_OK) st = oracle_boxes(prims, n, kind, perm, left, right, lb, ib);
    }
    if (!codes_out) free(codes);
    if (!perm_out) free(perm);
    if (!sorted_out) free(sorted);
    if (!left_out) free(left);
    if (!right_out) free(right);
    if (!range_l_out) free(rl);
    if (!range_r_out) free(rr);
    if (!split_out) free(sp);
    if (!skip_internal_out) free(si);
    if (!skip_leaf_out) free(sl);
    if (!leaf_box_out) free(lb);
    if (!internal_box_out) free(ib);
    return st;
}

/* ------------------------------------------------------------------ */
/* Predicates and queries (Algorithm 1)                                */
/* ------------------------------------------------------------------ */

/* Closed ball against a closed box. Per axis the gap is
 * e = max(lo - c, c - hi, 0); d2 = fma(ez, ez, fma(ey, ey, ex*ex)). */
static int sphere_box_r2(const float *c, float r2, const float *box) {
    float e[3];
    for (int a = 0; a < 3; ++a) {
        if (isnan(c[a])) return 0; /* a centre with a NaN coordinate hits nothing */
        float below = box[a] - c[a];
        float above = c[a] - box[3 + a];
        e[a] = fmaxf(fmaxf(below, above), 0.0f);
    }
    /* d2 = ex*ex, then + ey*ey and + ez*ez each as one fused multiply-add
     * (a single rounding per step) */
    float d2 = e[0] * e[0];
    d2 = fmaf(e[1], e[1], d2);
    d2 = fmaf(e[2], e[2], d2);
    return d2 <= r2;
}

/* Squared distance from a point to a closed box, by the same steps as the
 * ball test above: e = max(lo - c, c - hi, 0) per axis, d2 = ex*ex, then
 * + ey*ey and + ez*ez each as one fused multiply-add. */
static float point_box_d2(const float *c, const float *box) {
    float e[3];
    for (int a = 0; a < 3; ++a) {
        float below = box[a] - c[a];
        float above = c[a] - box[3 + a];
        e[a] = fmaxf(fmaxf(below, above), 0.0f);
    }
    float d2 = e[0] * e[0];
    d2 = fmaf(e[1], e[1], d2);
    d2 = fmaf(e[2], e[2], d2);
    return d2;
}

float oracle_point_box_d2(const float *point, const float *box6) { return point_box_d2(point, box6); }

/* The k nearest primitives of each query point by brute force: every
 * primitive's squared distance (point_box_d2) and the first k in the order
 * (d2, primitive index). A query with a coordinate that is not finite has no
 * neighbours. Row qi of idx / d2 (uint32 / float [nq][k]) holds them in that
 * order; entries past min(k, n), and every entry of a query without
 * neighbours, are 0xffffffff / +inf. */
int oracle_knn_bruteforce(const float *prims, int64_t n, int kind, const float *queries, int64_t nq, int k,
                          uint32_t *idx, float *d2_out) {
    if (n < 0 || nq < 0 || k < 1 || (kind != ORACLE_POINTS && kind != ORACLE_BOXES)) return ORACLE_INVALID;
    const int64_t m = n < k ? n : k;
    float *bd = (float *)malloc((size_t)(k > 0 ? k : 1) * sizeof(float));
    uint32_t *bi = (uint32_t *)malloc((size_t)(k > 0 ? k : 1) * sizeof(uint32_t));
    if (!bd || !bi) {
        free(bd);
        free(bi);
        return ORACLE_INVALID;
    }
    for (int64_t qi = 0; qi < nq; ++qi) {
        const float *c = queries + 3 * qi;
        int64_t have = 0;
        if (isfinite(c[0]) && isfinite(c[1]) && isfinite(c[2])) {
            for (int64_t j = 0; j < n; ++j) {
                float box[6];
                for (int a = 0; a < 3; ++a) {
                    box[a] = kind == ORACLE_POINTS ? prims[3 * j + a] : prims[6 * j + a];
                    box[3 + a] = kind == ORACLE_POINTS ? prims[3 * j + a] : prims[6 * j + 3 + a];
                }
                const float d = point_box_d2(c, box);
                /* j is larger than every index kept so far, so among equal
                 * distances it goes last */
                if (have == m && !(d < bd[m - 1])) continue;
                int64_t at = have < m ? have : m - 1;
                while (at > 0 && d < bd[at - 1]) {
                    bd[at] = bd[at - 1];
                    bi[at] = bi[at - 1];
                    --at;
                }
                bd[at] = d;
                bi[at] = (uint32_t)j;
                if (have < m) ++have;
            }
        }
        for (int64_t r = 0; r < k; ++r) {
            idx[qi * k + r] = r < have ? bi[r] : 0xffffffffu;
            if (d2_out) d2_out[qi * k + r] = r < have ? bd[r] : INFINITY;
        }
    }
    free(bd);
    free(bi);
    return ORACLE_OK;
}

int oracle_sphere_box(const float *centre, float radius, const float *box6) {
    float r2 = radius * radius;
    return sphere_box_r2(centre, r2, box6);
}

int oracle_box_box(const float *a, const float *b) {
    for (int k = 0; k < 3; ++k) {
        if (!(a[k] <= b[3 + k] && b[k] <= a[3 + k])) return 0;
    }
    return 1;
}

/* A ray segment {origin.xyz, tmin, direction.xyz, tmax} against a closed box
 * (the slab test; range search for rays is Sec. 1's second example). Per axis:
 * inv = 1/d (IEEE division); when d == 0 or inv is infinite the ray is
 * parallel to the slab and stays in it only if lo <= o <= hi; otherwise
 * t1 = (lo - o) * inv and t2 = (hi - o) * inv, each operation rounded once.
 * tnear = max(tmin, min(t1, t2)) and tfar = min(tmax, max(t1, t2)) over the
 * axes; hit iff tnear <= tfar. A ray whose origin or direction is not finite,
 * or whose tmin or tmax is NaN, hits nothing. Every step is monotone in the
 * box, so a node's test passes whenever a box inside it passes. */
static int ray_box(const float *ray, const float *box) {
    for (int a = 0; a < 3; ++a)
        if (!isfinite(ray[a]) || !isfinite(ray[4 + a])) return 0;
    if (isnan(ray[3]) || isnan(ray[7])) return 0;
    float tnear = ray[3], tfar = ray[7];
    for (int a = 0; a < 3; ++a) {
        const float o = ray[a], d = ray[4 + a];
        const float inv = 1.0f / d;
        if (d == 0.0f || isinf(inv)) {
            if (!(box[a] <= o && o <= box[3 + a])) return 0;
            continue;
        }
        const float t1 = (box[a] - o) * inv;
        const float t2 = (box[3 + a] - o) * inv;
        const float tlo = t1 < t2 ? t1 : t2, thi = t1 < t2 ? t2 : t1;
        if (tlo > tnear) tnear = tlo;
        if (thi < tfar) tfar = thi;
    }
    return tnear <= tfar;
}

int oracle_ray_box(const float *ray8, const float *box6) { return ray_box(ray8, box6); }

static int cmp_u32(const void *pa, const void *pb) {
    uint32_t a = *(const uint32_t *)pa, b = *(const uint32_t *)pb;
    return a < b ? -1 : (a > b ? 1 : 0);
}

static int query_hits(int qkind, const float *q, float r2, const float *box) {
    if (qkind == ORACLE_RAY) return ray_box(q, box);
    return qkind == ORACLE_SPHERE ? sphere_box_r2(q, r2, box) : oracle_box_box(q, box);
}

static int query_dim(int qkind) { return qkind == ORACLE_SPHERE ? 3 : (qkind == ORACLE_BOX ? 6 : 8); }

int64_t oracle_query_traverse(int64_t n, const int32_t *left, const int32_t *skip_internal,
                              const int32_t *skip_leaf, const float *leaf_box,
                              const float *internal_box, const uint32_t *perm,
                              const float *queries, int64_t nq, int qkind,
                              const float *radii, float radius, int64_t *offsets,
                              uint32_t *hits, int64_t cap) {
    if (n < 0 || nq < 0 || (qkind != ORACLE_SPHERE && qkind != ORACLE_BOX && qkind != ORACLE_RAY)) return -1;
    const int64_t ni = n - 1;
    const int qdim = query_dim(qkind);
    const int64_t max_steps = 2 * (2 * n - 1) + 1;
    int64_t total = 0;
    for (int64_t qi = 0; qi < nq; ++qi) {
        const float *q = queries + qdim * qi;
        float r = radii ? radii[qi] : radius;
        float r2 = r * r;
        offsets[qi] = total;
        const int64_t start = total;
        int32_t node = n >= 1 ? 0 : -1; /* root: I_0 (or L_0 when n == 1) */
        int64_t steps = 0;
        while (node != -1) { /* Algorithm 1 */
            if (++steps > max_steps) return -1;
            const int is_leaf = node >= ni;
            const float *box = is_leaf ? leaf_box + 6 * (int64_t)(node - ni)
                                       : internal_box + 6 * (int64_t)node;
            if (query_hits(qkind, q, r2, box)) {
                if (is_leaf) {
                    if (hits && total < cap) hits[total] = perm[node - ni];
                    ++total;
                    node = skip_leaf[node - ni];
                } else {
                    node = left[node];
                }
            } else {
                node = is_leaf ? skip_leaf[node - ni] : skip_internal[node];
            }
        }
        if (hits && total <= cap && total > start)
            qsort(hits + start, (size_t)(total - start), sizeof(uint32_t), cmp_u32);
    }
    offsets[nq] = total;
    return total;
}

int64_t oracle_query_bruteforce(const float *prims, int64_t n, int kind, const float *queries,
                                int64_t nq, int qkind, const float *radii, float radius,
                                int64_t *offsets, uint32_t *hits, int64_t cap) {
    if (n < 0 || nq < 0 || (qkind != ORACLE_SPHERE && qkind != ORACLE_BOX && qkind != ORACLE_RAY)) return -1;
    if (kind != ORACLE_POINTS && kind != ORACLE_BOXES) return -1;
    const int qdim = query_dim(qkind);
    int64_t total = 0;
    for (int64_t qi = 0; qi < nq; ++qi) {
        const float *q = queries + qdim * qi;
        float r = radii ? radii[qi] : radius;
        float r2 = r * r;
        offsets[qi] = total;
        for (int64_t j = 0; j < n; ++j) {
            float box[6];
            for (int a = 0; a < 3; ++a) {
                box[a] = kind == ORACLE_POINTS ? prims[3 * j + a] : prims[6 * j + a];
                box[3 + a] = kind == ORACLE_POINTS ? prims[3 * j + a] : prims[6 * j + 3 + a];
            }
            if (query_hits(qkind, q, r2, box)) {
                if (hits && total < cap) hits[total] = (uint32_t)j;
                ++total;
            }
        }
    }
    offsets[nq] = total;
    return total;
}
