/*
 * lbvh_oracle.h -- CPU oracle for the linear BVH with skip connections of
 * Prokopenko & Lebrun-Grandie, "Revising Apetrei's bounding volume hierarchy
 * construction algorithm to allow stackless traversal" (arXiv 2402.00665).
 *
 * TEST INFRASTRUCTURE ONLY. This library is the independent reference that the
 * CUDA path is checked against. Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load it. It shares no code, header, table or
 * helper with the CUDA library, and it never calls it.
 *
 * Everything here is the plain definition of what the method computes, written
 * for a reader to check against the paper by eye:
 *   - Morton codes (Sec. 3.1, Karras step 1): quantise each centroid inside the
 *     scene bounds and interleave the bits (the paper leaves the encoding open;
 *     the reading used is spelled out in lbvh_oracle.c).
 *   - Sort (Sec. 3.1, Karras step 2): by code, ties by primitive index.
 *   - Binary radix tree (Sec. 3.1): each internal node covers a key range and
 *     splits it at the unique gap whose delta* is largest; children of split g
 *     are numbered g and g+1 (Karras ordering). delta compares the keys
 *     augmented with their sorted position (Sec. 3.2).
 *   - Skip connections (Sec. 2, Fig. 1): the pre-order successor that skips the
 *     node's subtree, or the sentinel on the right-most path.
 *   - Boxes (Sec. 3.1, Karras step 4): union of the children's boxes.
 *   - Range queries (Algorithm 1) and brute force over all primitives.
 *
 * Canonical node ids: internal node k -> k, leaf k -> (n-1)+k, sentinel -> -1.
 * Leaf k is sorted position k; perm[k] is its primitive index.
 *
 * Status codes: 0 ok, 1 invalid argument, 2 non-finite input.
 */
#ifndef LBVH_ORACLE_H
#define LBVH_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORACLE_OK = 0, ORACLE_INVALID = 1, ORACLE_NONFINITE = 2 };
enum { ORACLE_POINTS = 0, ORACLE_BOXES = 1 };
enum { ORACLE_SPHERE = 0, ORACLE_BOX = 1, ORACLE_RAY = 2 };

/* Centroid of each primitive. points: float[n][3]; boxes: float[n][6] as
 * (lo.x, lo.y, lo.z, hi.x, hi.y, hi.z). out: float[n][3]. */
int oracle_centroids(const float *prims, int64_t n, int kind, float *out);

/* Per-axis min/max of the centroids: out = (min.x, min.y, min.z, max.x,
 * max.y, max.z). Returns ORACLE_NONFINITE if any centroid is NaN or inf. */
int oracle_scene_bounds(const float *centroids, int64_t n, float *out);

/* Quantise one coordinate to b bits inside [lo, hi]. */
uint32_t oracle_quantize(float c, float lo, float hi, int b);

/* Interleave three b-bit integers, x the most significant of each triple. */
uint64_t oracle_interleave(uint32_t qx, uint32_t qy, uint32_t qz, int b);

/* Morton code of every primitive. bits: multiple of 3 in [3, 63].
 * codes: uint64[n]; bounds_out (nullable): 6 floats. */
int oracle_morton_codes(const float *prims, int64_t n, int kind, int bits,
                        uint64_t *codes, float *bounds_out);

/* Order by (code, primitive index). perm[k] = primitive at sorted position k,
 * sorted[k] = its code. */
int oracle_sort_codes(const uint64_t *codes, int64_t n, uint32_t *perm,
                      uint64_t *sorted);

/* delta(i, j) of Sec. 3.1 with the XOR reading of Sec. 3.2: the index of the
 * highest bit in which the augmented keys (sorted[i], i) and (sorted[j], j)
 * differ, counting the 32 position bits below the 64 code bits. Returns
 * INT32_MAX ("+infinity") when i or j is outside [0, n-1] or i == j. */
int32_t oracle_delta(const uint64_t *sorted, int64_t n, int64_t i, int64_t j);

/* Karras topology of the sorted keys, top-down from the root I_0.
 * left/right: int32[n-1] canonical child ids; range_l/range_r/split:
 * int32[n-1]. n >= 2 for any internal node to exist. */
int oracle_topology(const uint64_t *sorted, int64_t n, int32_t *left,
                    int32_t *right, int32_t *range_l, int32_t *range_r,
                    int32_t *split);

/* Skip connections from an explicit pre-order walk. skip_internal: int32[n-1],
 * skip_leaf: int32[n], preorder (nullable): int32[2n-1] canonical ids. */
int oracle_skips(int64_t n, const int32_t *left, const int32_t *right,
                 int32_t *skip_internal, int32_t *skip_leaf, int32_t *preorder);

/* Leaf boxes in sorted order (float[n][6]) and internal boxes
 * (float[n-1][6]) as the post-order union of the children. */
int oracle_boxes(const float *prims, int64_t n, int kind, const uint32_t *perm,
                 const int32_t *left, const int32_t *right, float *leaf_box,
                 float *internal_box);

/* The whole build. Any output pointer may be NULL except those that later
 * steps need, which are allocated internally when NULL. Sizes as above. */
int oracle_build(const float *prims, int64_t n, int kind, int bits,
                 uint64_t *codes_out, float *bounds_out, uint32_t *perm_out,
                 uint64_t *sorted_out, int32_t *left_out, int32_t *right_out,
                 int32_t *skip_internal_out, int32_t *skip_leaf_out,
                 int32_t *range_l_out, int32_t *range_r_out,
                 int32_t *split_out, float *leaf_box_out,
                 float *internal_box_out);

/* Algorithm 1 over the oracle tree, one query at a time.
 * queries: sphere centres float[nq][3] or boxes float[nq][6]. radii: float[nq]
 * or NULL to use `radius` for every query. offsets: int64[nq+1] (always
 * written). hits: int64 capacity `cap`; NULL to only count. Hits of each query
 * are primitive indices in ascending order. Returns the total hit count, or -1
 * on invalid arguments. */
int64_t oracle_query_traverse(int64_t n, const int32_t *left,
                              const int32_t *skip_internal,
                              const int32_t *skip_leaf, const float *leaf_box,
                              const float *internal_box, const uint32_t *perm,
                              const float *queries, int64_t nq, int qkind,
                              const float *radii, float radius,
                              int64_t *offsets, uint32_t *hits, int64_t cap);

/* All-pairs brute force with the same predicates; same output convention. */
int64_t oracle_query_bruteforce(const float *prims, int64_t n, int kind,
                                const float *queries, int64_t nq, int qkind,
                                const float *radii, float radius,
                                int64_t *offsets, uint32_t *hits, int64_t cap);

/* k nearest neighbours (the distance range search of Sec. 1 turned into its
 * k closest answers) by brute force: for each query point the first k
 * primitives in the order (squared point-to-box distance, primitive index).
 * queries float[nq][3]; idx uint32[nq][k], d2 float[nq][k] (nullable); rows
 * are padded with 0xffffffff / +inf past min(k, n), and a query with a
 * non-finite coordinate has no neighbours. Returns ORACLE_OK or
 * ORACLE_INVALID. */
int oracle_knn_bruteforce(const float *prims, int64_t n, int kind, const float *queries, int64_t nq, int k,
                          uint32_t *idx, float *d2);
/* The squared distance used above (the ball test's d2). */
float oracle_point_box_d2(const float *point, const float *box6);

/* The predicates themselves, exported for tests. */
int oracle_sphere_box(const float *centre, float radius, const float *box6);
int oracle_box_box(const float *a6, const float *b6);
/* Ray segment {origin.xyz, tmin, direction.xyz, tmax} against a closed box (slab test). */
int oracle_ray_box(const float *ray8, const float *box6);

#ifdef __cplusplus
}
#endif
#endif
