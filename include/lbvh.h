/*
 * lbvh.h -- C ABI of the GB300 (sm_103a) linear BVH with skip connections.
 *
 * Method: Prokopenko & Lebrun-Grandie, "Revising Apetrei's bounding volume
 * hierarchy construction algorithm to allow stackless traversal",
 * arXiv 2402.00665. The build computes Morton codes (Sec. 3.1 step 1), sorts
 * them (step 2), and runs the modified Apetrei bottom-up pass (Sec. 4,
 * Algorithm 4) that writes every internal node in Karras' ordering with its
 * left child, its skip connection (Sec. 2, Algorithm 2) and its box (step 4),
 * in one pass. Queries walk the tree without a stack (Algorithm 1).
 *
 * Conventions for every function below
 *   - Pointers named d_* are device pointers (cudaMalloc, cudaMallocAsync or
 *     a PyTorch CUDA tensor), h_* are host pointers. The library never frees
 *     memory the caller passed in.
 *   - `stream` is a cudaStream_t (CUstream) handle passed as void*; NULL is
 *     the legacy default stream. Work is enqueued on it and ordered with the
 *     caller's other work on that stream. Calls that must know a size on the
 *     host (a query's hit count, an export) synchronise that stream and say so.
 *   - Every function returns an lbvh_status and never throws. A device-side
 *     error found during a build (non-finite input, a sort wait that ran out)
 *     is latched in the tree and reported by the next call that synchronises:
 *     lbvh_tree_status, lbvh_query*, lbvh_tree_export.
 *   - Floating-point layouts: points float[n][3] (x, y, z); boxes float[n][6]
 *     (lo.x, lo.y, lo.z, hi.x, hi.y, hi.z); sphere queries float[nq][3]
 *     centres; box queries float[nq][6]. Arrays are contiguous, row-major.
 *   - Canonical node ids (export): internal node k -> k, leaf k -> (n-1)+k,
 *     sentinel -> -1. Leaf k is the k-th primitive in sorted Morton order and
 *     perm[k] is its primitive index. The root is id 0 (I_0; L_0 when n == 1).
 *   - Results are exact (bit-identical to the CPU oracle): codes, topology,
 *     skips and FP32 boxes (min/max only), and the CSR hit lists, whose
 *     entries are primitive indices in ascending order within each query.
 */
#ifndef LBVH_H
#define LBVH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbvh_tree_s *lbvh_tree_t; /* opaque; device storage owned by the library */
typedef void *lbvh_stream_t;             /* cudaStream_t */

typedef enum {
    LBVH_OK = 0,
    LBVH_ERR_INVALID = 1,   /* bad argument: null pointer, size out of range, bad kind/bits */
    LBVH_ERR_NONFINITE = 2, /* a primitive centroid is NaN or infinite */
    LBVH_ERR_OOM = 3,       /* device allocation failed */
    LBVH_ERR_CUDA = 4,      /* a CUDA runtime call failed (see lbvh_last_cuda_error) */
    LBVH_ERR_TIMEOUT = 5,   /* a bounded device-side wait ran out; results are invalid */
    LBVH_ERR_CORRUPT = 6,   /* a traversal exceeded 2(2n-1) steps; the tree is not valid */
    LBVH_ERR_CAPACITY = 7   /* the caller's hit buffer is too small; *total holds the need */
} lbvh_status;

typedef enum { LBVH_PRIM_POINTS = 0, LBVH_PRIM_BOXES = 1 } lbvh_prim_kind;
typedef enum { LBVH_Q_SPHERE = 0, LBVH_Q_BOX = 1, LBVH_Q_RAY = 2 } lbvh_query_kind;

/* Largest primitive count of one tree: the sort's look-back words carry a
 * 30-bit count and node ids are int32 over 2n-1 nodes. */
#define LBVH_MAX_PRIMS ((int64_t)((1 << 30) - 1))

/* ---------------------------------------------------------------- tree */

/* A tree handle may be used by one call at a time (builds, queries, refits,
 * exports and saves share its scratch buffers); different trees may be used
 * from different threads at once. */

/* Create an empty tree handle (no device memory yet). *out receives it. */
lbvh_status lbvh_tree_create(lbvh_tree_t *out);

/* Release the tree and all device memory it owns. Waits for the tree's own
 * last build and last query to finish first (not for whole streams). Accepts
 * NULL. */
void lbvh_tree_destroy(lbvh_tree_t tree);

/* Build (or rebuild in place) the whole hierarchy: scene bounds, Morton codes
 * (Sec. 3.1 step 1), stable radix sort of the codes with the primitive index
 * as payload (step 2), and the single bottom-up pass of Algorithm 4 that
 * writes internal nodes in Karras' ordering with left child, skip and box, and
 * every leaf's skip and box (Sec. 4).
 *   d_prims      device float[n][3] (points) or float[n][6] (boxes); read only
 *                during the call's stream work; the tree keeps its own copy of
 *                the geometry in its leaves.
 *   n            0 <= n <= LBVH_MAX_PRIMS (n == 0 gives an empty tree).
 *   kind         lbvh_prim_kind.
 *   morton_bits  total code bits, a multiple of 3 in [3, 63] (30 and 63 are
 *                the usual choices: 10 or 21 bits per axis).
 * Asynchronous on `stream`; device storage grows (from the library's
 * stream-ordered pool) only when n exceeds what the tree already holds. Errors found on the device are latched
 * (see lbvh_tree_status). Returns LBVH_ERR_INVALID for bad arguments. */
lbvh_status lbvh_build(lbvh_tree_t tree, const float *d_prims, int64_t n, int kind,
                       int morton_bits, lbvh_stream_t stream);

/* The hierarchy algorithms the paper compares (Sec. 3-5). */
typedef enum {
    LBVH_BUILD_MODIFIED_APETREI = 0, /* Algorithm 4: one bottom-up pass, Karras ordering, skips, boxes */
    LBVH_BUILD_KARRAS = 1,           /* Karras (Sec. 3.1): a thread per internal node finds its range
                                        and split by binary search; a bottom-up pass writes boxes */
    LBVH_BUILD_APETREI = 2           /* Algorithm 3: bottom-up with compare-and-swap, nodes in
                                        Apetrei's ordering (index = split); a second pass converts to
                                        Karras' ordering and installs skips (Algorithm 2) */
} lbvh_build_algorithm;

/* lbvh_build with the hierarchy step of the chosen algorithm. Scene bounds,
 * codes and the sort are the same; every algorithm ends in the same tree
 * (Karras' ordering, left children, skips, boxes: the radix tree of the
 * augmented keys is unique), so the result equals lbvh_build's bit for bit
 * and is queried and exported the same way. For timing the three against
 * each other: stage LBVH_STAGE_CONSTRUCT is the hierarchy kernel (Algorithm 4,
 * Karras' per-node search, Algorithm 3) and LBVH_STAGE_SECOND the extra pass
 * the other two need (Karras: boxes; Apetrei: ordering and skips). The Karras
 * and Apetrei builds use scratch of 20 and 48 bytes per primitive. Returns
 * LBVH_ERR_INVALID for an unknown algorithm, else as lbvh_build. */
lbvh_status lbvh_build_variant(lbvh_tree_t tree, const float *d_prims, int64_t n, int kind,
                               int morton_bits, int algorithm, lbvh_stream_t stream);

/* Checkpoint: the whole tree as one flat host byte image, and back.
 * Image (version 1, little-endian): "LBVHTREE" (8 bytes), uint32 version,
 * kind, morton_bits, 0; uint64 n; float bounds[6] (scene bounds of the
 * centroids), 8 bytes of padding; uint64 sorted codes[n]; uint32 perm[n];
 * then the device node records as they are (internal node k: float4 {lo.xyz,
 * left}, float4 {hi.xyz, skip}; leaves: float4 {x, y, z, word} for points or
 * {lo.xyz, word}, {hi.xyz, 0} for boxes, as described at lbvh_build).
 * lbvh_tree_save: with h_buf == NULL (or capacity too small: then
 * LBVH_ERR_CAPACITY) only *bytes is set to the image size; otherwise the
 * image is written to h_buf (host memory; synchronises the tree's stream).
 * Trees kept by the request server hold no codes and return
 * LBVH_ERR_INVALID. lbvh_tree_load: replaces the tree with the image (the
 * copies run on `stream`, which is synchronised before the call returns); a
 * bad magic, version, kind, bit count, size or n returns LBVH_ERR_INVALID
 * before anything is copied. A loaded tree is
 * queried, exported, refitted and saved like a built one. */
lbvh_status lbvh_tree_save(lbvh_tree_t tree, void *h_buf, uint64_t capacity, uint64_t *bytes);
lbvh_status lbvh_tree_load(lbvh_tree_t tree, const void *h_buf, uint64_t bytes, lbvh_stream_t stream);

/* Refit: new boxes for moved primitives on the tree's existing topology.
 * Every leaf box is re-read from d_prims (leaf k holds primitive perm[k] as
 * before) and the bottom-up pass of Algorithm 4 runs again over the stored
 * sorted codes, so every node keeps its children and skip connection and gets
 * the union of its new child boxes; the scene bounds are recomputed (they
 * only steer the query order). Codes are not recomputed: queries stay exact
 * however far the primitives move, but the tree's quality decays with the
 * motion, and a rebuild restores it.
 *   d_prims  device float[n][3] or float[n][6], the same n, kind and index
 *            order as the tree's last build.
 * Asynchronous on `stream`. Returns LBVH_ERR_INVALID for a tree without a
 * build or without stored codes (trees kept by the request server); device
 * errors (non-finite input) are latched as in lbvh_build. */
lbvh_status lbvh_refit(lbvh_tree_t tree, const float *d_prims, lbvh_stream_t stream);

/* Build from codes that are already sorted (Sec. 3.1 steps 3-4 and Sec. 4
 * only): d_sorted_codes uint64[n] ascending, d_perm uint32[n] the primitive
 * index of each sorted position, d_prims the geometry as for lbvh_build.
 * Used to test the bottom-up pass on the paper's worked example. */
lbvh_status lbvh_build_from_sorted(lbvh_tree_t tree, const uint64_t *d_sorted_codes,
                                   const uint32_t *d_perm, const float *d_prims, int64_t n,
                                   int kind, lbvh_stream_t stream);

/* Synchronise the tree's stream and return the first error latched by its
 * last build (LBVH_OK if none). */
lbvh_status lbvh_tree_status(lbvh_tree_t tree);

/* Number of primitives of the last build. */
lbvh_status lbvh_tree_size(lbvh_tree_t tree, int64_t *n);

/* Device bytes the tree currently holds (nodes, leaves, sort and query
 * scratch). */
lbvh_status lbvh_tree_bytes(lbvh_tree_t tree, uint64_t *bytes);

/* Copy the canonical arrays of the last build to host memory. Synchronises
 * the tree's stream. Any pointer may be NULL to skip that array.
 *   h_perm          uint32[n]   primitive index of sorted position k
 *   h_sorted_codes  uint64[n]   Morton code of sorted position k
 *   h_left          int32[n-1]  left child id of internal node k
 *   h_skip_internal int32[n-1]  skip id of internal node k
 *   h_skip_leaf     int32[n]    skip id of leaf k
 *   h_internal_box  float[n-1][6] box of internal node k (lo.xyz, hi.xyz)
 *   h_leaf_box      float[n][6]   box of leaf k (points: lo == hi)
 *   h_bounds        float[6]      scene bounds of the centroids (min, max) */
lbvh_status lbvh_tree_export(lbvh_tree_t tree, uint32_t *h_perm, uint64_t *h_sorted_codes,
                             int32_t *h_left, int32_t *h_skip_internal, int32_t *h_skip_leaf,
                             float *h_internal_box, float *h_leaf_box, float *h_bounds);

/* ---------------------------------------------------------------- queries */

/* Stackless range query (Algorithm 1) of every query against the tree, with
 * results in caller-owned CSR buffers. Sec. 1 gives the two kinds of range
 * search: objects within a distance, and objects a ray meets.
 *   d_queries  sphere centres float[nq][3], boxes float[nq][6], or ray
 *              segments float[nq][8] = {origin.xyz, tmin, direction.xyz,
 *              tmax} (16-byte aligned).
 *   qkind      lbvh_query_kind. Sphere: closed ball, hit iff the squared
 *              distance from the centre to the primitive's box is <= r*r,
 *              in FP32: d2 = ex*ex, then + ey*ey and + ez*ez each as one
 *              fused multiply-add (e = the centre's gap to the box on that
 *              axis); a NaN centre coordinate or radius hits nothing. Box:
 *              closed overlap on all three axes. Ray: the slab test, each
 *              operation rounded once: per axis inv = 1/d; an axis with d == 0
 *              (or an infinite inv) needs lo <= o <= hi; else t1 = (lo-o)*inv,
 *              t2 = (hi-o)*inv, tnear = max(tmin, min(t1,t2)), tfar =
 *              min(tmax, max(t1,t2)); hit iff tnear <= tfar. A ray with a
 *              non-finite origin or direction, or a NaN tmin/tmax, hits
 *              nothing. Rays are walked in the order given; spheres and boxes
 *              in the Morton order of their centres.
 *   d_radii    float[nq] per-query radius, or NULL to use `radius` for all
 *              (`radius` must then be finite and >= 0).
 *   d_offsets  int64[nq+1]: hits of query q are d_hits[d_offsets[q] ..
 *              d_offsets[q+1]), primitive indices in ascending order.
 *   d_hits     uint32[capacity].
 *   total      out: the total number of hits.
 * Synchronises `stream` once (to learn the total). If total > capacity the
 * call returns LBVH_ERR_CAPACITY with *total set and d_offsets valid, and
 * leaves d_hits unspecified; call again with a larger buffer. */
lbvh_status lbvh_query_into(lbvh_tree_t tree, const float *d_queries, int64_t nq, int qkind,
                            const float *d_radii, float radius, int64_t *d_offsets,
                            uint32_t *d_hits, uint64_t capacity, uint64_t *total,
                            lbvh_stream_t stream);

/* As lbvh_query_into, but the CSR arrays are in page-locked host memory
 * (cudaMallocHost, cudaHostAlloc or cudaHostRegister): h_offsets int64[nq+1],
 * h_hits uint32[capacity], owned by the caller. The queries go through the
 * device path in chunks (in index order; at least 2^23 queries each, at most
 * 4 chunks unless lbvh_tree_set_host_chunks says otherwise), each into one of
 * two device staging areas that the tree owns; a
 * chunk's offsets and hits are copied to the host on the tree's own copy
 * stream while the GPU works on the next chunk. Like every call here it
 * returns once the last chunk is counted; the host arrays are complete once
 * `stream` has been synchronised (it waits for the copies). Over capacity:
 * the offsets are still written, no hit is, LBVH_ERR_CAPACITY with the full
 * *total. Host memory that is not page-locked (pageable or device memory)
 * -> LBVH_ERR_INVALID, nothing is launched. Other errors as lbvh_query_into. */
lbvh_status lbvh_query_into_host(lbvh_tree_t tree, const float *d_queries, int64_t nq, int qkind,
                                 const float *d_radii, float radius, int64_t *h_offsets,
                                 uint32_t *h_hits, uint64_t capacity, uint64_t *total,
                                 lbvh_stream_t stream);

/* The most chunks lbvh_query_into_host cuts a tree's queries into (chunks
 * of at least 2^23 queries): 1 to 16, or 0 for the default of 4 (else
 * LBVH_ERR_INVALID). Every chunk costs a host round trip (its hit count);
 * in return a chunk's copy to the host overlaps the next chunk's work. A
 * caller that waits for each result does best with 3-4 (2^25 sphere queries
 * of ~17 hits: 27.0 ms with 4 chunks, 32.6 ms with 1); a caller that keeps
 * two queries in flight on two trees, so that one tree's copy overlaps the
 * other tree's build and walk, does best with 1. Fewer chunks hold more at
 * once: a chunk's query scratch (about 330 bytes per query) and its staged
 * CSR live on the device together, so 1 chunk of 2^25 queries of ~17 hits
 * needs about 14 GB (LBVH_ERR_OOM if it cannot be had). Results do not
 * depend on it. Not an operation of the paper: a transfer setting of this
 * library. */
lbvh_status lbvh_tree_set_host_chunks(lbvh_tree_t tree, int max_chunks);

/* As lbvh_query_into, but the library allocates the CSR arrays
 * (*d_offsets int64[nq+1], *d_hits uint32[*total]); free them with lbvh_free. */
lbvh_status lbvh_query(lbvh_tree_t tree, const float *d_queries, int64_t nq, int qkind,
                       const float *d_radii, float radius, int64_t **d_offsets,
                       uint32_t **d_hits, uint64_t *total, lbvh_stream_t stream);

/* Measurement: the number of leaves and internal nodes Algorithm 1 visits
 * for these queries (the collecting walk's work), summed over all queries,
 * walked in the same order as lbvh_query_into; no hits are kept. Arguments
 * as lbvh_query_into. Synchronises `stream`. */
lbvh_status lbvh_tree_walk_visits(lbvh_tree_t tree, const float *d_queries, int64_t nq, int qkind,
                                  const float *d_radii, float radius, uint64_t *leaf_visits,
                                  uint64_t *internal_visits, lbvh_stream_t stream);

/* Largest k accepted by lbvh_knn. */
#define LBVH_KNN_MAX_K 256

/* The k nearest primitives of each query point: the distance range search of
 * Sec. 1 asked for its k closest answers, walked stacklessly (Algorithm 1)
 * with a ball whose radius is the current k-th best distance, which only
 * shrinks, so the walk never skips a subtree that could hold an answer.
 *   d_queries  query points float[nq][3].
 *   k          1 .. LBVH_KNN_MAX_K.
 *   d_idx      uint32[nq][k] out: row q holds the min(k, n) nearest primitive
 *              indices in the order (squared distance, primitive index), then
 *              0xffffffff padding. The squared distance is the one of the
 *              sphere query (the point's gap to the primitive's box per axis,
 *              FP32, d2 = ex*ex, + ey*ey, + ez*ez as fused multiply-adds). A
 *              query with a non-finite coordinate has no neighbours.
 *   d_dist2    float[nq][k] out or NULL: the squared distances, +inf padding.
 * Buffers are the caller's. Synchronises `stream` once (for the status).
 * LBVH_ERR_INVALID on bad arguments or an unbuilt tree; the build's error if
 * it failed; LBVH_ERR_CORRUPT if a walk met an id outside the tree. */
lbvh_status lbvh_knn(lbvh_tree_t tree, const float *d_queries, int64_t nq, int k, uint32_t *d_idx,
                     float *d_dist2, lbvh_stream_t stream);

/* Free device memory returned by lbvh_query. Accepts NULL. */
void lbvh_free(void *d_ptr);

/* Device memory that trees, batches and servers allocate comes from one
 * stream-ordered pool per device that the library owns and that keeps freed
 * blocks for reuse (so repeated builds do not map and unmap memory). This
 * returns the pool's unused blocks to the device; blocks held by live trees,
 * batches and servers stay. */
lbvh_status lbvh_release_cached_memory(void);

/* ---------------------------------------------------------------- stages */

/* Scene bounds and Morton code of every primitive (Sec. 3.1 step 1): the
 * centroid (a box's is (lo + hi) * 0.5) is quantised per axis to b =
 * morton_bits/3 bits inside the bounds, t = (c - min)/(max - min) in FP32,
 * cell = clamp(trunc(t * 2^b), 0, 2^b - 1), 0 on an axis of zero extent; the
 * bits are interleaved with x the most significant of each triple.
 *   d_codes   uint64[n] out.   d_bounds  float[6] out (min.xyz, max.xyz).
 * Returns LBVH_ERR_NONFINITE (after synchronising `stream`) if any centroid
 * is not finite. */
lbvh_status lbvh_morton_codes(const float *d_prims, int64_t n, int kind, int morton_bits,
                              uint64_t *d_codes, float *d_bounds, lbvh_stream_t stream);

/* Stable LSD radix sort of 64-bit keys with 32-bit payloads (Sec. 3.1 step
 * 2). Only the low `key_bits` bits (1..64) of each key are sorted on. d_vals
 * may be NULL for the payload 0, 1, ..., n-1 (the primitive index). Inputs are
 * not modified; outputs must not alias inputs. Synchronises `stream` and
 * returns LBVH_ERR_TIMEOUT if a bounded device wait ran out. */
lbvh_status lbvh_sort_pairs(const uint64_t *d_keys, const uint32_t *d_vals, int64_t n,
                            int key_bits, uint64_t *d_keys_out, uint32_t *d_vals_out,
                            lbvh_stream_t stream);

/* ---------------------------------------------------------------- batches */

typedef struct lbvh_batch_s *lbvh_batch_t; /* opaque; device storage owned by the library */

/* Most instances in one batch call (the sort keeps 1 KiB of digit counts per
 * instance and pass). */
#define LBVH_MAX_BATCH (1 << 20)

/* Create an empty batch handle. */
lbvh_status lbvh_batch_create(lbvh_batch_t *out);

/* Release the batch and its device memory (waits for its stream). Accepts NULL. */
void lbvh_batch_destroy(lbvh_batch_t batch);

/* Build `count` independent trees and answer each tree's own queries (spheres
 * or boxes; rays: LBVH_ERR_INVALID) in one
 * pass over all of them: the same method as lbvh_build + lbvh_query_into per
 * instance (Sec. 3.1 steps 1-4, Algorithm 4, Algorithm 1), with every step
 * run once for the whole batch (per-instance scene bounds; one segmented
 * radix sort in which every instance's codes are sorted on their own; the
 * bottom-up pass of all trees at once; one walk kernel for all queries). Each
 * instance's tree and hit lists are identical to what a single build of that
 * instance produces.
 *   d_prims          concatenated primitives (layout of lbvh_build), device.
 *   count            number of instances, 1 <= count <= LBVH_MAX_BATCH.
 *   h_prim_offsets   host int64[count+1], h_prim_offsets[0] == 0: instance b
 *                    owns primitives [off[b], off[b+1]) (may be empty).
 *   morton_bits      as lbvh_build (any width; instances are sorted apart).
 *   d_queries        concatenated queries (layout of lbvh_query_into).
 *   h_query_offsets  host int64[count+1]: queries of instance b.
 *   d_radii/radius   as lbvh_query_into (per query, or one for all).
 *   d_offsets        int64[total queries + 1]; d_hits uint32[capacity]: one
 *                    CSR over all queries in their concatenated order; hit
 *                    ids are primitive indices local to the query's instance.
 *   total            out: total hits. If total > capacity, returns
 *                    LBVH_ERR_CAPACITY (d_offsets valid, d_hits unspecified).
 * The first call with a given set of arguments (pointers, offsets, kinds,
 * bits, radius, capacity) sets up buffers, tunes the sort's tile shape on the
 * batch (CUDA-event timing) and records the whole pipeline as one CUDA graph;
 * later calls with the same arguments launch that graph once. Every call
 * synchronises `stream` once at the end (to report total and status). Totals
 * of primitives and of queries are each below 2^31. */
lbvh_status lbvh_batch_build_query(lbvh_batch_t batch, const float *d_prims,
                                   const int64_t *h_prim_offsets, int64_t count, int kind,
                                   int morton_bits, const float *d_queries,
                                   const int64_t *h_query_offsets, int qkind, const float *d_radii,
                                   float radius, int64_t *d_offsets, uint32_t *d_hits,
                                   uint64_t capacity, uint64_t *total, lbvh_stream_t stream);

/* Canonical arrays of one instance of the last batch run (as
 * lbvh_tree_export; perm holds indices local to the instance). */
lbvh_status lbvh_batch_export(lbvh_batch_t batch, int64_t instance, uint32_t *h_perm,
                              uint64_t *h_sorted_codes, int32_t *h_left, int32_t *h_skip_internal,
                              int32_t *h_skip_leaf, float *h_internal_box, float *h_leaf_box,
                              float *h_bounds);

/* The sort tile shape the batch's autotuner chose (-1: default, not tuned). */
lbvh_status lbvh_batch_sort_variant(lbvh_batch_t batch, int *variant);

/* ---------------------------------------------------------------- serving */

typedef struct lbvh_server_s *lbvh_server_t; /* opaque */

/* One request. A build request (n > 0) builds a tree of its primitives and
 * answers its queries (spheres or boxes); a query-only request (n == 0)
 * queries the resident tree stored under `key` (spheres, boxes or rays). Every pointer is device memory that the caller
 * keeps valid (inputs) or reserved (outputs) until lbvh_server_wait returns
 * for the request. */
typedef struct {
    const float *d_prims;  /* build: float[n][3] or float[n][6] */
    int64_t n;             /* primitives; 0 = query the resident tree `key` */
    int kind;              /* lbvh_prim_kind */
    int morton_bits;       /* as lbvh_build */
    const float *d_queries;
    int64_t nq;
    int qkind;             /* lbvh_query_kind */
    float radius;
    const float *d_radii;  /* nullable: per-query radii */
    int64_t *d_offsets;    /* out: int64[nq+1], the request's own CSR */
    uint32_t *d_hits;      /* out: uint32[capacity] */
    uint64_t capacity;
    uint64_t key;          /* build: nonzero keeps the tree resident under this key
                              (replacing an older one); query-only: the tree to use */
} lbvh_request;

typedef struct {
    lbvh_status status;   /* LBVH_ERR_CAPACITY: `total` is the need; LBVH_ERR_INVALID for a
                             query on a key that is not resident (never built, or evicted) */
    uint64_t total;       /* hits of the request */
    double queued_s;      /* submission -> start of the batch that ran it */
    double service_s;     /* start of that batch -> results in the request's buffers */
    double latency_s;     /* submission -> results in the request's buffers */
    int batch_size;       /* requests that ran in the same batch */
} lbvh_result;

/* Start a request server: `slots` worker streams (1..16), each running one
 * batch at a time, so up to `slots` batches overlap on the device (a batch
 * of 2^23 primitives or more, which fills the GPU alone, starts only when no
 * other batch runs); at most `max_batch` requests per batch. The scheduler admits queued requests in
 * arrival order while their estimated working bytes plus the bytes of the
 * resident trees fit `hbm_budget_bytes`, evicting the least recently used
 * resident trees (not in use) to make room; requests that arrive while others
 * run join the next batch as soon as a slot and memory are free (continuous
 * batching). Build requests in one batch share primitive kind, Morton bits
 * and query kind (a request of another kind starts the next batch). Each
 * request's results equal those of lbvh_build + lbvh_query_into on it alone. */
lbvh_status lbvh_server_create(uint64_t hbm_budget_bytes, int slots, int max_batch,
                               lbvh_server_t *out);

/* Queue a request (copied; returns at once). *ticket identifies it. */
lbvh_status lbvh_server_submit(lbvh_server_t server, const lbvh_request *request, uint64_t *ticket);

/* Block until the request has finished; fills *result and forgets the ticket. */
lbvh_status lbvh_server_wait(lbvh_server_t server, uint64_t ticket, lbvh_result *result);

/* Resident-tree bytes and count, evictions and batches so far (any pointer may be NULL). */
lbvh_status lbvh_server_stats(lbvh_server_t server, uint64_t *resident_bytes, uint64_t *resident_trees,
                              uint64_t *evictions, uint64_t *batches);

/* Latency (submission to results, seconds) of every request answered so far:
 * nearest-rank p50 and p99 and the count (any pointer may be NULL). */
lbvh_status lbvh_server_latency(lbvh_server_t server, double *p50_s, double *p99_s, uint64_t *count);

/* Where the workers' time went, summed over all batches so far (host wall
 * clock, so with several slots the sums can exceed the elapsed time):
 *   seconds[0]  staging a batch's inputs (copies into one concatenated batch),
 *   seconds[1]  the batched build + query (lbvh_batch_build_query, which
 *               waits for its own results),
 *   seconds[2]  handing the results to each request and copying the trees
 *               that stay resident, up to the wait for those copies,
 *   seconds[3]  query-only requests.
 * `seconds` holds LBVH_SERVER_PHASES doubles. */
#define LBVH_SERVER_PHASES 4
lbvh_status lbvh_server_phase_seconds(lbvh_server_t server, double *seconds);

/* Device spans of the jobs run so far: for each job (a batch, or a
 * query-only request) a triple {slot, begin s, end s} measured by CUDA
 * events on the slot's stream, in seconds from one reference event recorded
 * when the server was created, so spans of different slots can be compared
 * (overlapping spans ran on the device at the same time). spans: double
 * [capacity][3]; *count receives the number of jobs (which may exceed
 * capacity; the first `capacity` are written). */
lbvh_status lbvh_server_device_spans(lbvh_server_t server, double *spans, uint64_t capacity, uint64_t *count);

/* Finish all queued work, then stop the threads and free everything. */
void lbvh_server_destroy(lbvh_server_t server);

/* ---------------------------------------------------------------- no allocation */

/* Largest n accepted by lbvh_construct_static. */
#define LBVH_STATIC_MAX_PRIMS ((int64_t)((1 << 20) + 1))

/* The bottom-up pass of lbvh_build_from_sorted (nodes, boxes, skip
 * connections from sorted codes) without any device allocation. The paper has
 * no counterpart: this entry point exists for callers that may not allocate
 * device memory through this library -- for example a host application whose
 * own pool allocator owns the whole device heap and forbids other
 * allocations, or a code path that must not call cudaMalloc / cudaFree
 * because those synchronise the device. The caller passes every input and
 * output buffer; the scratch words of the merge live in a file-scope device
 * array of LBVH_STATIC_MAX_PRIMS - 1 64-bit words (8 MiB) that every GPU which
 * loads this library keeps until the process exits.
 *   d_sorted_codes uint64[n] ascending; d_perm uint32[n] primitive index of
 *     each sorted position; d_prims float[n][3] points or float[n][6] boxes.
 *   1 <= n <= LBVH_STATIC_MAX_PRIMS, else LBVH_ERR_INVALID (nothing runs).
 *   d_inodes float4[2(n-1)] out (may be NULL when n == 1): internal node k =
 *     {lo.x, lo.y, lo.z, left}, {hi.x, hi.y, hi.z, skip}, ids as int bits.
 *   d_leaves out: points float4[n] = {x, y, z, word}; boxes float4[2n] =
 *     {lo.xyz, word}, {hi.xyz, 0}; word (uint32 bits) = primitive index |
 *     (1u << 31 if the leaf's skip is internal node k+1, else leaf k+1; the
 *     last leaf's skip is the sentinel).
 *   d_flags uint32 device word or NULL: bit 2 is set if a perm entry is out
 *     of range, two adjacent codes are out of order, or the merge leaves the
 *     tree (the outputs are then invalid). A perm that repeats an index is
 *     not detected. The caller clears the word.
 * Asynchronous on `stream`; allocates nothing (no cudaMalloc, cudaFree or
 * allocating library call). Every call looks up the device address of the
 * scratch array (cudaGetSymbolAddress) with the calling thread's current
 * device, so an address is never kept past a device reset; the first call on
 * a device also loads the library's device code there, so make that first
 * call before any stream capture. Each call
 * clears the scratch words it uses; calls that overlap on the GPU (on
 * different streams, or from different threads) share the one array and race,
 * so serialise them. */
lbvh_status lbvh_construct_static(const uint64_t *d_sorted_codes, const uint32_t *d_perm,
                                  const float *d_prims, int64_t n, int kind, float *d_inodes,
                                  float *d_leaves, uint32_t *d_flags, lbvh_stream_t stream);

/* ---------------------------------------------------------------- failure tests */

/* Test hook for failure detection, off by default (-1). While set, tile
 * `tile` of the first pass of every radix sort publishes nothing to the
 * decoupled look-back, so the later tiles' waits on it run out (each wait is
 * bounded to about one second): the build then reports LBVH_ERR_TIMEOUT, its
 * output is invalid and nothing is written out of bounds; the next build
 * after the hook is cleared is correct again. Nothing faults, traps or hangs. */
lbvh_status lbvh_test_hold_sort_tile(int64_t tile);

/* Test hook for the order of arrivals in Algorithm 4, off by default
 * (max_ns = 0). While set, every thread of the bottom-up construct waits a
 * pseudo-random time of up to max_ns nanoseconds (drawn from `seed`, the
 * node and the level) before each exchange that decides which child's
 * thread carries on, so that nodes are completed in other orders than the
 * hardware's usual one; the tree must not change. Each wait is bounded (a
 * clock check with an iteration cap); max_ns above 10^6 -> LBVH_ERR_INVALID.
 * The paper has no counterpart: it tests Algorithm 4 under other
 * interleavings. Builds without the hook run kernels that carry no trace of
 * it. */
lbvh_status lbvh_test_construct_jitter(unsigned long long seed, unsigned max_ns);

/* ---------------------------------------------------------------- profiling */

/* Stage ids of lbvh_tree_stage_times (device time of one kernel launch, or of
 * one sort pass). */
enum {
    LBVH_STAGE_BOUNDS = 0,     /* scene bounds reduction */
    LBVH_STAGE_ENCODE = 1,     /* Morton codes + sort digit histograms */
    LBVH_STAGE_SORT0 = 2,      /* radix-sort pass k is LBVH_STAGE_SORT0 + k, k < 8 */
    LBVH_STAGE_CONSTRUCT = 10, /* Algorithm 4: nodes, boxes, skips */
    LBVH_STAGE_QCOUNT = 11,    /* Algorithm 1 walk: counts, short sorted hit lists */
    LBVH_STAGE_QSCAN = 12,     /* exclusive scan of the counts */
    LBVH_STAGE_QFILL = 13,     /* short lists copied to their CSR positions */
    LBVH_STAGE_QFIXUP = 14,    /* second walk + sort for lists longer than 32 */
    LBVH_STAGE_QORDER = 15,    /* Morton order of the query centres (encode + sort) */
    LBVH_STAGE_SECOND = 16,    /* second pass of lbvh_build_variant's Karras / Apetrei builds */
    LBVH_STAGE_SORTRUNS = 17,  /* codes wider than 30 bits: the sort passes cover the codes' top bits
                                  beside the index; this stage orders the runs of equal top bits */
    LBVH_STAGE_COUNT = 18
};

/* Turn per-stage timing of this tree's builds and queries on or off (off by
 * default). When on, a CUDA event pair is recorded around each stage on the
 * stream the stage runs on. */
lbvh_status lbvh_tree_set_profiling(lbvh_tree_t tree, int on);

/* Device milliseconds of each stage of the tree's last build and last query
 * (ms: float[LBVH_STAGE_COUNT]; NaN for a stage that did not run or was not
 * timed). Synchronises the streams involved. */
lbvh_status lbvh_tree_stage_times(lbvh_tree_t tree, float *ms);

/* Name of a stage id ("" if unknown). */
const char *lbvh_stage_name(int stage);

/* Number of CUDA kernels this library has launched in this process. */
uint64_t lbvh_kernel_launches(void);

/* ---------------------------------------------------------------- autotuner */

/* The library's own tuning parameters, none of which changes any result (the
 * paper has no counterpart; they choose how the kernels run):
 *   sort variant  the radix sort's tile shape (keys per thread, CTAs per SM)
 *                 and how a warp finds the lanes sharing a digit (eight
 *                 ballots, or a per-warp table in shared memory), an index
 *                 in [0, lbvh_sort_variant_count()): with V =
 *                 lbvh_sort_variant_count() / 2, variant v takes tile shape
 *                 v % V, and for codes wider than 30 bits v >= V sorts one
 *                 byte (one pass) fewer of the codes' top bits, leaving more
 *                 elements in runs of equal sorted bits for the runs stage
 *                 (Sec. 3.1 step 2 either way: the same sorted order);
 *   walk variant  how Algorithm 1's collecting walk runs: 0 one thread per
 *                 query, 1/2/3 groups of 8/16/32 lanes walking the union of
 *                 their queries' paths together, 4 one thread per query in
 *                 CTAs of 512 threads instead of 256; 5-9 the same with the
 *                 queries put in the Morton order of 24-bit codes of their
 *                 centres (one sort pass fewer) instead of 30-bit ones
 *                 (lbvh_walk_variant_count() = 10).
 * A process-wide cache holds the choice for each configuration (the GPU's
 * name, ceil(log2 n), Morton bits, primitive kind, query kind, trees built
 * together); builds and queries use the cached choice for their
 * configuration, else variant 0. */
int lbvh_sort_variant_count(void);
int lbvh_walk_variant_count(void);

/* Times every sort variant on this build (two builds each, device time of
 * the sort passes and the runs stage) and, when nq > 0, every walk variant on these queries
 * (two runs each, device time of the query order and the collecting walk),
 * stores the fastest of each in the cache and leaves the tree built with the
 * chosen sort variant.
 * Arguments as lbvh_build and lbvh_query_into; sort_variant / walk_variant
 * (nullable) receive the choices. Synchronises `stream`. */
lbvh_status lbvh_tree_autotune(lbvh_tree_t tree, const float *d_prims, int64_t n, int kind, int morton_bits,
                               const float *d_queries, int64_t nq, int query_kind, const float *d_radii,
                               float radius, lbvh_stream_t stream, int *sort_variant, int *walk_variant);

/* Fix this tree's variants (-1: use the cache; LBVH_ERR_INVALID if out of
 * range). Every variant gives the same, exact results. */
lbvh_status lbvh_tree_set_tuning(lbvh_tree_t tree, int sort_variant, int walk_variant);

/* The cache as a small JSON file: save writes every entry (atomically, via a
 * temporary file beside `path`); load merges a saved file's entries into the
 * cache, dropping variant indices this library does not have
 * (LBVH_ERR_INVALID if the file cannot be read or parsed; the cache is then
 * unchanged). clear empties the cache; entries counts it. */
lbvh_status lbvh_tune_save(const char *path);
lbvh_status lbvh_tune_load(const char *path);
void lbvh_tune_clear(void);
int lbvh_tune_entries(void);

/* ---------------------------------------------------------------- misc */

/* Human-readable name of a status. */
const char *lbvh_status_str(lbvh_status status);

/* Text of the last CUDA runtime error seen by this thread ("" if none). */
const char *lbvh_last_cuda_error(void);

#ifdef __cplusplus
}
#endif

#endif /* LBVH_H */
