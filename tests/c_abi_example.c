/* A plain C program against include/lbvh.h and the built library, with no
 * Python or PyTorch: build a tree of points, query it, check every hit list
 * against a brute-force scan on the host, save and reload the tree. Used by
 * tests/test_gpu_c_abi.py; exits 0 on success. */
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "lbvh.h"

#define CHECK(x)                                                                      \
    do {                                                                              \
        lbvh_status st_ = (x);                                                        \
        if (st_ != LBVH_OK) {                                                         \
            fprintf(stderr, "%s:%d %s -> %s (%s)\n", __FILE__, __LINE__, #x,          \
                    lbvh_status_str(st_), lbvh_last_cuda_error());                    \
            return 1;                                                                 \
        }                                                                             \
    } while (0)

static uint64_t rng = 88172645463325252ull; /* xorshift64, fixed seed */
static float uniform(void) {
    rng ^= rng << 13;
    rng ^= rng >> 7;
    rng ^= rng << 17;
    return (float)(rng >> 40) / (float)(1u << 24);
}

static int cmp_u32(const void *a, const void *b) {
    uint32_t x = *(const uint32_t *)a, y = *(const uint32_t *)b;
    return x < y ? -1 : x > y;
}

int main(void) {
    const int64_t n = 20000, nq = 2000;
    const float r = 0.04f;
    float *h_pts = malloc(sizeof(float) * 3 * n);
    for (int64_t i = 0; i < 3 * n; ++i) h_pts[i] = uniform();
    float *d_pts = NULL;
    int64_t *d_off = NULL;
    uint32_t *d_hits = NULL;
    const uint64_t cap = 64 * (uint64_t)nq;
    if (cudaMalloc((void **)&d_pts, sizeof(float) * 3 * n) != cudaSuccess) return 2;
    if (cudaMalloc((void **)&d_off, sizeof(int64_t) * (nq + 1)) != cudaSuccess) return 2;
    if (cudaMalloc((void **)&d_hits, sizeof(uint32_t) * cap) != cudaSuccess) return 2;
    cudaMemcpy(d_pts, h_pts, sizeof(float) * 3 * n, cudaMemcpyHostToDevice);

    lbvh_tree_t tree = NULL;
    CHECK(lbvh_tree_create(&tree));
    CHECK(lbvh_build(tree, d_pts, n, LBVH_PRIM_POINTS, 63, NULL));
    CHECK(lbvh_tree_status(tree));
    uint64_t total = 0;
    /* the first nq points are the query centres */
    CHECK(lbvh_query_into(tree, d_pts, nq, LBVH_Q_SPHERE, NULL, r, d_off, d_hits, cap, &total, NULL));
    cudaDeviceSynchronize();
    int64_t *off = malloc(sizeof(int64_t) * (nq + 1));
    uint32_t *hits = malloc(sizeof(uint32_t) * (total ? total : 1));
    cudaMemcpy(off, d_off, sizeof(int64_t) * (nq + 1), cudaMemcpyDeviceToHost);
    cudaMemcpy(hits, d_hits, sizeof(uint32_t) * total, cudaMemcpyDeviceToHost);

    /* brute force: the closed ball, d2 = fma(ez, ez, fma(ey, ey, ex*ex)) as in lbvh.h */
    uint32_t *want = malloc(sizeof(uint32_t) * n);
    for (int64_t q = 0; q < nq; ++q) {
        int64_t m = 0;
        const float *c = h_pts + 3 * q;
        for (int64_t j = 0; j < n; ++j) {
            const float *p = h_pts + 3 * j;
            float ex = p[0] - c[0], ey = p[1] - c[1], ez = p[2] - c[2];
            if (ex < 0) ex = -ex;
            if (ey < 0) ey = -ey;
            if (ez < 0) ez = -ez;
            float d2 = __builtin_fmaf(ez, ez, __builtin_fmaf(ey, ey, ex * ex));
            if (d2 <= r * r) want[m++] = (uint32_t)j;
        }
        qsort(want, (size_t)m, sizeof(uint32_t), cmp_u32);
        if (off[q + 1] - off[q] != m || memcmp(hits + off[q], want, sizeof(uint32_t) * (size_t)m) != 0) {
            fprintf(stderr, "query %lld differs from brute force\n", (long long)q);
            return 1;
        }
    }

    /* checkpoint round trip: the reloaded tree answers the same */
    uint64_t bytes = 0;
    CHECK(lbvh_tree_save(tree, NULL, 0, &bytes));
    void *image = malloc(bytes);
    CHECK(lbvh_tree_save(tree, image, bytes, &bytes));
    lbvh_tree_t back = NULL;
    CHECK(lbvh_tree_create(&back));
    CHECK(lbvh_tree_load(back, image, bytes, NULL));
    uint64_t total2 = 0;
    CHECK(lbvh_query_into(back, d_pts, nq, LBVH_Q_SPHERE, NULL, r, d_off, d_hits, cap, &total2, NULL));
    if (total2 != total) {
        fprintf(stderr, "reloaded tree: %llu hits, expected %llu\n", (unsigned long long)total2,
                (unsigned long long)total);
        return 1;
    }
    lbvh_tree_destroy(back);
    lbvh_tree_destroy(tree);
    printf("c abi ok: %lld queries, %llu hits, image %llu bytes, %llu kernels\n", (long long)nq,
           (unsigned long long)total, (unsigned long long)bytes, (unsigned long long)lbvh_kernel_launches());
    free(image);
    free(want);
    free(hits);
    free(off);
    free(h_pts);
    cudaFree(d_pts);
    cudaFree(d_off);
    cudaFree(d_hits);
    return 0;
}
