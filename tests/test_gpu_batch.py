"""Batched build + query (many independent trees in one pass, one CUDA graph)
against single-instance builds and the oracle: every instance's tree and hit
lists must be identical to building and querying that instance alone."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2402_00665_gb300 import _build, inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    _build.build()
    from paper_2402_00665_gb300 import lbvh
    return lbvh.load()


def L():
    from paper_2402_00665_gb300 import lbvh
    return lbvh


def offsets_of(sizes):
    return np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)


def csr_segments(off, hits, lo, hi):
    off = off.cpu().numpy()
    hits = hits.cpu().numpy().view(np.uint32)
    return [hits[off[q]:off[q + 1]] for q in range(lo, hi)]


def assert_tree_equal(g, o):
    for k in ("perm", "sorted", "left", "skip_internal", "skip_leaf"):
        assert np.array_equal(g[k], o[k]), k
    for k in ("internal_box", "leaf_box"):
        assert np.array_equal(np.asarray(g[k]).view(np.uint32), np.asarray(o[k]).view(np.uint32)), k


def run_and_compare(sizes, kind, bits, qkind, self_query, seed, qsizes=None):
    lbvh = L()
    po = offsets_of(sizes)
    n = int(po[-1])
    if kind == lbvh.POINTS:
        prims = inputs.uniform_points(n, seed=seed)
    else:
        prims = inputs.gaussian_mixture_boxes(n, seed=seed, components=16)
    dp = torch.from_numpy(prims).cuda()
    if self_query:
        dq, qo = dp, po
        queries = prims
    else:
        qo = offsets_of(qsizes if qsizes is not None else sizes)
        nq = int(qo[-1])
        if qkind == lbvh.SPHERE:
            queries = inputs.uniform_points(nq, seed=seed + 1)
        else:
            queries = inputs.gaussian_mixture_boxes(nq, seed=seed + 1, components=16, component_seed=seed)
        dq = torch.from_numpy(queries).cuda()
    nq = int(qo[-1])
    radii = None
    if qkind == lbvh.SPHERE:
        per_inst = np.array([inputs.radius_for_neighbours(max(int(s), 1)) for s in sizes], np.float32)
        radii_h = np.repeat(per_inst, np.diff(qo)).astype(np.float32)
        radii = torch.from_numpy(radii_h).cuda()
    b = lbvh.Batch()
    off, hits, total, st = b.build_query(dp, po, kind, bits, dq, qo, qkind, radii=radii, capacity=40 * nq + 64)
    assert st == lbvh.OK
    # the graph replay gives the same result
    off2, hits2, total2, st2 = b.build_query(dp, po, kind, bits, dq, qo, qkind, radii=radii, capacity=40 * nq + 64)
    assert st2 == lbvh.OK and total2 == total
    assert torch.equal(off, off2) and torch.equal(hits[:total], hits2[:total])
    hits = hits[:total]
    for inst in range(len(sizes)):
        a, e = int(po[inst]), int(po[inst + 1])
        qa, qe = int(qo[inst]), int(qo[inst + 1])
        if e - a == 0:
            assert all(len(x) == 0 for x in csr_segments(off, hits, qa, qe))
            continue
        t = lbvh.Tree().build(dp[a:e], kind, bits)
        assert_tree_equal(b.export(inst), t.export())
        if qe > qa:
            r = None if radii is None else radii[qa:qe]
            toff, thits = t.query(dq[qa:qe], qkind, radii=r)
            assert [x.tolist() for x in csr_segments(off, hits, qa, qe)] == \
                   [x.tolist() for x in csr_segments(toff, thits, 0, qe - qa)], f"instance {inst}"
        if e - a <= 3000 and inst % 3 == 0:
            o = oracle.build(prims[a:e], kind, bits)
            assert_tree_equal(b.export(inst), o)
    return b


def test_batch_points_self_query_mixed_sizes():
    sizes = [0, 1, 2, 3, 17, 256, 1000, 4097, 20000, 5, 0, 9000]
    run_and_compare(sizes, 0, 30, 0, True, seed=1)


def test_batch_points_separate_queries_63bit():
    sizes = [300, 7000, 1, 64, 12345]
    run_and_compare(sizes, 0, 51, 0, False, seed=2, qsizes=[10, 5000, 3, 0, 7000])


# Instances whose sizes sit on and around the sort's tile sizes (2048, 3072
# and 4096 keys), so tiles of one instance end exactly at, or one key past, a
# tile boundary; 63-bit codes with many instances (each instance's codes are
# sorted apart, so the code width does not limit the instance count).
TILE_EDGE_SIZES = [3071, 3072, 3073, 6144, 6145, 2047, 2048, 2049, 4095, 4096, 4097, 1, 0, 2, 12289]


def test_batch_63bit_many_instances_tile_edges():
    rng = np.random.default_rng(8)
    sizes = TILE_EDGE_SIZES + [int(x) for x in rng.integers(1, 900, size=40)]
    run_and_compare(sizes, 0, 63, 0, True, seed=8)


def test_batch_boxes_63bit_tile_edges():
    run_and_compare(TILE_EDGE_SIZES, 1, 63, 1, False, seed=9, qsizes=[s // 2 for s in TILE_EDGE_SIZES])


def test_batch_boxes_box_queries():
    sizes = [2000, 1, 5000, 3, 10000]
    run_and_compare(sizes, 1, 30, 1, False, seed=3, qsizes=[700, 2, 1500, 0, 3000])


def test_batch_many_small_instances_and_autotune():
    rng = np.random.default_rng(4)
    sizes = np.floor(np.exp(rng.uniform(np.log(16), np.log(3000), size=600))).astype(np.int64)
    sizes[::50] = 0
    b = run_and_compare(list(sizes), 0, 30, 0, True, seed=4)
    assert b.sort_variant() >= -1


def test_batch_large_triggers_autotune_and_graph_picks_up_new_data():
    lbvh = L()
    sizes = [1 << 19, 1 << 19, 123457]
    po = offsets_of(sizes)
    n = int(po[-1])
    dp = torch.from_numpy(inputs.uniform_points(n, seed=5)).cuda()
    b = lbvh.Batch()
    off, hits, total, st = b.build_query(dp, po, lbvh.POINTS, 30, radius=0.01, capacity=40 * n)
    assert st == lbvh.OK and b.sort_variant() >= 0
    # same buffers, new contents: the recorded graph reads the new points
    dp.copy_(torch.from_numpy(inputs.uniform_points(n, seed=6)).cuda())
    off, hits, total, st = b.build_query(dp, po, lbvh.POINTS, 30, radius=0.01, capacity=40 * n)
    assert st == lbvh.OK
    t = lbvh.Tree().build(dp[po[1]:po[2]], lbvh.POINTS, 30)
    toff, thits = t.query(dp[po[1]:po[2]], lbvh.SPHERE, radius=0.01)
    got = csr_segments(off, hits[:total], int(po[1]), int(po[2]))
    want = csr_segments(toff, thits, 0, sizes[1])
    assert all(np.array_equal(x, y) for x, y in zip(got, want))


def test_batch_long_hit_lists():
    # per-instance radii that give lists of ~30-90 hits (register and warp
    # sorts, and the second walk), ~190 (warp sort after the second walk), a
    # few thousand (CTA sort in shared memory) and all 12,000 points (CTA sort
    # in global memory)
    lbvh = L()
    sizes = [3000, 12000, 500, 6000]
    rads = [0.17, 2.0, 0.45, 0.5]
    po = offsets_of(sizes)
    pts = inputs.uniform_points(int(po[-1]), seed=21)
    qsizes = [300, 40, 50, 200]
    qo = offsets_of(qsizes)
    q = np.concatenate([pts[po[k]:po[k] + qsizes[k]] for k in range(len(sizes))])
    radii = np.repeat(np.array(rads, np.float32), qsizes)
    b = lbvh.Batch()
    cap = int(sum(qs * n for qs, n in zip(qsizes, sizes)))
    off, hits, total, st = b.build_query(torch.from_numpy(pts).cuda(), po, lbvh.POINTS, 30,
                                         torch.from_numpy(q).cuda(), qo, lbvh.SPHERE,
                                         radii=torch.from_numpy(radii).cuda(), capacity=cap)
    assert st == lbvh.OK
    hits = hits[:total]
    for k in range(len(sizes)):
        o = oracle.build(pts[po[k]:po[k + 1]], oracle.POINTS, 30)
        ooff, ohits = oracle.query(o, q[qo[k]:qo[k + 1]], oracle.SPHERE, radius=np.float32(rads[k]))
        got = csr_segments(off, hits, int(qo[k]), int(qo[k + 1]))
        want = [ohits[ooff[j]:ooff[j + 1]] for j in range(qsizes[k])]
        assert all(np.array_equal(x, y) for x, y in zip(got, want)), k
        assert max(len(x) for x in want) > 32


def test_batch_capacity_error():
    lbvh = L()
    sizes = [5000, 3000]
    po = offsets_of(sizes)
    dp = torch.from_numpy(inputs.uniform_points(8000, seed=7)).cuda()
    b = lbvh.Batch()
    off, hits, total, st = b.build_query(dp, po, lbvh.POINTS, 30, radius=0.05, capacity=100)
    assert st == lbvh.ERR_CAPACITY and total > 100
    off, hits, total2, st = b.build_query(dp, po, lbvh.POINTS, 30, radius=0.05, capacity=total)
    assert st == lbvh.OK and total2 == total
