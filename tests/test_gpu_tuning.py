"""The autotuner's variants against the oracle: every sort variant (tile
shape, digit-peer ranking) gives the oracle's tree and every walk variant
(one thread per query, or groups of 8/16/32 lanes walking together) gives
the oracle's CSR, bit-exact, including lists longer than the walk's slot and
ray queries; lbvh_tree_autotune picks valid variants, fills the cache, and a
saved cache loads back into a fresh cache."""
from __future__ import annotations

import json
import math

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


def assert_tree_equal(g, o):
    for k in ("perm", "sorted", "left", "skip_internal", "skip_leaf"):
        assert np.array_equal(g[k], o[k]), k
    for k in ("internal_box", "leaf_box", "bounds"):
        assert np.array_equal(np.asarray(g[k]).view(np.uint32), np.asarray(o[k]).view(np.uint32)), k


CASES = {
    "uniform_63bit": lambda: (inputs.uniform_points(70001, seed=21), 0, 63),
    "mixture_boxes_30bit": lambda: (inputs.gaussian_mixture_boxes(60000, seed=22), 1, 30),
    "duplicates_63bit": lambda: (inputs.duplicated_points(30000, 100, seed=23), 0, 63),
    "uniform_39bit": lambda: (inputs.uniform_points(9000, seed=24), 0, 39),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_every_sort_variant_builds_the_oracle_tree(case):
    lbvh = L()
    prims, kind, bits = CASES[case]()
    o = oracle.build(prims, kind, bits)
    for v in range(lbvh.sort_variant_count()):
        t = lbvh.Tree()
        t.set_tuning(v, -1)
        t.build(prims, kind, bits)
        t.check()
        assert_tree_equal(t.export(), o)
        t.close()


@pytest.mark.parametrize("radius", [0.03, 0.2])
def test_every_walk_variant_gives_the_oracle_csr_on_points(radius):
    lbvh = L()
    n = 20001  # not a multiple of a warp: the last warp has lanes without a query
    pts = inputs.uniform_points(n, seed=31)
    q = inputs.uniform_points(n, seed=32)
    o = oracle.build(pts, oracle.POINTS, 30)
    ooff, ohits = oracle.query(o, q, oracle.SPHERE, radius=radius)
    assert (np.diff(ooff) > 64).any() == (radius > 0.1)  # the large radius spills past the slot
    for w in range(lbvh.walk_variant_count()):
        t = lbvh.Tree()
        t.set_tuning(-1, w)
        t.build(pts, lbvh.POINTS, 30)
        off, hits = t.query(q, lbvh.SPHERE, radius=radius)
        assert np.array_equal(off.cpu().numpy(), ooff), w
        assert np.array_equal(hits.cpu().numpy().view(np.uint32), ohits), w
        t.close()


def test_every_walk_variant_on_boxes_and_rays():
    lbvh = L()
    prims = inputs.gaussian_mixture_boxes(30000, seed=41, components=16, log_half_mu=math.log(0.002))
    bq = inputs.gaussian_mixture_boxes(5003, seed=42, component_seed=41, components=16,
                                       log_half_mu=math.log(0.002))
    rays = inputs.random_rays(3001, seed=43, tmax=0.2)
    o = oracle.build(prims, oracle.BOXES, 63)
    want_b = oracle.query(o, bq, oracle.BOX)
    want_r = oracle.query(o, rays, oracle.RAY)
    for w in range(lbvh.walk_variant_count()):
        t = lbvh.Tree()
        t.set_tuning(-1, w)
        t.build(prims, lbvh.BOXES, 63)
        for qs, qk, want in ((bq, lbvh.BOX, want_b), (rays, lbvh.RAY, want_r)):
            off, hits = t.query(qs, qk)
            assert np.array_equal(off.cpu().numpy(), want[0]), (w, qk)
            assert np.array_equal(hits.cpu().numpy().view(np.uint32), want[1]), (w, qk)
        t.close()


def test_set_tuning_rejects_out_of_range():
    lbvh = L()
    t = lbvh.Tree()
    with pytest.raises(lbvh.LbvhError):
        t.set_tuning(lbvh.sort_variant_count(), -1)
    with pytest.raises(lbvh.LbvhError):
        t.set_tuning(-1, lbvh.walk_variant_count())
    with pytest.raises(lbvh.LbvhError):
        t.set_tuning(-2, -1)
    t.close()


def test_autotune_fills_the_cache_and_the_cache_survives_a_file(tmp_path):
    lbvh = L()
    lbvh.tune_clear()
    n = 1 << 18
    pts = inputs.uniform_points(n, seed=51)
    r = inputs.radius_for_neighbours(n)
    t = lbvh.Tree()
    sv, wv = t.autotune(pts, lbvh.POINTS, 63, queries=pts, qkind=lbvh.SPHERE, radius=float(r))
    assert 0 <= sv < lbvh.sort_variant_count() and 0 <= wv < lbvh.walk_variant_count()
    assert lbvh.tune_entries() == 2  # the build's sort and the sphere walk
    # the tree is left built, and a build with the cached choice matches the oracle
    t.check()
    o = oracle.build(pts, oracle.POINTS, 63)
    assert_tree_equal(t.export(), o)
    t.build(pts, lbvh.POINTS, 63)
    assert_tree_equal(t.export(), o)
    path = str(tmp_path / "tune.json")
    lbvh.tune_save(path)
    saved = json.load(open(path))
    assert len(saved["entries"]) == 2
    assert {e["sort_variant"] for e in saved["entries"]} >= {sv}
    lbvh.tune_clear()
    assert lbvh.tune_entries() == 0
    lbvh.tune_load(path)
    assert lbvh.tune_entries() == 2
    lbvh.tune_clear()
    t.close()


def test_walk_visits_counts_the_nodes_algorithm_1_visits():
    """lbvh_tree_walk_visits against Algorithm 1 walked in Python over the
    oracle's canonical arrays (leaves and internal nodes counted apart)."""
    lbvh = L()
    n = 3000
    pts = inputs.uniform_points(n, seed=61)
    q = inputs.uniform_points(400, seed=62)
    r = 0.06
    o = oracle.build(pts, oracle.POINTS, 30)
    ni = n - 1
    leaf_box, ibox = o["leaf_box"], o["internal_box"]
    want_l = want_i = 0
    r2 = np.float32(r) * np.float32(r)
    for c in q:
        node = 0
        while node != -1:
            leaf = node >= ni
            box = leaf_box[node - ni] if leaf else ibox[node]
            hit = oracle.sphere_box(c, r, box)
            if leaf:
                want_l += 1
                node = o["skip_leaf"][node - ni]
            else:
                want_i += 1
                node = o["left"][node] if hit else o["skip_internal"][node]
    t = lbvh.Tree().build(pts, lbvh.POINTS, 30)
    assert t.walk_visits(q, lbvh.SPHERE, radius=r) == (want_l, want_i)
    t.close()
