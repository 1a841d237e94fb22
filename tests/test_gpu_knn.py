"""k nearest neighbours (lbvh_knn: Algorithm 1 with a shrinking ball) on the
GPU against the oracle's brute force, bit-exact (indices and squared
distances, rows in the order (d2, index)): D1's points, Gaussian-mixture
boxes at 63 and 30 bits, k in {1, 16, 64, 256}, ties, padding, non-finite
queries and a tree built from caller codes (no Morton seeding)."""
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


def check_knn(t, prims, kind, q, k, want=None):
    """GPU rows against the oracle's (or a given oracle result's first k columns)."""
    idx, d2 = t.knn(q, k)
    if want is None:
        want = oracle.knn(prims, kind, q, k)
    wi, wd = want[0][:, :k], want[1][:, :k]
    gi = idx.cpu().numpy().view(np.uint32)
    gd = d2.cpu().numpy()
    bad = np.nonzero((gi != wi).any(axis=1))[0]
    assert len(bad) == 0, (k, bad[:5], gi[bad[:1]], wi[bad[:1]])
    assert np.array_equal(gd.view(np.uint32), wd.view(np.uint32)), k


def test_knn_d1_all_queries():
    """D1: 16,384 uniform points, 30-bit codes, every point as a query."""
    lbvh = L()
    pts = inputs.uniform_points(16384, seed=0)
    t = lbvh.Tree().build(pts, lbvh.POINTS, 30)
    want = oracle.knn(pts, oracle.POINTS, pts, 64)
    for k in (1, 16, 64):
        check_knn(t, pts, oracle.POINTS, pts, k, want)
    # the nearest point of each query is itself (distance 0; a duplicate with a
    # lower index would come first, and uniform floats have none here)
    assert (want[0][:, 0] == np.arange(16384)).all()


@pytest.mark.parametrize("bits", [63, 30])
def test_knn_mixture_boxes(bits):
    lbvh = L()
    n = 1 << 20
    boxes = inputs.gaussian_mixture_boxes(n, seed=3)
    t = lbvh.Tree().build(boxes, lbvh.BOXES, bits)
    rng = np.random.default_rng(4)
    qb = inputs.gaussian_mixture_boxes(384, seed=5, component_seed=3)
    q = np.concatenate([(qb[:, :3] + qb[:, 3:]) * np.float32(0.5), rng.random((128, 3), dtype=np.float32)])
    want = oracle.knn(boxes, oracle.BOXES, q, 64)
    for k in (1, 16, 64):
        check_knn(t, boxes, oracle.BOXES, q, k, want)


def test_knn_largest_k_and_padding():
    lbvh = L()
    pts = inputs.uniform_points(3000, seed=6)
    q = inputs.uniform_points(700, seed=7)
    t = lbvh.Tree().build(pts, lbvh.POINTS, 63)
    check_knn(t, pts, oracle.POINTS, q, lbvh.KNN_MAX_K)
    small = inputs.uniform_points(5, seed=8)
    t2 = lbvh.Tree().build(small, lbvh.POINTS, 63)
    check_knn(t2, small, oracle.POINTS, q[:50], 9)  # k > n: padded rows
    one = inputs.uniform_points(1, seed=9)
    t3 = lbvh.Tree().build(one, lbvh.POINTS, 30)
    check_knn(t3, one, oracle.POINTS, q[:40], 3)
    with pytest.raises(lbvh.LbvhError):
        t.knn(q, lbvh.KNN_MAX_K + 1)
    with pytest.raises(lbvh.LbvhError):
        t.knn(q, 0)


def test_knn_ties_duplicates_and_non_finite_queries():
    lbvh = L()
    same = np.full((2000, 3), 0.25, np.float32)  # every distance ties: index order
    t = lbvh.Tree().build(same, lbvh.POINTS, 63)
    q = np.array([[0.25, 0.25, 0.25], [0.9, 0.1, 0.5], [np.nan, 0.5, 0.5], [0.5, -np.inf, 0.5]], np.float32)
    check_knn(t, same, oracle.POINTS, q, 16)
    dup = inputs.duplicated_points(20000, 300, seed=10)
    t2 = lbvh.Tree().build(dup, lbvh.POINTS, 30)
    qd = np.concatenate([dup[:200], inputs.uniform_points(200, seed=11), q[2:]])
    check_knn(t2, dup, oracle.POINTS, qd, 64)
    # boxes holding the query: distance 0, index order among them
    boxes = inputs.gaussian_mixture_boxes(5000, seed=12, components=4, sigma=0.001, log_half_mu=np.log(0.01))
    t3 = lbvh.Tree().build(boxes, lbvh.BOXES, 30)
    qc = (boxes[:300, :3] + boxes[:300, 3:]) * np.float32(0.5)
    check_knn(t3, boxes, oracle.BOXES, qc, 16)


def test_knn_without_morton_seeds_is_still_exact():
    """A tree built from caller codes (no Morton grid): walks start from the
    first k leaves instead of the query's place in Morton order."""
    lbvh = L()
    n = 8000
    pts = inputs.uniform_points(n, seed=13)
    codes, _ = oracle.morton_codes(pts, oracle.POINTS, 63)
    perm = np.argsort(codes, kind="stable").astype(np.uint32)
    t = lbvh.Tree().build_from_sorted(codes[perm], perm, pts, lbvh.POINTS)
    q = inputs.uniform_points(500, seed=14)
    check_knn(t, pts, oracle.POINTS, q, 16)


def test_knn_no_queries_and_unbuilt_tree():
    lbvh = L()
    t = lbvh.Tree()
    with pytest.raises(lbvh.LbvhError):
        t.knn(np.zeros((3, 3), np.float32), 4)
    t.build(inputs.uniform_points(100, seed=1), lbvh.POINTS, 30)
    idx, d2 = t.knn(np.zeros((0, 3), np.float32), 4)
    assert idx.shape == (0, 4)
