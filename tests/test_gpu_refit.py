"""Refit on the GPU (lbvh_refit) against the oracle's refit, bit-exact: the
topology of the original build is kept and every box is recomputed from the
moved primitives; queries on the refitted tree equal brute force on them."""
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


def assert_tree_equal(g, o):
    for k in ("perm", "sorted", "left", "skip_internal", "skip_leaf"):
        assert np.array_equal(g[k], o[k]), k
    for k in ("internal_box", "leaf_box", "bounds"):
        assert np.array_equal(np.asarray(g[k]).view(np.uint32), np.asarray(o[k]).view(np.uint32)), k


def moved(prims, kind, sigma, seed):
    rng = np.random.default_rng(seed)
    d = rng.normal(0, sigma, size=(prims.shape[0], 3))
    if kind == 1:
        d = np.concatenate([d, d], axis=1)
    return (prims + d).astype(np.float32)


@pytest.mark.parametrize("n,kind,bits", [(1, 0, 30), (2, 0, 30), (5000, 0, 63), (12289, 0, 30),
                                          (3073, 1, 63), (20000, 1, 30)])
def test_refit_matches_oracle(n, kind, bits):
    lbvh = L()
    a = inputs.uniform_points(n, seed=50 + n) if kind == 0 else inputs.gaussian_mixture_boxes(n, seed=50 + n)
    b = moved(a, kind, 0.02, 60 + n)
    t = lbvh.Tree().build(a, kind, bits)
    db = torch.from_numpy(b).cuda()
    t.refit(db)
    t.check()
    want = oracle.refit(oracle.build(a, kind, bits), b)
    assert_tree_equal(t.export(), want)
    # queries on the refitted tree: the moved primitives, exactly
    if kind == 0:
        q = inputs.uniform_points(min(n, 2000), seed=70)
        r = np.float32(0.05)
        off, hits = t.query(q, lbvh.SPHERE, radius=float(r))
        ooff, ohits = oracle.query(want, q, oracle.SPHERE, radius=r)
        if n <= 4096:
            boff, bhits = oracle.bruteforce(b, oracle.POINTS, q, oracle.SPHERE, radius=r)
            assert np.array_equal(ooff, boff) and np.array_equal(ohits, bhits)
    else:
        q = inputs.gaussian_mixture_boxes(min(n, 2000), seed=71, component_seed=50 + n)
        off, hits = t.query(q, lbvh.BOX)
        ooff, ohits = oracle.query(want, q, oracle.BOX)
    assert np.array_equal(off.cpu().numpy(), ooff)
    assert np.array_equal(hits.cpu().numpy().view(np.uint32), ohits)


def test_refit_twice_and_back_to_the_original():
    lbvh = L()
    a = inputs.uniform_points(9000, seed=80)
    t = lbvh.Tree().build(a, lbvh.POINTS, 63)
    first = t.export()
    t.refit(moved(a, 0, 0.2, 81))
    t.refit(moved(a, 0, 0.01, 82))
    t.refit(torch.from_numpy(a).cuda())
    assert_tree_equal(t.export(), first)


def test_refit_self_query_uses_the_new_points():
    # a tree queried with the buffer it was refitted from takes the build's
    # permutation as query order: results must still be those of the new points
    lbvh = L()
    a = inputs.uniform_points(6000, seed=83)
    b = moved(a, 0, 0.05, 84)
    t = lbvh.Tree().build(a, lbvh.POINTS, 30)
    db = torch.from_numpy(b).cuda()
    t.refit(db)
    r = float(inputs.radius_for_neighbours(6000))
    off, hits = t.query(db, lbvh.SPHERE, radius=r)
    ooff, ohits = oracle.query(oracle.refit(oracle.build(a, oracle.POINTS, 30), b), b, oracle.SPHERE,
                               radius=np.float32(r))
    assert np.array_equal(off.cpu().numpy(), ooff)
    assert np.array_equal(hits.cpu().numpy().view(np.uint32), ohits)


def test_refit_errors():
    lbvh = L()
    lib = lbvh.load()
    h = lbvh.Tree()
    assert lib.lbvh_refit(h._h, None, None) == lbvh.ERR_INVALID  # never built
    a = inputs.uniform_points(3000, seed=85)
    t = lbvh.Tree().build(a, lbvh.POINTS, 30)
    bad = a.copy()
    bad[1234, 1] = np.nan
    t.refit(bad)
    assert t.status() == lbvh.ERR_NONFINITE
    t.refit(a)  # a good refit clears the latched error
    t.check()
