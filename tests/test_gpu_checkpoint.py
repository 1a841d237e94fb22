"""Checkpoint images (lbvh_tree_save / lbvh_tree_load): a loaded tree equals
the saved one bit for bit, answers the same queries, and refits like it."""
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


def same(a, b):
    for k in ("perm", "sorted", "left", "skip_internal", "skip_leaf"):
        assert np.array_equal(a[k], b[k]), k
    for k in ("internal_box", "leaf_box", "bounds"):
        assert np.array_equal(np.asarray(a[k]).view(np.uint32), np.asarray(b[k]).view(np.uint32)), k


@pytest.mark.parametrize("n,kind,bits", [(0, 0, 30), (1, 0, 30), (2, 1, 63), (5000, 0, 63), (20000, 1, 30)])
def test_save_load_round_trip(n, kind, bits):
    lbvh = L()
    prims = inputs.uniform_points(n, seed=70) if kind == 0 else inputs.gaussian_mixture_boxes(n, seed=70)
    t = lbvh.Tree().build(prims, kind, bits)
    image = t.save()
    assert len(image) == 64 + 12 * n + (max(n - 1, 0) * 32 + n * (16 if kind == 0 else 32))
    u = lbvh.Tree().load(image)
    u.check()
    if n == 0:
        assert u.size() == 0
        return
    same(u.export(), t.export())
    same(u.export(), oracle.build(prims, kind, bits))
    if kind == 0:
        q = prims[:: max(1, n // 300)]
        r = float(inputs.radius_for_neighbours(max(n, 2)))
        a = t.query(q, lbvh.SPHERE, radius=r)
        b = u.query(q, lbvh.SPHERE, radius=r)
    else:
        q = prims[:300]
        a = t.query(q, lbvh.BOX)
        b = u.query(q, lbvh.BOX)
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
    # the loaded tree refits like the original (it carries codes and permutation)
    moved = (prims + np.float32(0.01)).astype(np.float32)
    t.refit(moved)
    u.refit(moved)
    same(u.export(), t.export())
    assert u.save() == t.save()


def test_load_rejects_a_damaged_image():
    lbvh = L()
    t = lbvh.Tree().build(inputs.uniform_points(1000, seed=71), lbvh.POINTS, 30)
    image = bytearray(t.save())
    u = lbvh.Tree()
    with pytest.raises(Exception):
        u.load(bytes(image[:-4]))      # truncated
    image[0] = ord("X")
    with pytest.raises(Exception):
        u.load(bytes(image))           # bad magic
