"""The Karras and Apetrei (Algorithm 3) hierarchy builds of lbvh_build_variant
against the oracle, bit-exact: the radix tree of the augmented keys is unique,
so every algorithm must end in the same Karras-ordered tree with the same
skips and boxes as Algorithm 4."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2402_00665_gb300 import _build, inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

ALGORITHMS = [1, 2]  # Karras, Apetrei


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


CASES = [
    ("uniform", 1, 0, 30), ("uniform", 2, 0, 30), ("uniform", 3, 0, 63), ("uniform", 100, 0, 30),
    ("uniform", 4097, 0, 63), ("uniform", 20000, 0, 30), ("mixture_boxes", 6000, 1, 30),
    ("mixture_boxes", 3000, 1, 63), ("duplicates", 5000, 0, 30), ("all_equal", 777, 0, 63),
    ("collinear", 2500, 0, 63), ("hollow_cube", 9000, 0, 30),
]


def make(name, n, seed):
    if name == "uniform":
        return inputs.uniform_points(n, seed=seed)
    if name == "mixture_boxes":
        return inputs.gaussian_mixture_boxes(n, seed=seed, components=8)
    if name == "duplicates":
        return inputs.duplicated_points(n, distinct=n // 10, seed=seed)
    if name == "all_equal":
        return np.full((n, 3), 0.25, np.float32)
    if name == "collinear":
        return inputs.collinear_points(n, seed=seed)
    return inputs.hollow_cube(n, seed=seed)


@pytest.mark.parametrize("algorithm", ALGORITHMS)
@pytest.mark.parametrize("name,n,kind,bits", CASES)
def test_variant_build_matches_oracle(algorithm, name, n, kind, bits):
    lbvh = L()
    prims = make(name, n, 90 + n)
    t = lbvh.Tree().build(prims, kind, bits, algorithm=algorithm)
    t.check()
    o = oracle.build(prims, kind, bits)
    assert_tree_equal(t.export(), o)
    if kind == 0 and n > 1:
        q = prims[:: max(1, n // 500)]
        r = np.float32(inputs.radius_for_neighbours(n))
        off, hits = t.query(q, lbvh.SPHERE, radius=float(r))
        ooff, ohits = oracle.query(o, q, oracle.SPHERE, radius=r)
        assert np.array_equal(off.cpu().numpy(), ooff)
        assert np.array_equal(hits.cpu().numpy().view(np.uint32), ohits)


@pytest.mark.parametrize("algorithm", ALGORITHMS)
def test_variant_full_size_equals_algorithm4(algorithm):
    # 2^25 points at 63 bits (the bench configuration): the variant's tree
    # equals the Algorithm 4 tree (itself checked against the oracle at this
    # size in test_gpu_full_size.py)
    lbvh = L()
    n = 1 << 25
    pts = torch.from_numpy(inputs.uniform_points(n, seed=0)).cuda()
    a = lbvh.Tree().build(pts, lbvh.POINTS, 63)
    a.check()
    ea = a.export()
    a.close()
    b = lbvh.Tree().build(pts, lbvh.POINTS, 63, algorithm=algorithm)
    b.check()
    eb = b.export()
    b.close()
    assert_tree_equal(eb, ea)


def test_variant_rejects_unknown_algorithm():
    lbvh = L()
    lib = lbvh.load()
    t = lbvh.Tree()
    pts = torch.from_numpy(inputs.uniform_points(100, seed=1)).cuda()
    import ctypes
    st = lib.lbvh_build_variant(t._h, ctypes.c_void_p(pts.data_ptr()), 100, 0, 30, 3, None)
    assert st == lbvh.ERR_INVALID
