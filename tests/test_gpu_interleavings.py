"""Algorithm 4 under other orders of arrival (Sec. 4: at every node the
second thread up carries on, whichever child's it is). With
lbvh_test_construct_jitter set, every thread of the bottom-up construct
waits a bounded pseudo-random time before each exchange, so that nodes are
completed in orders the hardware does not usually produce; the tree stays
the oracle's, bit for bit, through both construct kernels (the build's,
which derives the codes itself, and the one that takes sorted codes), and
the next build without the hook is exact too. The waits are bounded: nothing
faults, traps or hangs."""
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
    for k in ("internal_box", "leaf_box"):
        assert np.array_equal(np.asarray(g[k]).view(np.uint32), np.asarray(o[k]).view(np.uint32)), k


def cases():
    rng = np.random.default_rng(90)
    few = rng.random((300, 3), dtype=np.float32)
    dup = few[rng.integers(0, 300, 20000)]  # many equal points: splits on the position bits
    return [
        ("uniform 70001, 63 bits", inputs.uniform_points(70001, seed=91), 0, 63),  # many groups, ragged tail
        ("duplicates 20000, 30 bits", dup, 0, 30),
        ("mixture boxes 40000, 30 bits", inputs.gaussian_mixture_boxes(40000, seed=92, components=8), 1, 30),
        ("uniform 257, 30 bits", inputs.uniform_points(257, seed=93), 0, 30),  # one group and one leaf
        ("uniform 2", inputs.uniform_points(2, seed=94), 0, 63),
    ]


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_jittered_arrivals_give_the_oracle_tree(lib, seed):
    lbvh = L()
    assert lib.lbvh_test_construct_jitter(seed, 20000) == lbvh.OK  # waits of up to 20 us
    try:
        for name, prims, kind, bits in cases():
            o = oracle.build(prims, kind, bits)
            t = lbvh.Tree().build(prims, kind, bits)  # the build's construct (codes derived again)
            t.check()
            assert_tree_equal(t.export(), o)
            t.close()
            t = lbvh.Tree().build_from_sorted(o["sorted"], o["perm"], prims, kind)  # from sorted codes
            t.check()
            e = t.export()
            for k in ("left", "skip_internal", "skip_leaf"):
                assert np.array_equal(e[k], o[k]), (name, k)
            assert np.array_equal(e["internal_box"].view(np.uint32), o["internal_box"].view(np.uint32)), name
            t.close()
    finally:
        assert lib.lbvh_test_construct_jitter(0, 0) == lbvh.OK
    # the hook off: the scratch words were left clean, the next build is exact
    prims = inputs.uniform_points(70001, seed=95)
    t = lbvh.Tree().build(prims, lbvh.POINTS, 63)
    assert_tree_equal(t.export(), oracle.build(prims, oracle.POINTS, 63))
    t.close()


def test_the_waits_take_place(lib):
    # the hook is not a no-op: with waits of up to 200 us before each exchange
    # the construct takes at least that long on the device
    lbvh = L()
    prims = torch.from_numpy(inputs.uniform_points(70001, seed=96)).cuda()
    t = lbvh.Tree()
    t.set_profiling(True)
    t.build(prims, lbvh.POINTS, 63)
    plain = t.stage_times()["construct"]
    assert lib.lbvh_test_construct_jitter(5, 200000) == lbvh.OK
    try:
        t.build(prims, lbvh.POINTS, 63)
        torch.cuda.synchronize()
        waited = t.stage_times()["construct"]
    finally:
        assert lib.lbvh_test_construct_jitter(0, 0) == lbvh.OK
    t.close()
    assert waited > plain + 0.2, (plain, waited)  # ms
