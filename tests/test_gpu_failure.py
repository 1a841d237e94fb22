"""Failure detection on the GPU without a fault: a sort tile that never
publishes makes the later tiles' bounded look-back waits run out (about one
second each); the build reports LBVH_ERR_TIMEOUT, queries on it report the
same, and the next build is correct again. Nothing faults, traps or hangs."""
from __future__ import annotations

import time

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


def test_look_back_wait_runs_out_and_the_next_build_recovers():
    from paper_2402_00665_gb300 import lbvh
    lib = lbvh.load()
    n = 200000  # about 65 sort tiles
    pts = inputs.uniform_points(n, seed=61)
    dp = torch.from_numpy(pts).cuda()
    t = lbvh.Tree()
    assert lib.lbvh_test_hold_sort_tile(3) == lbvh.OK
    try:
        t0 = time.perf_counter()
        t.build(dp, lbvh.POINTS, 30)
        st = t.status()
        waited = time.perf_counter() - t0
    finally:
        assert lib.lbvh_test_hold_sort_tile(-1) == lbvh.OK
    assert st == lbvh.ERR_TIMEOUT
    assert waited < 30.0
    # a query on the failed tree reports the failure instead of walking it
    off = torch.empty(11, dtype=torch.int64, device="cuda")
    hits = torch.empty(100, dtype=torch.int32, device="cuda")
    st, _ = t.query_into(dp[:10], lbvh.SPHERE, off, hits, radius=0.01)
    assert st == lbvh.ERR_TIMEOUT
    # the next build (hook off) is correct again, bit for bit
    t.build(dp, lbvh.POINTS, 30)
    t.check()
    o = oracle.build(pts, oracle.POINTS, 30)
    e = t.export()
    for k in ("perm", "left", "skip_internal", "skip_leaf"):
        assert np.array_equal(e[k], o[k]), k
    assert np.array_equal(e["internal_box"].view(np.uint32), o["internal_box"].view(np.uint32))


def test_hook_argument_checked():
    from paper_2402_00665_gb300 import lbvh
    assert lbvh.load().lbvh_test_hold_sort_tile(-2) == lbvh.ERR_INVALID


def test_allocation_failure_is_reported_and_the_tree_stays_usable():
    # a count-only query of 2^30 - 1 queries needs about 275 GB of walk slots
    # (256 bytes each), more than the device has: the library's allocation
    # fails and the call reports LBVH_ERR_OOM (after ~52 GB of smaller
    # buffers were had); the tree then answers queries exactly and the
    # library's cached memory can be given back
    from paper_2402_00665_gb300 import lbvh
    lib = lbvh.load()
    n = 1 << 16
    pts = inputs.uniform_points(n, seed=71)
    t = lbvh.Tree().build(pts, lbvh.POINTS, 30)
    nq = (1 << 30) - 1
    q = torch.zeros((nq, 3), dtype=torch.float32, device="cuda")
    off = torch.empty(nq + 1, dtype=torch.int64, device="cuda")
    st, _ = t.query_into(q, lbvh.SPHERE, off, None, radius=0.01)
    assert st == lbvh.ERR_OOM
    del q, off
    torch.cuda.synchronize()
    r = float(inputs.radius_for_neighbours(n))
    o = oracle.build(pts, oracle.POINTS, 30)
    ooff, ohits = oracle.query(o, pts[:5000], oracle.SPHERE, radius=r)
    doff, dhits = t.query(pts[:5000], lbvh.SPHERE, radius=r)
    assert np.array_equal(doff.cpu().numpy(), ooff)
    assert np.array_equal(dhits.cpu().numpy().view(np.uint32), ohits)
    t.close()
    assert lib.lbvh_release_cached_memory() == lbvh.OK
