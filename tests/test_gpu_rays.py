"""Ray-segment range queries (slab test) on the GPU against the oracle,
bit-exact CSR: boxes and points, 30- and 63-bit trees, special rays, lists
longer than the walk's buffer, and query-only ray requests on a resident tree
of the request server."""
from __future__ import annotations

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


def check(t, o, rays):
    lbvh = L()
    off, hits = t.query(rays, lbvh.RAY)
    ooff, ohits = oracle.query(o, rays, oracle.RAY)
    assert np.array_equal(off.cpu().numpy(), ooff)
    assert np.array_equal(hits.cpu().numpy().view(np.uint32), ohits)
    return ooff, ohits


@pytest.mark.parametrize("n,bits,tmax", [(3000, 30, 0.2), (20000, 63, 0.05), (50000, 30, np.inf)])
def test_rays_against_boxes(n, bits, tmax):
    lbvh = L()
    prims = inputs.gaussian_mixture_boxes(n, seed=n, components=16, log_half_mu=math.log(0.002))
    t = lbvh.Tree().build(prims, lbvh.BOXES, bits)
    o = oracle.build(prims, oracle.BOXES, bits)
    rays = inputs.random_rays(3000, seed=n + 1, tmax=tmax)
    # half of the rays start near a primitive (so that short segments meet some)
    k = np.random.default_rng(n + 2).integers(0, n, size=1500)
    back = min(float(tmax), 0.1) * 0.5
    rays[:1500, :3] = (prims[k, :3] + prims[k, 3:]) * 0.5 - rays[:1500, 4:7] * back
    ooff, ohits = check(t, o, rays)
    assert len(ohits) > 1500
    if n <= 3000:
        boff, bhits = oracle.bruteforce(prims, oracle.BOXES, rays, oracle.RAY)
        assert np.array_equal(boff, ooff) and np.array_equal(bhits, ohits)


def test_rays_long_lists_take_the_second_walk():
    # unbounded rays through a dense cluster: hundreds to thousands of hits
    lbvh = L()
    n = 30000
    prims = inputs.gaussian_mixture_boxes(n, seed=3, components=2, sigma=0.01, log_half_mu=math.log(0.003))
    t = lbvh.Tree().build(prims, lbvh.BOXES, 63)
    o = oracle.build(prims, oracle.BOXES, 63)
    c = (prims[:, :3] + prims[:, 3:]) * 0.5
    rays = inputs.random_rays(500, seed=4)
    rays[:, :3] = c[:500] - rays[:, 4:7] * 0.5  # aimed through a primitive's centre
    ooff, ohits = check(t, o, rays)
    assert np.diff(ooff).max() > 64


def test_rays_against_points_axis_parallel():
    # a ray meets a point only exactly: axis-parallel rays through points
    lbvh = L()
    n = 10000
    pts = inputs.uniform_points(n, seed=5)
    t = lbvh.Tree().build(pts, lbvh.POINTS, 30)
    o = oracle.build(pts, oracle.POINTS, 30)
    rng = np.random.default_rng(6)
    k = rng.integers(0, n, size=1000)
    rays = np.zeros((1000, 8), np.float32)
    rays[:, :3] = pts[k]
    axis = rng.integers(0, 3, size=1000)
    rays[np.arange(1000), axis] -= 0.25
    rays[np.arange(1000), 4 + axis] = 1.0
    rays[:, 7] = 0.5
    ooff, ohits = check(t, o, rays)
    assert (np.diff(ooff) >= 1).all()


def test_special_rays():
    lbvh = L()
    prims = inputs.gaussian_mixture_boxes(4000, seed=7, components=4, log_half_mu=math.log(0.01))
    t = lbvh.Tree().build(prims, lbvh.BOXES, 30)
    o = oracle.build(prims, oracle.BOXES, 30)
    rays = inputs.random_rays(64, seed=8, tmax=0.5)
    rays[0, 0] = np.nan                                  # NaN origin
    rays[1, 4:7] = 0.0                                   # zero direction: a point query
    rays[2, 4:7] = [1e-40, 0.0, 1.0]                     # subnormal component: parallel axis
    rays[3, 3], rays[3, 7] = 0.4, 0.1                    # tmin > tmax
    rays[4, 7] = np.nan
    rays[5, 4] = np.inf
    rays[6, 3], rays[6, 7] = -np.inf, np.inf             # a full line
    rays[7, :3] = (prims[0, :3] + prims[0, 3:]) * 0.5    # starts inside a box, tmax = 0
    rays[7, 7] = 0.0
    ooff, ohits = check(t, o, rays)
    assert ooff[1] - ooff[0] == 0 and ooff[4] - ooff[3] == 0 and ooff[5] - ooff[4] == 0
    assert ooff[8] - ooff[7] >= 1


def test_ray_query_alignment_and_batch_rejection():
    lbvh = L()
    lib = lbvh.load()
    import ctypes
    t = lbvh.Tree().build(inputs.uniform_points(100, seed=9), lbvh.POINTS, 30)
    buf = torch.zeros(8 * 10 + 1, dtype=torch.float32, device="cuda")
    off = torch.zeros(11, dtype=torch.int64, device="cuda")
    total = ctypes.c_uint64()
    st = lib.lbvh_query_into(t._h, ctypes.c_void_p(buf.data_ptr() + 4), 10, lbvh.RAY, None, 0.0,
                             ctypes.c_void_p(off.data_ptr()), None, 0, ctypes.byref(total), None)
    assert st == lbvh.ERR_INVALID  # not 16-byte aligned
    b = lbvh.Batch()
    pts = torch.from_numpy(inputs.uniform_points(100, seed=9)).cuda()
    rays = torch.from_numpy(inputs.random_rays(10, seed=10)).cuda()
    _, _, _, st = b.build_query(pts, np.array([0, 100]), lbvh.POINTS, 30, rays, np.array([0, 10]), lbvh.RAY,
                                capacity=100)
    assert st == lbvh.ERR_INVALID


def test_server_query_only_rays_on_a_resident_tree():
    lbvh = L()
    prims = inputs.gaussian_mixture_boxes(20000, seed=11, components=8, log_half_mu=math.log(0.003))
    dp = torch.from_numpy(prims).cuda()
    srv = lbvh.Server(budget_bytes=1 << 30, slots=1, max_batch=4)
    q = dp[:100]
    _, _, info = srv.wait(srv.submit(dp, lbvh.BOXES, 30, q, lbvh.BOX, key=5, capacity=1 << 16))
    assert info["status"] == lbvh.OK
    rays = inputs.random_rays(2000, seed=12, tmax=0.2)
    off, hits, info = srv.wait(srv.submit(None, lbvh.BOXES, 30, rays, lbvh.RAY, key=5, capacity=1 << 20))
    assert info["status"] == lbvh.OK
    o = oracle.build(prims, oracle.BOXES, 30)
    ooff, ohits = oracle.query(o, rays, oracle.RAY)
    assert np.array_equal(off.cpu().numpy(), ooff) and np.array_equal(hits.cpu().numpy(), ohits)
    # build requests with rays are refused (the batched path takes spheres and boxes)
    with pytest.raises(Exception):
        srv.submit(dp, lbvh.BOXES, 30, rays, lbvh.RAY, capacity=1 << 20)
    srv.close()
