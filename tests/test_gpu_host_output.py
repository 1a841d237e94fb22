"""lbvh_query_into_host: the CSR in page-locked host memory (chunks staged on
the device, copied while the next chunk runs) equals the device-buffer query,
with one chunk and with several; memory that is not page-locked is refused
before anything is launched."""
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


@pytest.mark.parametrize("radius", [None, 0.2])
def test_host_csr_equals_device_csr(radius):
    lbvh = L()
    n = 16384
    pts = inputs.uniform_points(n, seed=0)
    r = float(inputs.radius_for_neighbours(n)) if radius is None else radius  # 0.2: lists past the slot
    t = lbvh.Tree().build(pts, lbvh.POINTS, 63)
    q = torch.from_numpy(pts[::3].copy()).cuda()
    doff, dhits = t.query(q, lbvh.SPHERE, radius=r)
    total = int(doff[-1].item())
    hoff = torch.empty(q.shape[0] + 1, dtype=torch.int64).pin_memory()
    hhits = torch.empty(total + 5, dtype=torch.int32).pin_memory()
    st, tot = t.query_into_host(q, lbvh.SPHERE, hoff, hhits, radius=r)
    torch.cuda.synchronize()
    assert st == lbvh.OK and tot == total
    assert np.array_equal(hoff.numpy(), doff.cpu().numpy())
    assert np.array_equal(hhits[:tot].numpy(), dhits.cpu().numpy())
    o = oracle.build(pts, oracle.POINTS, 63)
    ooff, ohits = oracle.query(o, pts[::3], oracle.SPHERE, radius=np.float32(r))
    assert np.array_equal(hoff.numpy(), ooff) and np.array_equal(hhits[:tot].numpy().view(np.uint32), ohits)


@pytest.mark.parametrize("host_chunks", [0, 1, 2])
def test_several_chunks(host_chunks):
    # 9e6 queries: two chunks (at least 2^23 queries each), two staging areas;
    # with lbvh_tree_set_host_chunks(1) one chunk of all the queries
    lbvh = L()
    pts = torch.from_numpy(inputs.uniform_points(1 << 20, seed=5)).cuda()
    q = torch.rand((9_000_000, 3), generator=torch.Generator().manual_seed(6)).cuda()
    r = float(inputs.radius_for_neighbours(1 << 20)) * 0.6
    t = lbvh.Tree().build(pts, lbvh.POINTS, 63)
    t.set_host_chunks(host_chunks)
    doff, dhits = t.query(q, lbvh.SPHERE, radius=r)
    total = int(doff[-1].item())
    hoff = torch.empty(q.shape[0] + 1, dtype=torch.int64).pin_memory()
    hhits = torch.empty(total, dtype=torch.int32).pin_memory()
    st, tot = t.query_into_host(q, lbvh.SPHERE, hoff, hhits, radius=r)
    torch.cuda.synchronize()
    assert st == lbvh.OK and tot == total
    assert torch.equal(hoff, doff.cpu()) and torch.equal(hhits, dhits.cpu())
    # capacity running out in the second chunk: offsets all written, the total reported
    half = int(doff[q.shape[0] // 2].item())
    hoff2 = torch.full((q.shape[0] + 1,), -1, dtype=torch.int64).pin_memory()
    st, tot = t.query_into_host(q, lbvh.SPHERE, hoff2, torch.empty(half + 7, dtype=torch.int32).pin_memory(),
                                radius=r)
    torch.cuda.synchronize()
    assert st == lbvh.ERR_CAPACITY and tot == total and torch.equal(hoff2, doff.cpu())


def test_capacity_too_small_reports_the_need():
    lbvh = L()
    pts = inputs.uniform_points(4000, seed=3)
    t = lbvh.Tree().build(pts, lbvh.POINTS, 30)
    hoff = torch.empty(4001, dtype=torch.int64).pin_memory()
    hhits = torch.empty(10, dtype=torch.int32).pin_memory()
    st, tot = t.query_into_host(pts, lbvh.SPHERE, hoff, hhits, radius=0.05)
    torch.cuda.synchronize()
    assert st == lbvh.ERR_CAPACITY and tot > 10


def test_memory_that_is_not_page_locked_is_refused():
    lbvh = L()
    pts = inputs.uniform_points(3000, seed=4)
    t = lbvh.Tree().build(pts, lbvh.POINTS, 30)
    good_off = torch.empty(3001, dtype=torch.int64).pin_memory()
    good_hits = torch.empty(1 << 16, dtype=torch.int32).pin_memory()
    pageable_off = torch.empty(3001, dtype=torch.int64)
    pageable_hits = torch.empty(1 << 16, dtype=torch.int32)
    device_off = torch.empty(3001, dtype=torch.int64, device="cuda")
    for off, hits in ((pageable_off, good_hits), (good_off, pageable_hits), (device_off, good_hits)):
        st, _ = t.query_into_host(pts, lbvh.SPHERE, off, hits, radius=0.01)
        assert st == lbvh.ERR_INVALID
    st, tot = t.query_into_host(pts, lbvh.SPHERE, good_off, good_hits, radius=0.01)
    torch.cuda.synchronize()
    assert st == lbvh.OK and good_off[-1].item() == tot


def test_no_queries_and_ray_chunks():
    lbvh = L()
    boxes = inputs.gaussian_mixture_boxes(1 << 16, seed=7, components=8)
    t = lbvh.Tree().build(boxes, lbvh.BOXES, 63)
    hoff = torch.full((1,), -1, dtype=torch.int64).pin_memory()
    st, tot = t.query_into_host(torch.empty((0, 8), device="cuda"), lbvh.RAY, hoff, None)
    torch.cuda.synchronize()
    assert st == lbvh.OK and tot == 0 and hoff[0].item() == 0
    # 9e6 ray segments (two chunks; each chunk's rays start 32-byte aligned)
    rays = torch.from_numpy(inputs.random_rays(9_000_000, seed=8, tmax=0.05)).cuda()
    doff, dhits = t.query(rays, lbvh.RAY)
    total = int(doff[-1].item())
    hoff = torch.empty(rays.shape[0] + 1, dtype=torch.int64).pin_memory()
    hhits = torch.empty(max(total, 1), dtype=torch.int32).pin_memory()
    st, tot = t.query_into_host(rays, lbvh.RAY, hoff, hhits)
    torch.cuda.synchronize()
    assert st == lbvh.OK and tot == total
    assert torch.equal(hoff, doff.cpu()) and torch.equal(hhits[:tot], dhits.cpu())


def test_two_trees_in_flight_on_two_streams():
    # the end-to-end pattern: step k builds and queries on tree k % 2 and
    # stream k % 2, its inputs uploaded on a side stream while step k - 1
    # queries, so one step's last result copy overlaps the next step's build;
    # every step's host CSR equals the same query run alone
    lbvh = L()
    n, nq, steps = 1 << 19, (1 << 23) + (1 << 20), 4  # two chunks per query
    r = float(inputs.radius_for_neighbours(n))
    host_pts = [torch.from_numpy(inputs.uniform_points(n, seed=40 + k)).pin_memory() for k in range(steps)]
    host_q = [torch.rand((nq, 3), generator=torch.Generator().manual_seed(50 + k)).pin_memory()
              for k in range(steps)]
    want = []
    alone = lbvh.Tree()
    for k in range(steps):
        alone.build(host_pts[k].cuda(), lbvh.POINTS, 63)
        doff, dhits = alone.query(host_q[k].cuda(), lbvh.SPHERE, radius=r)
        want.append((doff.cpu(), dhits.cpu()))
    alone.close()
    cap = max(int(w[0][-1]) for w in want) + 16
    trees = [lbvh.Tree(), lbvh.Tree()]
    trees[0].set_host_chunks(1)  # one tree copies its whole CSR at once, the other in two chunks
    lanes = [torch.cuda.Stream(), torch.cuda.Stream()]
    side = torch.cuda.Stream()
    dpts = [torch.empty((n, 3), device="cuda"), torch.empty((n, 3), device="cuda")]
    dq = [torch.empty((nq, 3), device="cuda"), torch.empty((nq, 3), device="cuda")]
    uploaded = [torch.cuda.Event(), torch.cuda.Event()]
    consumed = [torch.cuda.Event(), torch.cuda.Event()]
    hoff = [torch.empty(nq + 1, dtype=torch.int64).pin_memory() for _ in range(steps)]
    hhits = [torch.empty(cap, dtype=torch.int32).pin_memory() for _ in range(steps)]
    totals = [0] * steps

    def upload(k):
        slot = k & 1
        with torch.cuda.stream(side):
            side.wait_event(consumed[slot])
            dpts[slot].copy_(host_pts[k], non_blocking=True)
            dq[slot].copy_(host_q[k], non_blocking=True)
            uploaded[slot].record(side)

    upload(0)
    for k in range(steps):
        slot = k & 1
        lanes[slot].synchronize()
        lanes[slot].wait_event(uploaded[slot])
        trees[slot].build(dpts[slot], lbvh.POINTS, 63, stream=lanes[slot])
        if k + 1 < steps:
            upload(k + 1)
        st, totals[k] = trees[slot].query_into_host(dq[slot], lbvh.SPHERE, hoff[k], hhits[k], radius=r,
                                                    stream=lanes[slot])
        assert st == lbvh.OK
        consumed[slot].record(lanes[slot])
    for s in lanes:
        s.synchronize()
    for k in range(steps):
        woff, whits = want[k]
        assert totals[k] == int(woff[-1])
        assert torch.equal(hoff[k], woff) and torch.equal(hhits[k][:totals[k]], whits)
    for t in trees:
        t.close()
