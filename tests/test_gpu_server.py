"""The request server: results of requests served together (batched, several
batches in flight, trees resident) equal each request run alone, and the HBM
budget is enforced by eviction and refusal."""
from __future__ import annotations

import numpy as np
import pytest

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


def alone(prims, kind, bits, queries, qkind, radius):
    lbvh = L()
    t = lbvh.Tree().build(prims, kind, bits)
    off, hits = t.query(queries, qkind, radius=radius)
    return off.cpu().numpy(), hits.cpu().numpy()


def test_mixed_requests_equal_their_results_alone():
    lbvh = L()
    rng = np.random.default_rng(11)
    srv = lbvh.Server(budget_bytes=8 << 30, slots=3, max_batch=16)
    reqs = []
    for k in range(48):
        n = int(np.exp(rng.uniform(np.log(50), np.log(60000))))
        if k % 3 == 2:  # boxes with separate box queries
            prims = torch.from_numpy(inputs.gaussian_mixture_boxes(n, seed=100 + k, components=8)).cuda()
            queries = torch.from_numpy(inputs.gaussian_mixture_boxes(n // 2 + 1, seed=200 + k, components=8,
                                                                      component_seed=100 + k)).cuda()
            spec = (prims, lbvh.BOXES, 30, queries, lbvh.BOX, 0.0)
        else:  # points, queried with themselves; two Morton widths
            src = inputs.uniform_points if k % 2 else inputs.gaussian_mixture_points
            prims = torch.from_numpy(src(n, seed=100 + k)).cuda()
            spec = (prims, lbvh.POINTS, 63 if k % 4 == 0 else 30, prims, lbvh.SPHERE,
                    float(inputs.radius_for_neighbours(n)))
        reqs.append((k, spec, alone(*spec)))  # the request run alone (also sizes its hit buffer)
    # submit everything in one burst so that requests queue up and share batches
    reqs = [(srv.submit(spec[0], spec[1], spec[2], None if spec[3] is spec[0] else spec[3], spec[4],
                        radius=spec[5], key=k + 1, capacity=len(want[1]) + 16), spec, want)
            for k, spec, want in reqs]
    batch_sizes = []
    for ticket, spec, (ooff, ohits) in reqs:
        off, hits, info = srv.wait(ticket)
        assert info["status"] == lbvh.OK, info
        batch_sizes.append(info["batch_size"])
        assert np.array_equal(off.cpu().numpy(), ooff)
        assert np.array_equal(hits.cpu().numpy(), ohits)
    assert max(batch_sizes) > 1  # requests really were served together
    # query-only requests on the resident trees
    st = srv.stats()
    assert st["resident_trees"] == 48 and st["evictions"] == 0
    for k in (0, 5, 47):
        ticket, spec, _ = reqs[k]
        q = spec[3][: max(spec[3].shape[0] // 3, 1)]
        ooff, ohits = alone(spec[0], spec[1], spec[2], q, spec[4], spec[5])
        t2 = srv.submit(None, spec[1], spec[2], q, spec[4], radius=spec[5], key=k + 1, capacity=len(ohits) + 16)
        off, hits, info = srv.wait(t2)
        assert info["status"] == lbvh.OK
        assert np.array_equal(off.cpu().numpy(), ooff) and np.array_equal(hits.cpu().numpy(), ohits)
    srv.close()


def test_wide_codes_share_batches():
    # a burst of 63-bit requests: they queue up and run in shared batches
    lbvh = L()
    srv = lbvh.Server(budget_bytes=8 << 30, slots=1, max_batch=32)
    reqs = []
    for k in range(24):
        n = 3000 + 997 * k
        prims = torch.from_numpy(inputs.gaussian_mixture_points(n, seed=300 + k, components=4)).cuda()
        r = float(inputs.radius_for_neighbours(n))
        want = alone(prims, lbvh.POINTS, 63, prims, lbvh.SPHERE, r)
        reqs.append((prims, r, want))
    tickets = [srv.submit(p, lbvh.POINTS, 63, radius=r, capacity=len(w[1]) + 16) for p, r, w in reqs]
    sizes = []
    for t, (p, r, (ooff, ohits)) in zip(tickets, reqs):
        off, hits, info = srv.wait(t)
        assert info["status"] == lbvh.OK, info
        sizes.append(info["batch_size"])
        assert np.array_equal(off.cpu().numpy(), ooff) and np.array_equal(hits.cpu().numpy(), ohits)
    assert max(sizes) > 2
    lat = srv.latency()
    assert lat["count"] == 24 and 0.0 < lat["p50_s"] <= lat["p99_s"]
    srv.close()


def test_queries_on_one_resident_tree_from_several_slots():
    # query-only requests on the same key queue behind each other (a tree is
    # used by one call at a time) while other slots stay free
    lbvh = L()
    pts = torch.from_numpy(inputs.uniform_points(50000, seed=21)).cuda()
    r = float(inputs.radius_for_neighbours(50000))
    srv = lbvh.Server(budget_bytes=1 << 30, slots=4, max_batch=8)
    _, _, info = srv.wait(srv.submit(pts, lbvh.POINTS, 30, radius=r, key=9, capacity=1 << 22))
    assert info["status"] == lbvh.OK
    qs = [pts[k * 5000:(k + 1) * 5000] for k in range(8)]
    tickets = [srv.submit(None, lbvh.POINTS, 30, q, radius=r, key=9, capacity=1 << 20) for q in qs]
    for q, t in zip(qs, tickets):
        off, hits, info = srv.wait(t)
        assert info["status"] == lbvh.OK
        ooff, ohits = alone(pts, lbvh.POINTS, 30, q, lbvh.SPHERE, r)
        assert np.array_equal(off.cpu().numpy(), ooff) and np.array_equal(hits.cpu().numpy(), ohits)
    srv.close()


def test_budget_evicts_least_recently_used_and_refuses_what_never_fits():
    lbvh = L()
    pts = [torch.from_numpy(inputs.uniform_points(20000, seed=k)).cuda() for k in range(10)]
    r = float(inputs.radius_for_neighbours(20000))
    # each request needs ~7-10 MB while it runs and leaves a ~1 MB tree (nodes
    # only): with 14 MB, ten requests cannot all stay resident
    srv = lbvh.Server(budget_bytes=14 << 20, slots=1, max_batch=1)
    for k, p in enumerate(pts):
        off, hits, info = srv.wait(srv.submit(p, lbvh.POINTS, 30, radius=r, key=k + 1))
        assert info["status"] == lbvh.OK
    st = srv.stats()
    assert st["evictions"] > 0 and st["resident_bytes"] <= 14 << 20
    # the oldest tree was evicted: a query on it is refused; the newest answers
    _, _, info = srv.wait(srv.submit(None, lbvh.POINTS, 30, pts[0][:100], radius=r, key=1))
    assert info["status"] == lbvh.ERR_INVALID
    off, hits, info = srv.wait(srv.submit(None, lbvh.POINTS, 30, pts[9][:100], radius=r, key=10))
    assert info["status"] == lbvh.OK
    ooff, ohits = alone(pts[9], lbvh.POINTS, 30, pts[9][:100], lbvh.SPHERE, r)
    assert np.array_equal(off.cpu().numpy(), ooff) and np.array_equal(hits.cpu().numpy(), ohits)
    # a request larger than the whole budget is refused
    big = torch.from_numpy(inputs.uniform_points(400000, seed=9)).cuda()
    _, _, info = srv.wait(srv.submit(big, lbvh.POINTS, 30, radius=r))
    assert info["status"] == lbvh.ERR_OOM
    srv.close()


def test_capacity_too_small_reports_the_need():
    lbvh = L()
    p = torch.from_numpy(inputs.uniform_points(3000, seed=3)).cuda()
    srv = lbvh.Server(budget_bytes=1 << 30, slots=2, max_batch=8)
    _, _, info = srv.wait(srv.submit(p, lbvh.POINTS, 30, radius=0.1, capacity=10))
    assert info["status"] == lbvh.ERR_CAPACITY and info["total"] > 10
    srv.close()


def test_device_spans_cover_every_job_and_slots_overlap():
    """lbvh_server_device_spans: one (slot, begin, end) row per job, each
    well formed; with two slots and a burst of requests both slots run jobs,
    and at least two of them are on the device at the same time."""
    lbvh = L()
    srv = lbvh.Server(budget_bytes=16 << 30, slots=2, max_batch=4)
    pts = [torch.from_numpy(inputs.uniform_points(200000 + 1000 * k, seed=300 + k)).cuda() for k in range(24)]
    tickets = [srv.submit(p, lbvh.POINTS, 63, radius=float(inputs.radius_for_neighbours(len(p))),
                          capacity=40 * len(p)) for p in pts]
    for t in tickets:
        _, _, info = srv.wait(t)
        assert info["status"] == lbvh.OK
    spans = srv.device_spans()
    assert len(spans) == srv.stats()["batches"]
    assert set(spans[:, 0].astype(int)) == {0, 1}
    assert (spans[:, 2] >= spans[:, 1]).all() and (spans[:, 1] >= 0).all()
    s0, s1 = spans[spans[:, 0] == 0], spans[spans[:, 0] == 1]
    overlaps = [(a[1] < b[2] and b[1] < a[2]) for a in s0 for b in s1]
    assert any(overlaps)
    srv.close()
