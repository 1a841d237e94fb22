"""GPU parity: every stage of the CUDA path against the CPU oracle, bit-exact.

Builds (Morton codes, sort, Algorithm 4 with boxes and skips) and queries
(Algorithm 1, CSR) are compared element by element with the oracle on the same
seeded inputs: small and ragged sizes that span several sort tiles, the
degenerate cases, and the full 2^25-primitive configurations in the launch
configuration the benchmark uses (full tree, sampled queries).
"""
from __future__ import annotations

import json
import os

import numpy as np
import pytest

import oracle
from paper_2402_00665_gb300 import _build, inputs
from tests import tree_checks as tc

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


def gpu_build(prims, kind, bits):
    lbvh = L()
    t = lbvh.Tree().build(prims, kind, bits)
    t.check()
    return t


def assert_tree_equal(g, o):
    for k in ("perm", "sorted", "left", "skip_internal", "skip_leaf"):
        assert np.array_equal(g[k], o[k]), k
    for k in ("internal_box", "leaf_box", "bounds"):
        assert np.array_equal(np.asarray(g[k]).view(np.uint32), np.asarray(o[k]).view(np.uint32)), k


def assert_csr_equal(goff, ghits, ooff, ohits):
    goff = goff.cpu().numpy()
    ghits = ghits.cpu().numpy().view(np.uint32)
    assert np.array_equal(goff, ooff)
    assert np.array_equal(ghits, ohits)


# ---------------------------------------------------------------- worked example


def test_golden_fig_example_bottom_up():
    """Algorithm 4 on the 8 keys of Fig. 2a gives the tree and skips of Fig. 1."""
    lbvh = L()
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "fig_karras_8_keys.json")))
    keys = np.array([int(b, 2) for b in g["keys_bits"]], np.uint64)
    n = len(keys)
    pts = inputs.uniform_points(n, seed=3)
    t = lbvh.Tree().build_from_sorted(keys, np.arange(n, dtype=np.uint32), pts, lbvh.POINTS)
    e = t.export()
    for name, node in g["karras_internal"].items():
        k = tc.parse_node(name, n)
        assert e["left"][k] == tc.parse_node(node["left"], n), name
    for name, target in g["skips"].items():
        k = tc.parse_node(name, n)
        got = e["skip_leaf"][k - (n - 1)] if name[0] == "L" else e["skip_internal"][k]
        assert got == tc.parse_node(target, n), name
    o = oracle.tree_from_sorted(keys)
    tc.check_boxes(n, o["range_l"], o["range_r"], e["leaf_box"], e["internal_box"])


@pytest.mark.parametrize("seed", range(4))
def test_bottom_up_on_sorted_keys_with_duplicates(seed):
    lbvh = L()
    rng = np.random.default_rng(seed)
    n = int(rng.integers(2, 20000))
    codes = np.sort(rng.integers(0, 1 << int(rng.integers(1, 63)), size=n).astype(np.uint64))
    pts = inputs.uniform_points(n, seed=seed)
    t = lbvh.Tree().build_from_sorted(codes, np.arange(n, dtype=np.uint32), pts, lbvh.POINTS)
    e = t.export()
    o = oracle.tree_from_sorted(codes)
    assert np.array_equal(e["left"], o["left"])
    assert np.array_equal(e["skip_internal"], o["skip_internal"])
    assert np.array_equal(e["skip_leaf"], o["skip_leaf"])
    tc.check_boxes(n, o["range_l"], o["range_r"], e["leaf_box"], e["internal_box"])


# ---------------------------------------------------------------- stages


@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("bits", [3, 30, 63])
@pytest.mark.parametrize("n", [1, 5, 1000, 4099, 100003])
def test_morton_codes(kind, bits, n):
    lbvh = L()
    prims = inputs.uniform_points(n, seed=n) if kind == 0 else inputs.gaussian_mixture_boxes(n, seed=n)
    codes, bounds = lbvh.morton_codes(prims, kind, bits)
    oc, ob = oracle.morton_codes(prims, kind, bits)
    assert np.array_equal(lbvh.to_u64(codes), oc)
    assert np.array_equal(bounds.cpu().numpy().view(np.uint32), ob.view(np.uint32))


def test_morton_codes_unaligned_and_degenerate():
    lbvh = L()
    base = torch.as_tensor(inputs.uniform_points(10001, seed=1)).cuda()
    flat = base.reshape(-1)[3:]  # starts 12 bytes in: the scalar path
    p = flat.reshape(-1, 3)
    codes, _ = lbvh.morton_codes(p, 0, 63)
    oc, _ = oracle.morton_codes(p.cpu().numpy(), 0, 63)
    assert np.array_equal(lbvh.to_u64(codes), oc)
    for prims in (inputs.collinear_points(777), np.full((300, 3), -0.0, np.float32),
                  np.concatenate([np.zeros((5, 3), np.float32), -np.zeros((5, 3), np.float32)])):
        codes, bounds = lbvh.morton_codes(prims, 0, 30)
        oc, ob = oracle.morton_codes(prims, 0, 30)
        assert np.array_equal(lbvh.to_u64(codes), oc)
        assert np.array_equal(bounds.cpu().numpy().view(np.uint32), ob.view(np.uint32))


def test_morton_codes_nonfinite():
    lbvh = L()
    p = inputs.uniform_points(5000, seed=2)
    p[4321, 2] = np.nan
    with pytest.raises(lbvh.LbvhError) as e:
        lbvh.morton_codes(p, 0, 30)
    assert e.value.status == lbvh.ERR_NONFINITE


@pytest.mark.parametrize("n", [1, 2, 4095, 4096, 4097, 65536 + 17, 1 << 20])
@pytest.mark.parametrize("key_bits,distinct", [(64, 1 << 64), (63, 1 << 63), (30, 1 << 30), (17, 50),
                                               (8, 256), (1, 2)])
def test_sort_pairs_stable(n, key_bits, distinct):
    lbvh = L()
    rng = np.random.default_rng(n + key_bits)
    keys = rng.integers(0, min(distinct, 1 << 63), size=n, dtype=np.uint64)
    if key_bits == 64:
        keys |= rng.integers(0, 2, size=n, dtype=np.uint64) << np.uint64(63)
    keys &= np.uint64((1 << key_bits) - 1) if key_bits < 64 else np.uint64(0xFFFFFFFFFFFFFFFF)
    ko, vo = lbvh.sort_pairs(keys, None, key_bits)
    want = np.argsort(keys, kind="stable")
    assert np.array_equal(lbvh.to_u32(vo), want.astype(np.uint32))
    assert np.array_equal(lbvh.to_u64(ko), keys[want])
    # explicit payloads
    vals = rng.integers(0, 1 << 32, size=n, dtype=np.uint64).astype(np.uint32)
    ko, vo = lbvh.sort_pairs(keys, vals, key_bits)
    assert np.array_equal(lbvh.to_u32(vo), vals[want])


# ---------------------------------------------------------------- builds


def signed_zero_points(n, seed):
    """Coordinates drawn from {-0.0, +0.0, 0.25, 1.0}: box unions must order
    -0.0 below +0.0 whichever child comes first."""
    rng = np.random.default_rng(seed)
    v = np.array([-0.0, 0.0, 0.25, 1.0], np.float32)
    return v[rng.integers(0, 4, size=(n, 3))]


def signed_zero_boxes(n, seed):
    rng = np.random.default_rng(seed)
    lo = np.array([-0.0, 0.0, 0.25], np.float32)[rng.integers(0, 3, size=(n, 3))]
    zero_hi = np.array([-0.0, 0.0], np.float32)[rng.integers(0, 2, size=(n, 3))]
    hi = np.where(lo == 0.0, zero_hi, lo + np.float32(0.5)).astype(np.float32)
    return np.concatenate([lo, hi], axis=1)


BUILD_CASES = {
    "signed_zero_points": lambda: (signed_zero_points(20000, seed=11), 0, 63),
    "signed_zero_boxes": lambda: (signed_zero_boxes(20000, seed=12), 1, 30),
    "d1_uniform_16384_30bit": lambda: (inputs.uniform_points(16384, seed=0), 0, 30),
    "uniform_ragged_63bit": lambda: (inputs.uniform_points(70001, seed=5), 0, 63),
    "boxes_mixture_30bit": lambda: (inputs.gaussian_mixture_boxes(60000, seed=6), 1, 30),
    "boxes_mixture_63bit": lambda: (inputs.gaussian_mixture_boxes(60000, seed=6), 1, 63),
    "duplicates": lambda: (inputs.duplicated_points(30000, 100, seed=7), 0, 63),
    "collinear": lambda: (inputs.collinear_points(20000, seed=8), 0, 30),
    "all_equal": lambda: (np.full((5000, 3), 0.75, np.float32), 0, 63),
    "filled_cube": lambda: (inputs.filled_cube(50000, seed=9), 0, 63),
    "hollow_cube": lambda: (inputs.hollow_cube(50000, seed=9), 0, 30),
    "n1": lambda: (inputs.uniform_points(1, seed=1), 0, 63),
    "n2": lambda: (inputs.uniform_points(2, seed=1), 0, 63),
    "n3_boxes": lambda: (inputs.gaussian_mixture_boxes(3, seed=1), 1, 30),
    "bits3": lambda: (inputs.uniform_points(3000, seed=2), 0, 3),
}


@pytest.mark.parametrize("case", sorted(BUILD_CASES))
def test_build_matches_oracle(case):
    prims, kind, bits = BUILD_CASES[case]()
    t = gpu_build(prims, kind, bits)
    e = t.export()
    o = oracle.build(prims, kind, bits)
    assert_tree_equal(e, o)
    if len(prims) <= 5000:
        tc.check_skips(e["sorted"], e["left"], o["right"], e["skip_internal"], e["skip_leaf"])


def test_rebuild_in_place_reuses_storage():
    lbvh = L()
    t = lbvh.Tree()
    for n, seed, bits in ((50000, 1, 63), (1000, 2, 30), (70000, 3, 63), (70000, 4, 63), (3, 5, 30)):
        p = inputs.uniform_points(n, seed=seed)
        t.build(p, lbvh.POINTS, bits)
        t.check()
        assert_tree_equal(t.export(), oracle.build(p, oracle.POINTS, bits))


def test_empty_tree_and_empty_queries():
    lbvh = L()
    t = lbvh.Tree().build(np.zeros((0, 3), np.float32), lbvh.POINTS, 30)
    t.check()
    assert t.size() == 0
    off, hits = t.query(inputs.uniform_points(10), lbvh.SPHERE, radius=1.0)
    assert off.cpu().numpy().tolist() == [0] * 11 and hits.numel() == 0
    t = gpu_build(inputs.uniform_points(100), lbvh.POINTS, 30)
    off, hits = t.query(np.zeros((0, 3), np.float32), lbvh.SPHERE, radius=1.0)
    assert off.cpu().numpy().tolist() == [0] and hits.numel() == 0


def test_build_nonfinite_is_reported():
    lbvh = L()
    p = inputs.uniform_points(9000, seed=3)
    p[17] = [np.inf, 0, 0]
    t = lbvh.Tree().build(p, lbvh.POINTS, 30)
    assert t.status() == lbvh.ERR_NONFINITE
    with pytest.raises(lbvh.LbvhError) as e:
        t.query(p[:10], lbvh.SPHERE, radius=0.1)
    assert e.value.status == lbvh.ERR_NONFINITE
    # a later good build on the same handle clears the error
    t.build(inputs.uniform_points(9000, seed=4), lbvh.POINTS, 30)
    assert t.status() == lbvh.OK


# ---------------------------------------------------------------- queries


def test_query_d1_exact():
    """16,384 uniform points, 30-bit, radius for ~16 neighbours, every point queried."""
    lbvh = L()
    pts = inputs.uniform_points(16384, seed=0)
    r = inputs.radius_for_neighbours(16384)
    t = gpu_build(pts, lbvh.POINTS, 30)
    off, hits = t.query(pts, lbvh.SPHERE, radius=float(r))
    o = oracle.build(pts, oracle.POINTS, 30)
    ooff, ohits = oracle.query(o, pts, oracle.SPHERE, radius=r)
    assert_csr_equal(off, hits, ooff, ohits)
    boff, bhits = oracle.bruteforce(pts[:2000], oracle.POINTS, pts[:300], oracle.SPHERE, radius=r)
    t2 = gpu_build(pts[:2000], lbvh.POINTS, 30)
    off2, hits2 = t2.query(pts[:300], lbvh.SPHERE, radius=float(r))
    assert_csr_equal(off2, hits2, boff, bhits)


@pytest.mark.parametrize("bits", [30, 63])
def test_box_queries_on_boxes(bits):
    lbvh = L()
    boxes = inputs.gaussian_mixture_boxes(50000, seed=11)
    q = inputs.gaussian_mixture_boxes(20000, seed=12, component_seed=11)
    t = gpu_build(boxes, lbvh.BOXES, bits)
    off, hits = t.query(q, lbvh.BOX)
    o = oracle.build(boxes, oracle.BOXES, bits)
    ooff, ohits = oracle.query(o, q, oracle.BOX)
    assert_csr_equal(off, hits, ooff, ohits)
    assert ooff[-1] > 0


def test_sphere_queries_on_boxes_per_query_radii():
    lbvh = L()
    boxes = inputs.gaussian_mixture_boxes(30000, seed=13, components=8)
    rng = np.random.default_rng(14)
    q = rng.random((5000, 3)).astype(np.float32)
    radii = (rng.random(5000) * 0.03).astype(np.float32)
    t = gpu_build(boxes, lbvh.BOXES, 63)
    off, hits = t.query(q, lbvh.SPHERE, radii=radii)
    o = oracle.build(boxes, oracle.BOXES, 63)
    assert_csr_equal(off, hits, *oracle.query(o, q, oracle.SPHERE, radii=radii))


def test_box_queries_on_points():
    lbvh = L()
    pts = inputs.uniform_points(40000, seed=15)
    rng = np.random.default_rng(16)
    lo = rng.random((3000, 3)).astype(np.float32)
    q = np.concatenate([lo, lo + np.float32(0.03)], axis=1).astype(np.float32)
    t = gpu_build(pts, lbvh.POINTS, 63)
    off, hits = t.query(q, lbvh.BOX)
    o = oracle.build(pts, oracle.POINTS, 63)
    assert_csr_equal(off, hits, *oracle.query(o, q, oracle.BOX))


@pytest.mark.parametrize("radius", [0.0, 0.05, 0.1, 0.2, 0.5, 2.0])
def test_long_hit_lists_use_the_fixup_sort(radius):
    """Lists of up to 32 hits are sorted in one thread's registers, 33..64 by
    a warp in registers; longer ones (past the walk's 64-hit buffer) walk again
    and are sorted by one warp up to 1024 hits, by one CTA in shared memory up
    to 8192, by one CTA in global memory above."""
    lbvh = L()
    pts = inputs.uniform_points(12000, seed=17)
    q = pts[::40]
    t = gpu_build(pts, lbvh.POINTS, 30)
    off, hits = t.query(q, lbvh.SPHERE, radius=radius)
    o = oracle.build(pts, oracle.POINTS, 30)
    assert_csr_equal(off, hits, *oracle.query(o, q, oracle.SPHERE, radius=np.float32(radius)))


def test_hit_lists_of_every_length_and_warp_maximum():
    """Lists of 0..~36 hits with the longest list of each group of 32
    consecutive queries in every range of the copy's pruned sorting networks
    (<= 8, 16, 24, 32, and past the register sort), primitive ids in random
    order along the line."""
    lbvh = L()
    rng = np.random.default_rng(21)
    n = 2000
    pts = np.zeros((n, 3), np.float32)
    pts[:, 0] = rng.permutation(n).astype(np.float32)
    scales = [0.3, 2.6, 3.9, 4.4, 7.9, 8.4, 11.9, 12.4, 15.9, 17.6]
    nq = 32 * len(scales) * 4
    q = np.zeros((nq, 3), np.float32)
    q[:, 0] = rng.integers(20, n - 20, nq).astype(np.float32)
    q[:, 1] = np.float32(0.1)
    radii = np.concatenate([rng.random(32).astype(np.float32) * np.float32(scales[g % len(scales)])
                            for g in range(nq // 32)]).astype(np.float32)
    t = gpu_build(pts, lbvh.POINTS, 30)
    off, hits = t.query(q, lbvh.SPHERE, radii=radii)
    o = oracle.build(pts, oracle.POINTS, 30)
    ooff, ohits = oracle.query(o, q, oracle.SPHERE, radii=radii)
    assert_csr_equal(off, hits, ooff, ohits)
    lens = np.diff(ooff).reshape(-1, 32).max(axis=1)
    for lo, hi in ((0, 1), (2, 8), (9, 16), (17, 24), (25, 32), (33, 64)):
        assert ((lens >= lo) & (lens <= hi)).any(), (lo, hi, lens)


def test_all_equal_points_every_query_hits_everything():
    lbvh = L()
    pts = np.full((9000, 3), 0.5, np.float32)
    t = gpu_build(pts, lbvh.POINTS, 63)
    off, hits = t.query(pts[:20], lbvh.SPHERE, radius=0.0)
    off = off.cpu().numpy()
    hits = hits.cpu().numpy().view(np.uint32)
    assert np.array_equal(off, np.arange(21) * 9000)
    assert np.array_equal(hits.reshape(20, 9000), np.tile(np.arange(9000, dtype=np.uint32), (20, 1)))


def test_query_capacity_error_reports_need():
    lbvh = L()
    pts = inputs.uniform_points(5000, seed=18)
    t = gpu_build(pts, lbvh.POINTS, 30)
    offsets = torch.empty(5001, dtype=torch.int64, device="cuda")
    hits = torch.empty(10, dtype=torch.int32, device="cuda")
    st, total = t.query_into(pts, lbvh.SPHERE, offsets, hits, radius=0.05)
    assert st == lbvh.ERR_CAPACITY and total > 10
    hits = torch.empty(total, dtype=torch.int32, device="cuda")
    st, total2 = t.query_into(pts, lbvh.SPHERE, offsets, hits, radius=0.05)
    assert st == lbvh.OK and total2 == total


def _view(ptr, n, typestr):
    """A torch view of library-allocated device memory (no copy)."""
    class _Arr:
        __cuda_array_interface__ = {"shape": (n,), "typestr": typestr, "data": (ptr, False),
                                    "version": 3}
    return torch.as_tensor(_Arr(), device="cuda")


def test_library_allocated_query_matches_caller_buffers():
    import ctypes
    lbvh = L()
    lib = lbvh.load()
    pts = inputs.uniform_points(3000, seed=19)
    t = gpu_build(pts, lbvh.POINTS, 63)
    q = torch.as_tensor(pts).cuda()
    d_off, d_hits, total = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_uint64()
    st = lib.lbvh_query(t.handle, ctypes.c_void_p(q.data_ptr()), 3000, 0, None, 0.05,
                        ctypes.byref(d_off), ctypes.byref(d_hits), ctypes.byref(total),
                        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == lbvh.OK
    torch.cuda.synchronize()
    off = _view(d_off.value, 3001, "<i8").clone()
    hits = _view(d_hits.value, total.value, "<i4").clone()
    ref_off, ref_hits = t.query(pts, lbvh.SPHERE, radius=0.05)
    assert torch.equal(off, ref_off) and torch.equal(hits, ref_hits)
    lib.lbvh_free(d_off)
    lib.lbvh_free(d_hits)


def test_self_query_reuses_build_order_same_result():
    """Queries that are the build's own primitives (same buffer) are walked in
    the build's Morton order; results equal those from a separate buffer."""
    lbvh = L()
    pts = torch.as_tensor(inputs.uniform_points(50000, seed=20)).cuda()
    r = float(inputs.radius_for_neighbours(50000))
    t = lbvh.Tree().build(pts, lbvh.POINTS, 63)
    off_a, hits_a = t.query(pts, lbvh.SPHERE, radius=r)           # aliased: build order
    off_b, hits_b = t.query(pts.clone(), lbvh.SPHERE, radius=r)   # encoded + sorted order
    assert torch.equal(off_a, off_b) and torch.equal(hits_a, hits_b)
    o = oracle.build(pts.cpu().numpy(), oracle.POINTS, 63)
    assert_csr_equal(off_a, hits_a, *oracle.query(o, pts.cpu().numpy(), oracle.SPHERE, radius=np.float32(r)))
    boxes = torch.as_tensor(inputs.gaussian_mixture_boxes(40000, seed=21)).cuda()
    t = lbvh.Tree().build(boxes, lbvh.BOXES, 30)
    off_a, hits_a = t.query(boxes, lbvh.BOX)
    off_b, hits_b = t.query(boxes.clone(), lbvh.BOX)
    assert torch.equal(off_a, off_b) and torch.equal(hits_a, hits_b)


def test_nan_and_infinite_query_centres():
    lbvh = L()
    pts = inputs.uniform_points(5000, seed=32)
    q = inputs.uniform_points(4000, seed=33)
    q[::7, 0] = np.nan
    q[3::11, 2] = np.inf
    q[5::13, 1] = -np.inf
    t = gpu_build(pts, lbvh.POINTS, 63)
    off, hits = t.query(q, lbvh.SPHERE, radius=0.2)
    o = oracle.build(pts, oracle.POINTS, 63)
    assert_csr_equal(off, hits, *oracle.query(o, q, oracle.SPHERE, radius=np.float32(0.2)))
