"""Pins of the CPU oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself: each test checks it against a
printed worked example (Figs. 1, 2a, 2b), a closed form, a library routine, an
independent brute force, or an invariant stated in the paper.
"""
from __future__ import annotations

import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2402_00665_gb300 import inputs
from tests import alg4_model, tree_checks as tc

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "fig_karras_8_keys.json")


def golden():
    with open(GOLDEN) as f:
        g = json.load(f)
    keys = np.array([int(b, 2) for b in g["keys_bits"]], np.uint64)
    return g, keys


# ---------------------------------------------------------------- Figs. 1, 2


def test_golden_karras_topology_fig2a():
    g, keys = golden()
    n = len(keys)
    t = oracle.tree_from_sorted(keys)
    for name, node in g["karras_internal"].items():
        k = tc.parse_node(name, n)
        assert [t["range_l"][k], t["range_r"][k]] == node["range"], name
        assert t["split"][k] == node["split"], name
        assert t["left"][k] == tc.parse_node(node["left"], n), name
        assert t["right"][k] == tc.parse_node(node["right"], n), name


def test_golden_skips_fig1():
    g, keys = golden()
    n = len(keys)
    t = oracle.tree_from_sorted(keys)
    for name, target in g["skips"].items():
        k = tc.parse_node(name, n)
        got = t["skip_leaf"][k - (n - 1)] if name[0] == "L" else t["skip_internal"][k]
        assert got == tc.parse_node(target, n), name


def test_golden_apetrei_splits_fig2b():
    """In Apetrei's ordering a node's index is its split (Sec. 3.2, Fig. 2b)."""
    g, keys = golden()
    n = len(keys)
    t = oracle.tree_from_sorted(keys)

    def apetrei_name(c):
        if c >= n - 1:
            return f"L{c - (n - 1)}"
        return f"A{t['split'][c]}"

    for k in range(n - 1):
        children = [apetrei_name(t["left"][k]), apetrei_name(t["right"][k])]
        assert g["apetrei_children"][f"A{t['split'][k]}"] == children
    assert f"A{t['split'][0]}" == g["apetrei_root"]


def test_golden_tree_invariants():
    _, keys = golden()
    t = oracle.tree_from_sorted(keys)
    tc.check_karras_tree(keys, t["left"], t["right"], t["range_l"], t["range_r"], t["split"])
    tc.check_skips(keys, t["left"], t["right"], t["skip_internal"], t["skip_leaf"])


# ---------------------------------------------------------------- Algorithm 4


@pytest.mark.parametrize("seed", range(6))
def test_algorithm4_model_matches_oracle_any_interleaving(seed):
    """Algorithm 4 (as read) builds the oracle's tree under any arrival order."""
    rng = np.random.default_rng(seed)
    for n in (1, 2, 3, 5, 8, 33, 200):
        codes = np.sort(rng.integers(0, 1 << int(rng.integers(2, 12)), size=n).astype(np.uint64))
        t = oracle.tree_from_sorted(codes)
        for sched_seed in range(3):
            m = alg4_model.run(codes, seed=sched_seed + 100 * seed)
            assert m["left"] == t["left"].tolist()
            assert m["skip_internal"] == t["skip_internal"].tolist()
            assert m["skip_leaf"] == t["skip_leaf"].tolist()


def test_algorithm4_golden_and_literal_left_child_line():
    """The printed left-child line of Algorithm 4 does not give Fig. 1's tree;
    the split reading (children of split p are p and p+1, Sec. 4) does."""
    g, keys = golden()
    n = len(keys)
    want = [tc.parse_node(g["karras_internal"][f"I{k}"]["left"], n) for k in range(n - 1)]
    for sched in ("random", "reverse", "forward"):
        m = alg4_model.run(keys, seed=3, schedule=sched)
        assert m["left"] == want
    lit = alg4_model.run(keys, seed=3, left_child_rule="literal")
    assert lit["left"] != want


# ---------------------------------------------------------------- Morton codes


def test_interleave_unit_bits():
    # x is the most significant bit of each triple
    assert oracle.interleave(1, 0, 0, 1) == 0b100
    assert oracle.interleave(0, 1, 0, 1) == 0b010
    assert oracle.interleave(0, 0, 1, 1) == 0b001
    assert oracle.interleave(2, 0, 0, 2) == 0b100000
    assert oracle.interleave(0, 0, 2, 2) == 0b001000
    top = (1 << 21) - 1
    assert oracle.interleave(top, top, top, 21) == (1 << 63) - 1


def test_interleave_is_z_order():
    """Z-order: comparing codes = comparing the tuples
    (x_{b-1}, y_{b-1}, z_{b-1}, x_{b-2}, ...) lexicographically; and the map is
    a bijection onto [0, 8^b)."""
    b = 3
    side = 1 << b
    cells = [(x, y, z) for x in range(side) for y in range(side) for z in range(side)]
    codes = [oracle.interleave(x, y, z, b) for x, y, z in cells]
    assert sorted(codes) == list(range(side ** 3))

    def bits(c):
        x, y, z = c
        return tuple(v for k in reversed(range(b)) for v in ((x >> k) & 1, (y >> k) & 1, (z >> k) & 1))

    by_code = [c for _, c in sorted(zip(codes, cells))]
    assert by_code == sorted(cells, key=bits)


def test_quantize_special_cases():
    for b in (1, 10, 21):
        top = (1 << b) - 1
        assert oracle.quantize(0.0, 0.0, 1.0, b) == 0
        assert oracle.quantize(1.0, 0.0, 1.0, b) == top  # the maximum lands in the last cell
        assert oracle.quantize(0.5, 0.0, 1.0, b) == 1 << (b - 1)
        assert oracle.quantize(3.0, 3.0, 3.0, b) == 0  # zero extent
        assert oracle.quantize(-2.0, -2.0, 6.0, b) == 0
        assert oracle.quantize(6.0, -2.0, 6.0, b) == top


def test_quantize_matches_exact_floor():
    """Cell index vs floor(2^b (c-lo)/(hi-lo)) in exact rational arithmetic:
    the FP32 steps may move a value across a cell boundary by rounding only."""
    from fractions import Fraction
    rng = np.random.default_rng(5)
    lo, hi = np.float32(-1.25), np.float32(3.5)
    for b in (10, 21):
        mismatches = 0
        for c in rng.uniform(lo, hi, 2000).astype(np.float32):
            exact = Fraction(float(c) - float(lo)) / Fraction(float(hi) - float(lo)) * (1 << b)
            want = min(math.floor(exact), (1 << b) - 1)
            got = oracle.quantize(float(c), float(lo), float(hi), b)
            assert abs(got - want) <= 1
            if got != want:
                # three FP32 roundings (two subtractions, one division) move
                # t by at most 3 ulp(1) = 3 * 2^-24, i.e. 3 * 2^(b-24) cells
                assert abs(exact - round(exact)) <= Fraction(3, 1 << 24) * (1 << b)
                mismatches += 1
        assert mismatches <= 2 + 2000 * 3 * 2.0 ** (b - 24)


def test_quantize_equals_reading_g7_rounded_exactly():
    """The cell index exactly as reading G7 computes it, each FP32 operation
    rounded once from exact rationals (extent = hi - lo, t = (c - lo) / extent,
    v = t * 2^b, then 0, the last cell, or trunc(v)), on centres at cell
    boundaries and one or two FP32 steps either side, where the roundings
    decide the cell. The reference is built from the reading alone."""
    from fractions import Fraction
    F = lambda v: Fraction(float(v))
    rng = np.random.default_rng(6)
    moved = 0
    for lo, hi in ((np.float32(-1.25), np.float32(3.5)), (np.float32(0.0), np.float32(1.0)),
                   (np.float32(1e-3), np.float32(7e-3)), (np.float32(-300.0), np.float32(2.5e4))):
        for b in (1, 10, 21):
            top = (1 << b) - 1
            extent = _rn32(F(hi) - F(lo))
            for k in rng.integers(0, 1 << b, 150):
                edge = np.float32(float(F(lo) + F(extent) * Fraction(int(k), 1 << b)))
                for c in (edge, np.nextafter(edge, np.float32(-np.inf)), np.nextafter(edge, np.float32(np.inf)),
                          np.nextafter(np.nextafter(edge, np.float32(np.inf)), np.float32(np.inf))):
                    t = _rn32(F(_rn32(F(c) - F(lo))) / F(extent))
                    v = _rn32(F(t) * (1 << b))
                    want = 0 if not v > 0 else (top if v >= top else int(math.floor(float(v))))
                    assert oracle.quantize(float(c), float(lo), float(hi), b) == want, (c, lo, hi, b)
                    exact = (F(c) - F(lo)) / (F(hi) - F(lo)) * (1 << b)
                    moved += int(want != min(max(math.floor(exact), 0), top))
    assert moved > 0  # some centres are put in the neighbouring cell by the roundings


def test_morton_codes_and_bounds():
    pts = inputs.uniform_points(1000, seed=3)
    codes, bounds = oracle.morton_codes(pts, oracle.POINTS, 30)
    assert np.array_equal(bounds[:3], pts.min(axis=0)) and np.array_equal(bounds[3:], pts.max(axis=0))
    # the points that reach each axis minimum / maximum land in cell 0 / 1023
    for a, shift in ((0, 2), (1, 1), (2, 0)):
        q = np.array([sum(((int(c) >> (3 * k + shift)) & 1) << k for k in range(10)) for c in codes])
        assert q[np.argmin(pts[:, a])] == 0 and q[np.argmax(pts[:, a])] == 1023
        # monotone: a larger coordinate never gets a smaller cell
        o = np.argsort(pts[:, a], kind="stable")
        assert np.all(np.diff(q[o]) >= 0)
    assert codes.max() < (1 << 30)


def test_box_centroids():
    boxes = inputs.gaussian_mixture_boxes(500, seed=4)
    c = np.zeros((500, 3), np.float32)
    lib = oracle._load()
    assert lib.oracle_centroids(boxes.ctypes.data, 500, oracle.BOXES, c.ctypes.data) == 0
    want = (boxes[:, :3] + boxes[:, 3:]) * np.float32(0.5)
    assert np.array_equal(c, want)


def test_nonfinite_rejected():
    pts = inputs.uniform_points(50, seed=1)
    for bad in (np.nan, np.inf, -np.inf):
        p = pts.copy()
        p[17, 1] = bad
        with pytest.raises(oracle.OracleError) as e:
            oracle.build(p, oracle.POINTS, 30)
        assert e.value.status == oracle.NONFINITE


def test_invalid_bits_rejected():
    pts = inputs.uniform_points(10)
    for bits in (0, 2, 31, 64, 66):
        with pytest.raises(oracle.OracleError):
            oracle.build(pts, oracle.POINTS, bits)


# ---------------------------------------------------------------- sort, delta


def test_sort_matches_stable_argsort():
    rng = np.random.default_rng(7)
    for distinct in (3, 100, 1 << 40):
        codes = rng.integers(0, distinct, size=5000).astype(np.uint64)
        perm, s = oracle.sort_codes(codes)
        want = np.argsort(codes, kind="stable")
        assert np.array_equal(perm, want.astype(np.uint32))
        assert np.array_equal(s, codes[want])


def test_delta_against_python_integers():
    rng = np.random.default_rng(8)
    codes = np.sort(rng.integers(0, 64, size=300).astype(np.uint64))
    aug = tc.aug_keys(codes)
    n = len(codes)
    for _ in range(500):
        i, j = sorted(rng.integers(0, n, size=2).tolist())
        if i == j:
            continue
        want = (aug[i] ^ aug[j]).bit_length() - 1
        assert oracle.delta(codes, i, j) == want
        # delta over a range is the largest delta* inside it (sorted keys)
        assert want == max(oracle.delta(codes, g, g + 1) for g in range(i, j))
    INF = 2 ** 31 - 1
    assert oracle.delta(codes, -1, 0) == INF and oracle.delta(codes, n - 1, n) == INF


# ---------------------------------------------------------------- trees


def _random_codes(rng, n, bits):
    return rng.integers(0, 1 << bits, size=n).astype(np.uint64)


@pytest.mark.parametrize("n,bits", [(2, 3), (3, 3), (17, 6), (64, 3), (257, 9), (1000, 30), (3000, 63)])
def test_tree_invariants_random(n, bits):
    rng = np.random.default_rng(n * 1000 + bits)
    codes = np.sort(_random_codes(rng, n, min(bits, 62)))
    t = oracle.tree_from_sorted(codes)
    tc.check_karras_tree(codes, t["left"], t["right"], t["range_l"], t["range_r"], t["split"])
    tc.check_skips(codes, t["left"], t["right"], t["skip_internal"], t["skip_leaf"])


def test_tree_all_codes_equal():
    """Equal codes: the position bits alone shape a balanced tree (Sec. 3.2)."""
    n = 1000
    codes = np.zeros(n, np.uint64)
    t = oracle.tree_from_sorted(codes)
    tc.check_karras_tree(codes, t["left"], t["right"], t["range_l"], t["range_r"], t["split"])
    tc.check_skips(codes, t["left"], t["right"], t["skip_internal"], t["skip_leaf"])
    depth = {0: 0}
    for k in tc.preorder(n, t["left"], t["right"]):
        if k < n - 1:
            for c in (t["left"][k], t["right"][k]):
                depth[int(c)] = depth[k] + 1
    assert max(depth.values()) <= math.ceil(math.log2(n)) + 1


def test_build_points_full():
    pts = inputs.uniform_points(2000, seed=11)
    t = oracle.build(pts, oracle.POINTS, 30)
    want = np.argsort(t["codes"], kind="stable").astype(np.uint32)
    assert np.array_equal(t["perm"], want)
    tc.check_karras_tree(t["sorted"], t["left"], t["right"], t["range_l"], t["range_r"], t["split"])
    tc.check_skips(t["sorted"], t["left"], t["right"], t["skip_internal"], t["skip_leaf"])
    lb = np.concatenate([pts[t["perm"]], pts[t["perm"]]], axis=1)
    assert np.array_equal(t["leaf_box"], lb)
    tc.check_boxes(2000, t["range_l"], t["range_r"], t["leaf_box"], t["internal_box"])


def test_build_boxes_duplicates_30bit():
    boxes = inputs.gaussian_mixture_boxes(3000, seed=12, components=4)
    t = oracle.build(boxes, oracle.BOXES, 30)
    assert len(np.unique(t["codes"])) < 3000  # duplicate codes present
    tc.check_karras_tree(t["sorted"], t["left"], t["right"], t["range_l"], t["range_r"], t["split"])
    tc.check_skips(t["sorted"], t["left"], t["right"], t["skip_internal"], t["skip_leaf"])
    assert np.array_equal(t["leaf_box"], boxes[t["perm"]])
    tc.check_boxes(3000, t["range_l"], t["range_r"], t["leaf_box"], t["internal_box"])


@pytest.mark.parametrize("n", [0, 1, 2, 3])
def test_tiny_builds(n):
    pts = inputs.uniform_points(n, seed=2)
    t = oracle.build(pts, oracle.POINTS, 63)
    assert t["left"].shape == (max(n - 1, 0),)
    if n == 1:
        assert t["skip_leaf"].tolist() == [-1] and t["codes"].tolist() == [0]
    if n >= 2:
        tc.check_karras_tree(t["sorted"], t["left"], t["right"], t["range_l"], t["range_r"], t["split"])
        tc.check_skips(t["sorted"], t["left"], t["right"], t["skip_internal"], t["skip_leaf"])
    off, hits = oracle.query(t, pts, oracle.SPHERE, radius=10.0)
    assert off.tolist() == [k * n for k in range(n + 1)]
    for q in range(n):
        assert hits[off[q]:off[q + 1]].tolist() == list(range(n))


def test_degenerate_axes_and_all_equal_points():
    p = inputs.collinear_points(500, seed=3)
    t = oracle.build(p, oracle.POINTS, 30)
    assert np.all(t["bounds"][[1, 2, 4, 5]] == 0)
    tc.check_skips(t["sorted"], t["left"], t["right"], t["skip_internal"], t["skip_leaf"])
    same = np.full((300, 3), 0.25, np.float32)
    t = oracle.build(same, oracle.POINTS, 63)
    assert np.all(t["codes"] == 0)
    assert np.array_equal(t["perm"], np.arange(300, dtype=np.uint32))
    tc.check_karras_tree(t["sorted"], t["left"], t["right"], t["range_l"], t["range_r"], t["split"])


# ---------------------------------------------------------------- predicates, queries


def test_sphere_predicate_against_fp64():
    """Away from the boundary the FP32 test agrees with the exact distance."""
    rng = np.random.default_rng(13)
    agree = 0
    for _ in range(3000):
        c = rng.random(3).astype(np.float32)
        lo = rng.random(3).astype(np.float32)
        hi = (lo + rng.random(3).astype(np.float32) * np.float32(0.2)).astype(np.float32)
        r = np.float32(rng.random() * 0.5)
        e = np.maximum(np.maximum(lo.astype(np.float64) - c, c - hi.astype(np.float64)), 0.0)
        d = math.sqrt(float((e * e).sum()))
        if abs(d - float(r)) < 1e-5:
            continue
        assert oracle.sphere_box(c, r, np.concatenate([lo, hi])) == (d <= float(r))
        agree += 1
    assert agree > 2900


def _rn32(x):
    """x (a Fraction) rounded to the nearest FP32 value, ties to even: the
    IEEE rounding of one FP32 operation, computed exactly."""
    from fractions import Fraction
    if x == 0:
        return np.float32(0.0)
    sign = -1 if x < 0 else 1
    a = abs(x)
    e = a.numerator.bit_length() - a.denominator.bit_length()  # 2^e <= a < 2^(e+2)
    if Fraction(2) ** e > a:
        e -= 1
    if Fraction(2) ** (e + 1) <= a:
        e += 1
    ulp = Fraction(2) ** (max(e, -126) - 23)  # subnormals below 2^-126
    q = a / ulp
    n = q.numerator // q.denominator
    rem = q - n
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and n % 2 == 1):
        n += 1
    v = n * ulp
    if v >= Fraction(2) ** 128:
        return np.float32(sign * np.inf)
    return np.float32(sign * float(v))  # n * ulp has at most 24 significant bits: exact


def _sphere_d2_exact(c, box):
    """Reading G8 computed with exact rationals: per axis the gap
    max(lo - c, c - hi, 0) from two FP32 subtractions, then d2 = ex*ex
    rounded once, + ey*ey and + ez*ez each as one fused multiply-add (the
    exact product plus the sum, rounded once)."""
    from fractions import Fraction
    F = lambda v: Fraction(float(v))  # an FP32 value is exact as a double
    e = []
    for a in range(3):
        below = _rn32(F(box[a]) - F(c[a]))
        above = _rn32(F(c[a]) - F(box[3 + a]))
        e.append(max(below, above, np.float32(0.0)))
    d2 = _rn32(F(e[0]) * F(e[0]))
    d2 = _rn32(F(e[1]) * F(e[1]) + F(d2))
    return _rn32(F(e[2]) * F(e[2]) + F(d2))


def test_sphere_predicate_at_the_boundary_against_exact_rounding():
    """The ball test and the kNN squared distance, exactly as reading G8 rounds
    them, at radii on both sides of the boundary: for each centre and box, r
    the FP32 square root of the exact d2 and its two neighbours, so that r*r
    falls just below, on or just above d2. The reference rounds exact
    rationals; nothing of it comes from the oracle's C code."""
    from fractions import Fraction
    rng = np.random.default_rng(17)
    cases = on_boundary = 0
    for k in range(1500):
        scale = np.float32(10.0 ** rng.integers(-6, 3))  # gaps from ~1e-6 to ~1e2
        lo = (rng.random(3) * scale).astype(np.float32)
        hi = (lo + rng.random(3).astype(np.float32) * scale).astype(np.float32)
        c = (rng.random(3) * np.float32(3) * scale - scale).astype(np.float32)
        if k % 3 == 0:  # one axis inside the slab, or two: fewer terms
            c[rng.integers(0, 3)] = (lo[0] + hi[0]) * np.float32(0.5) if lo[0] <= hi[0] else c[0]
        box = np.concatenate([lo, hi])
        d2 = _sphere_d2_exact(c, box)
        assert np.float32(oracle.point_box_d2(c, box)) == d2
        r0 = np.float32(math.sqrt(float(d2)))
        for r in (np.nextafter(r0, np.float32(0)), r0, np.nextafter(r0, np.float32(np.inf))):
            r2 = _rn32(Fraction(float(r)) * Fraction(float(r)))
            want = bool(d2 <= r2)
            assert oracle.sphere_box(c, r, box) == want, (c, box, r)
            cases += 1
            on_boundary += int(d2 == r2)
    assert cases == 4500 and on_boundary > 0


def test_predicate_closed_boundaries():
    box = np.array([0, 0, 0, 1, 1, 1], np.float32)
    assert oracle.sphere_box([2.0, 0.5, 0.5], 1.0, box)  # touching: closed ball
    assert not oracle.sphere_box([2.0, 0.5, 0.5], np.nextafter(np.float32(1), np.float32(0)), box)
    assert oracle.sphere_box([0.5, 0.5, 0.5], 0.0, box)  # centre inside: d = 0
    assert oracle.box_box(box, np.array([1, 1, 1, 2, 2, 2], np.float32))  # shared corner
    assert not oracle.box_box(box, np.array([1.0000001, 0, 0, 2, 1, 1], np.float32))


@pytest.mark.parametrize("case", ["uniform", "duplicates", "collinear", "all_equal", "boxes", "box_queries"])
def test_traversal_equals_bruteforce(case):
    rng = np.random.default_rng(21)
    kind, qkind = oracle.POINTS, oracle.SPHERE
    if case == "uniform":
        prims = inputs.uniform_points(4096, seed=1)
    elif case == "duplicates":
        prims = inputs.duplicated_points(3000, 200, seed=2)
    elif case == "collinear":
        prims = inputs.collinear_points(2000, seed=3)
    elif case == "all_equal":
        prims = np.full((500, 3), 0.5, np.float32)
    else:
        prims = inputs.gaussian_mixture_boxes(3000, seed=4, components=8)
        kind = oracle.BOXES
    n = prims.shape[0]
    if case == "box_queries":
        queries = inputs.gaussian_mixture_boxes(700, seed=5, components=8, component_seed=4)
        qkind = oracle.BOX
        radii = None
    else:
        queries = rng.random((700, 3)).astype(np.float32)
        # some queries sit on primitives (box primitives: at their low corner)
        queries[:100] = prims[rng.integers(0, n, size=100), :3]
        radii = (rng.random(700) * 0.08).astype(np.float32)
    for bits in (30, 63):
        t = oracle.build(prims, kind, bits)
        off, hits = oracle.query(t, queries, qkind, radii=radii)
        boff, bhits = oracle.bruteforce(prims, kind, queries, qkind, radii=radii)
        assert np.array_equal(off, boff) and np.array_equal(hits, bhits)
    assert off[-1] > 0


def test_query_radius_scalar_and_self_hits():
    pts = inputs.uniform_points(16384, seed=0)
    r = inputs.radius_for_neighbours(16384)
    assert r == np.float32(0.061546564)
    t = oracle.build(pts, oracle.POINTS, 30)
    off, hits = oracle.query(t, pts[:500], oracle.SPHERE, radius=r)
    counts = np.diff(off)
    # every query centred at a primitive reports that primitive
    for q in range(500):
        assert q in hits[off[q]:off[q + 1]]
        seg = hits[off[q]:off[q + 1]]
        assert np.all(np.diff(seg.astype(np.int64)) > 0)
    assert 10 < counts.mean() < 20  # about 16 expected, fewer at the faces


# ---------------------------------------------------------------- the checks catch planted mistakes


def test_checks_catch_planted_mistakes():
    """A mistake planted in the oracle's output (wrong index, off by one,
    swapped operands) must fail one of the independent checks."""
    pts = inputs.uniform_points(300, seed=9)
    t = oracle.build(pts, oracle.POINTS, 30)
    s = t["sorted"]

    def fails(fn):
        try:
            fn()
        except AssertionError:
            return True
        return False

    left = t["left"].copy(); left[[5, 9]] = left[[9, 5]]
    assert fails(lambda: tc.check_karras_tree(s, left, t["right"]))
    right = t["right"].copy(); right[0] = t["left"][0]
    assert fails(lambda: tc.check_karras_tree(s, t["left"], right))
    si = t["skip_internal"].copy(); si[3] = si[3] + 1 if si[3] >= 0 else 0
    assert fails(lambda: tc.check_skips(s, t["left"], t["right"], si, t["skip_leaf"]))
    sl = t["skip_leaf"].copy(); sl[10] = 299 + 11
    assert fails(lambda: tc.check_skips(s, t["left"], t["right"], t["skip_internal"], sl))
    ib = t["internal_box"].copy(); ib[7, [0, 3]] = ib[7, [3, 0]]
    assert fails(lambda: tc.check_boxes(300, t["range_l"], t["range_r"], t["leaf_box"], ib))
    swapped = s.copy(); swapped[[40, 41]] = swapped[[41, 40]]
    if swapped[40] != swapped[41]:
        assert fails(lambda: tc.check_karras_tree(swapped, t["left"], t["right"]))


def test_nan_queries_hit_nothing_and_signed_zero_bounds():
    pts = inputs.uniform_points(300, seed=31)
    t = oracle.build(pts, oracle.POINTS, 30)
    q = np.array([[np.nan, 0.5, 0.5], [0.5, 0.5, 0.5], [np.inf, 0.5, 0.5]], np.float32)
    off, hits = oracle.query(t, q, oracle.SPHERE, radius=10.0)
    assert np.diff(off).tolist() == [0, 300, 0]
    off, _ = oracle.query(t, q[1:2], oracle.SPHERE, radius=np.nan)
    assert off.tolist() == [0, 0]
    # -0.0 orders below +0.0 in the bounds, whatever the input order
    for order in ([0.0, -0.0], [-0.0, 0.0]):
        p = np.array([[v, 1.0, 2.0] for v in order], np.float32)
        _, b = oracle.morton_codes(p, oracle.POINTS, 30)
        assert np.signbit(b[0]) and not np.signbit(b[3])


# ---------------------------------------------------------------- refit


@pytest.mark.parametrize("kind", [oracle.POINTS, oracle.BOXES])
def test_refit_keeps_topology_and_boxes_are_leaf_range_unions(kind):
    rng = np.random.default_rng(41)
    n = 700
    if kind == oracle.POINTS:
        a = inputs.uniform_points(n, seed=41)
        b = (a + rng.normal(0, 0.05, size=a.shape)).astype(np.float32)
    else:
        a = inputs.gaussian_mixture_boxes(n, seed=41, components=6)
        b = (a + np.repeat(rng.normal(0, 0.02, size=(n, 3)), 2, axis=0).reshape(n, 6)).astype(np.float32)
    t = oracle.build(a, kind, 30)
    r = oracle.refit(t, b)
    for k in ("perm", "sorted", "left", "right", "skip_internal", "skip_leaf", "range_l", "range_r"):
        assert np.array_equal(r[k], t[k]), k
    # leaf k holds primitive perm[k] of the new coordinates
    lb = b[t["perm"]] if kind == oracle.BOXES else np.concatenate([b[t["perm"]], b[t["perm"]]], axis=1)
    assert np.array_equal(r["leaf_box"].view(np.uint32), lb.view(np.uint32))
    # every internal box is the min/max over its leaf range (brute force)
    tc.check_boxes(n, t["range_l"], t["range_r"], r["leaf_box"], r["internal_box"])
    # the scene bounds are the new centroids' min/max
    c = b if kind == oracle.POINTS else (b[:, :3] + b[:, 3:]) * np.float32(0.5)
    assert np.array_equal(r["bounds"], np.concatenate([c.min(axis=0), c.max(axis=0)]).astype(np.float32))
    # refitting with the original coordinates gives the original tree back
    r0 = oracle.refit(t, a)
    for k in ("leaf_box", "internal_box", "bounds"):
        assert np.array_equal(r0[k].view(np.uint32), t[k].view(np.uint32)), k
    # a stale box is caught by the same check (the refit really changed boxes)
    with pytest.raises(AssertionError):
        tc.check_boxes(n, t["range_l"], t["range_r"], r["leaf_box"], t["internal_box"])


def test_refit_tree_queries_equal_bruteforce_on_moved_points():
    rng = np.random.default_rng(42)
    a = inputs.uniform_points(1500, seed=42)
    b = (a + rng.normal(0, 0.1, size=a.shape)).astype(np.float32)  # far moves: a poor but valid tree
    r = oracle.refit(oracle.build(a, oracle.POINTS, 63), b)
    q = inputs.uniform_points(300, seed=43)
    rad = np.float32(0.07)
    off, hits = oracle.query(r, q, oracle.SPHERE, radius=rad)
    boff, bhits = oracle.bruteforce(b, oracle.POINTS, q, oracle.SPHERE, radius=rad)
    assert np.array_equal(off, boff) and np.array_equal(hits, bhits)


# ---------------------------------------------------------------- ray queries


def _ray(o, d, tmin=0.0, tmax=np.inf):
    return np.array([o[0], o[1], o[2], tmin, d[0], d[1], d[2], tmax], np.float32)


def _slab_exact(ray, box):
    """The slab test in exact rational arithmetic (fractions): hit iff the
    closed segment meets the closed box. Infinite tmax is handled as
    unbounded."""
    from fractions import Fraction as F
    o = [F(float(v)) for v in ray[:3]]
    d = [F(float(v)) for v in ray[4:7]]
    tn = F(float(ray[3])) if np.isfinite(ray[3]) else None
    tf = F(float(ray[7])) if np.isfinite(ray[7]) else None
    for a in range(3):
        lo, hi = F(float(box[a])), F(float(box[3 + a]))
        if d[a] == 0:
            if not (lo <= o[a] <= hi):
                return False
            continue
        t1, t2 = (lo - o[a]) / d[a], (hi - o[a]) / d[a]
        t1, t2 = min(t1, t2), max(t1, t2)
        tn = t1 if tn is None or t1 > tn else tn
        tf = t2 if tf is None or t2 < tf else tf
    return tn is None or tf is None or tn <= tf


def test_ray_box_special_cases():
    box = np.array([0, 0, 0, 1, 1, 1], np.float32)
    assert oracle.ray_box(_ray([-1, 0.5, 0.5], [1, 0, 0]), box)            # through the middle
    assert not oracle.ray_box(_ray([-1, 0.5, 0.5], [-1, 0, 0]), box)       # pointing away
    assert not oracle.ray_box(_ray([-1, 0.5, 0.5], [1, 0, 0], tmax=0.5), box)  # stops short
    assert oracle.ray_box(_ray([-1, 0.5, 0.5], [1, 0, 0], tmax=1.0), box)      # reaches the face (closed)
    assert oracle.ray_box(_ray([0.5, 0.5, 0.5], [0, 0, 1], tmax=0.0), box)     # starts inside
    assert oracle.ray_box(_ray([-1, 1, 0.5], [1, 0, 0]), box)              # grazes an edge (closed)
    assert not oracle.ray_box(_ray([-1, 1.0000001, 0.5], [1, 0, 0]), box)  # parallel, just outside
    assert not oracle.ray_box(_ray([-1, 0.5, 0.5], [1, 0, 0], tmin=2.5), box)  # starts past it
    assert not oracle.ray_box(_ray([np.nan, 0.5, 0.5], [1, 0, 0]), box)
    assert not oracle.ray_box(_ray([-1, 0.5, 0.5], [1, 0, 0], tmax=np.nan), box)
    assert not oracle.ray_box(_ray([-1, 0.5, 0.5], [np.inf, 0, 0]), box)
    # a degenerate box (a point leaf) is hit by a ray through it
    pt = np.array([0.25, 0.5, 0.75, 0.25, 0.5, 0.75], np.float32)
    assert oracle.ray_box(_ray([0.25, 0.5, -3], [0, 0, 1]), pt)
    assert not oracle.ray_box(_ray([0.25, 0.5000001, -3], [0, 0, 1]), pt)


def test_ray_box_matches_exact_slab_test_away_from_the_boundary():
    rng = np.random.default_rng(51)
    agree = 0
    for _ in range(3000):
        lo = rng.random(3)
        box = np.concatenate([lo, lo + rng.random(3) * 0.3]).astype(np.float32)
        o = (rng.random(3) * 2 - 0.5).astype(np.float32)
        d = rng.normal(size=3).astype(np.float32)
        ray = _ray(o, d, 0.0, float(rng.choice([np.inf, 0.5, 2.0])))
        want = _slab_exact(ray, box)
        # skip rays within a relative 1e-5 of touching (rounding may decide those)
        eps = 1e-5
        grown = box.astype(np.float64) + np.array([-eps] * 3 + [eps] * 3)
        shrunk = box.astype(np.float64) + np.array([eps] * 3 + [-eps] * 3)
        if _slab_exact(ray, grown.astype(np.float32)) != _slab_exact(ray, shrunk.astype(np.float32)):
            continue
        assert oracle.ray_box(ray, box) == want
        agree += 1
    assert agree > 2500


def _slab_g14(ray, box):
    """Reading G14 with every FP32 operation rounded exactly (rationals, one
    rounding each): inv = 1/d; an axis with d = 0 or an infinite inv needs
    lo <= o <= hi; else t1 = (lo - o) * inv and t2 = (hi - o) * inv, each
    difference and product rounded; tnear = max(tmin, min t), tfar = min(tmax,
    max t); hit iff tnear <= tfar. A non-finite origin or direction, or a NaN
    tmin or tmax, hits nothing."""
    from fractions import Fraction
    F = lambda v: Fraction(float(v))
    if not (np.all(np.isfinite(ray[:3])) and np.all(np.isfinite(ray[4:7]))) or np.isnan(ray[3]) or np.isnan(ray[7]):
        return False
    tnear, tfar = np.float32(ray[3]), np.float32(ray[7])
    for a in range(3):
        o, d = ray[a], ray[4 + a]
        inv = np.float32(np.inf) if d == 0 else _rn32(Fraction(1) / F(d))
        if d == 0 or np.isinf(inv):
            if not (box[a] <= o <= box[3 + a]):
                return False
            continue
        t1 = _rn32(F(_rn32(F(box[a]) - F(o))) * F(inv))
        t2 = _rn32(F(_rn32(F(box[3 + a]) - F(o))) * F(inv))
        tlo, thi = (t1, t2) if t1 < t2 else (t2, t1)
        tnear = tlo if tlo > tnear else tnear
        tfar = thi if thi < tfar else tfar
    return bool(tnear <= tfar)


def test_ray_box_at_the_boundary_against_exact_rounding():
    """Rays aimed at points of a box's surface with the segment ending where
    the rounded slab test puts the entry (tmax = that tnear) or one FP32 step
    before or after it, so that tnear <= tfar is decided by the last bit: the
    oracle against reading G14 rounded exactly (no oracle code in the
    reference)."""
    rng = np.random.default_rng(53)
    cases = flips = 0
    for _ in range(800):
        lo = rng.random(3).astype(np.float32)
        box = np.concatenate([lo, (lo + rng.random(3) * 0.3).astype(np.float32)]).astype(np.float32)
        target = (box[:3] + rng.random(3).astype(np.float32) * (box[3:] - box[:3])).astype(np.float32)
        target[rng.integers(0, 3)] = box[rng.integers(0, 2) * 3 + rng.integers(0, 3)]  # onto a face plane
        o = (rng.random(3) * 3 - 1).astype(np.float32)
        d = (target - o).astype(np.float32)
        if not np.all(np.isfinite(d)) or np.all(d == 0):
            continue
        probe = _ray(o, d, 0.0, np.inf)
        # the rounded entry parameter: tnear of the unbounded segment
        tn = np.float32(0.0)
        for a in range(3):
            if d[a] != 0:
                from fractions import Fraction
                inv = _rn32(Fraction(1) / Fraction(float(d[a])))
                t1 = _rn32(Fraction(float(_rn32(Fraction(float(box[a])) - Fraction(float(o[a]))))) * Fraction(float(inv)))
                t2 = _rn32(Fraction(float(_rn32(Fraction(float(box[3 + a])) - Fraction(float(o[a]))))) * Fraction(float(inv)))
                tn = max(tn, min(t1, t2))
        results = []
        for tmax in (np.nextafter(tn, np.float32(-np.inf)), tn, np.nextafter(tn, np.float32(np.inf))):
            ray = _ray(o, d, 0.0, tmax)
            want = _slab_g14(ray, box)
            assert oracle.ray_box(ray, box) == want, (ray, box)
            results.append(want)
            cases += 1
        flips += int(results[0] != results[1])
        assert _slab_g14(probe, box) == oracle.ray_box(probe, box)
    assert cases > 2000 and flips > 100


@pytest.mark.parametrize("kind", [oracle.POINTS, oracle.BOXES])
def test_ray_traversal_equals_bruteforce(kind):
    rng = np.random.default_rng(52)
    n = 3000
    if kind == oracle.BOXES:
        prims = inputs.gaussian_mixture_boxes(n, seed=52, components=8, log_half_mu=math.log(0.01))
    else:
        prims = inputs.uniform_points(n, seed=52)
    t = oracle.build(prims, kind, 30)
    nr = 400
    o = rng.random((nr, 3)).astype(np.float32)
    d = rng.normal(size=(nr, 3)).astype(np.float32)
    rays = np.concatenate([o, np.zeros((nr, 1)), d, np.full((nr, 1), 0.3)], axis=1).astype(np.float32)
    if kind == oracle.POINTS:
        # axis-parallel rays through existing points: exact hits on degenerate boxes
        k = rng.integers(0, n, size=nr // 2)
        rays[: nr // 2, :3] = prims[k]
        rays[: nr // 2, 2] -= 0.1
        rays[: nr // 2, 4:7] = [0, 0, 1]
    off, hits = oracle.query(t, rays, oracle.RAY)
    boff, bhits = oracle.bruteforce(prims, kind, rays, oracle.RAY)
    assert np.array_equal(off, boff) and np.array_equal(hits, bhits)
    assert len(hits) >= nr // 2


# ---------------------------------------------------------------- k nearest neighbours


def test_knn_hand_computed_line():
    """Points at x = 0..4 on a line, a query at x = 2.4: distances 2.4, 1.4,
    0.4, 0.6, 1.6, so the order is 2, 3, 1, 4, 0."""
    pts = np.array([[x, 0.0, 0.0] for x in range(5)], np.float32)
    q = np.array([[2.4, 0.0, 0.0]], np.float32)
    idx, d2 = oracle.knn(pts, oracle.POINTS, q, 3)
    assert idx.tolist() == [[2, 3, 1]]
    assert np.allclose(d2, [[0.16, 0.36, 1.96]], rtol=1e-6)
    idx, _ = oracle.knn(pts, oracle.POINTS, q, 5)
    assert idx.tolist() == [[2, 3, 1, 4, 0]]


def test_knn_ties_go_to_the_lower_index_and_padding():
    # indices 0 and 1 are both at distance 1; 2 and 3 are the same point
    pts = np.array([[1, 0, 0], [-1, 0, 0], [0, 3, 0], [0, 3, 0]], np.float32)
    q = np.zeros((1, 3), np.float32)
    idx, d2 = oracle.knn(pts, oracle.POINTS, q, 6)
    assert idx.tolist() == [[0, 1, 2, 3, 0xFFFFFFFF, 0xFFFFFFFF]]
    assert d2[0, :4].tolist() == [1.0, 1.0, 9.0, 9.0] and np.isinf(d2[0, 4:]).all()
    # the reverse listing keeps the index order among equal distances
    idx, _ = oracle.knn(pts[::-1].copy(), oracle.POINTS, q, 4)
    assert idx.tolist() == [[2, 3, 0, 1]]
    # no primitives: nothing but padding
    idx, d2 = oracle.knn(np.zeros((0, 3), np.float32), oracle.POINTS, q, 2)
    assert idx.tolist() == [[0xFFFFFFFF] * 2] and np.isinf(d2).all()


def test_knn_non_finite_query_has_no_neighbours():
    pts = inputs.uniform_points(50, seed=3)
    q = np.array([[np.nan, 0.5, 0.5], [0.5, np.inf, 0.5], [0.5, 0.5, 0.5]], np.float32)
    idx, d2 = oracle.knn(pts, oracle.POINTS, q, 4)
    assert (idx[:2] == 0xFFFFFFFF).all() and np.isinf(d2[:2]).all()
    assert (idx[2] != 0xFFFFFFFF).all()


def test_knn_boxes_distance_is_the_gap_to_the_box():
    boxes = np.array([
        [0, 0, 0, 1, 1, 1],        # contains the query: distance 0
        [-1, -1, -1, 2, 2, 2],     # contains it too: distance 0, higher index
        [3, 0, 0, 4, 1, 1],        # 2.5 away along x
        [2, 2, 0, 3, 3, 1],        # (1.5, 1.5, 0) away: 4.5
    ], np.float32)
    q = np.array([[0.5, 0.5, 0.5]], np.float32)
    idx, d2 = oracle.knn(boxes, oracle.BOXES, q, 4)
    assert idx.tolist() == [[0, 1, 3, 2]]
    assert d2.tolist() == [[0.0, 0.0, 4.5, 6.25]]


def test_knn_distance_is_the_ball_test_distance():
    """d2 <= r*r exactly when the (separately pinned) ball test holds."""
    rng = np.random.default_rng(7)
    for _ in range(400):
        c = rng.random(3, dtype=np.float32)
        lo = rng.random(3, dtype=np.float32)
        box = np.concatenate([lo, lo + rng.random(3, dtype=np.float32) * np.float32(0.3)])
        d2 = oracle.point_box_d2(c, box)
        r = float(np.sqrt(np.float32(d2)))
        for rr in (np.nextafter(np.float32(r), np.float32(0)), np.float32(r), np.nextafter(np.float32(r), np.float32(9))):
            assert oracle.sphere_box(c, float(rr), box) == (d2 <= np.float32(rr) * np.float32(rr))


def test_knn_matches_float64_distances_away_from_ties():
    rng = np.random.default_rng(11)
    pts = rng.random((3000, 3), dtype=np.float32)
    q = rng.random((200, 3), dtype=np.float32)
    k = 16
    idx, d2 = oracle.knn(pts, oracle.POINTS, q, k)
    d64 = ((q[:, None, :].astype(np.float64) - pts[None, :, :].astype(np.float64)) ** 2).sum(axis=2)
    order = np.argsort(d64, axis=1, kind="stable")
    checked = 0
    for i in range(len(q)):
        s = np.sort(d64[i])
        if s[k] - s[k - 1] < 1e-5 or np.min(np.diff(s[:k + 1])) < 1e-6:
            continue  # a near tie FP32 may order either way
        assert idx[i].tolist() == order[i, :k].tolist()
        assert np.allclose(d2[i], s[:k], rtol=1e-5, atol=1e-7)
        checked += 1
    assert checked > 150
