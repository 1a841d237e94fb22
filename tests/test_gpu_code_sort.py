"""The sort of codes wider than 32 bits: top bits beside the index, then the
runs of equal top bits put in code order (in one thread, in one CTA, or by
the fallback full sort), each against the oracle's stable sort and build.

Clusters of nearly equal primitives give runs whose elements share their top
code bits but differ in the low bits (so the runs are really reordered), and
exact duplicates give runs of equal codes (ties kept in index order). The
cluster sizes straddle each tier's limit: 16 elements per thread, 4096 per
CTA, longer runs through the fallback.
"""
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


def clustered_points(sizes, singles: int, seed: int, jitter: float = 2e-6, exact: bool = False) -> np.ndarray:
    """One cluster per entry of `sizes` (that many points within `jitter` of a
    uniform centre, or exactly on it), `singles` uniform points, shuffled."""
    rng = np.random.default_rng(seed)
    parts = [rng.random((singles, 3), dtype=np.float32)]
    for m in sizes:
        c = rng.random(3, dtype=np.float32) * np.float32(0.98) + np.float32(0.01)
        if exact:
            parts.append(np.tile(c, (m, 1)))
        else:
            parts.append((c + rng.uniform(-jitter, jitter, (m, 3))).astype(np.float32))
    p = np.concatenate(parts).astype(np.float32)
    return p[rng.permutation(len(p))]


def boxes_around(points: np.ndarray, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    h = rng.uniform(0, 1e-6, points.shape).astype(np.float32)
    return np.concatenate([points - h, points + h], axis=1).astype(np.float32)


def skip_choice(skip: int) -> int:
    """The sort choice with the default tile shape and `skip` (1: the
    top-bits sort covers one byte fewer, so more elements share their sorted
    bits and go through the runs stage)."""
    return skip * (L().sort_variant_count() // 2)


def assert_build_equal(prims, kind, bits, skip=0):
    lbvh = L()
    t = lbvh.Tree()
    t.set_tuning(skip_choice(skip), -1)
    t.build(prims, kind, bits)
    t.check()
    g = t.export()
    o = oracle.build(prims, kind, bits)
    for k in ("perm", "sorted", "left", "skip_internal", "skip_leaf"):
        assert np.array_equal(g[k], o[k]), k
    for k in ("internal_box", "leaf_box"):
        assert np.array_equal(np.asarray(g[k]).view(np.uint32), np.asarray(o[k]).view(np.uint32)), k
    t.close()


RUN_SIZES = [2, 3, 4, 7, 15, 16, 17, 18, 33, 100, 255, 256, 257, 1000, 4095, 4096]


@pytest.mark.parametrize("skip", [0, 1])
@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("exact", [False, True])
def test_runs_below_the_fallback(kind, exact, skip):
    p = clustered_points(RUN_SIZES, 9000, seed=21 + exact, exact=exact)
    prims = p if kind == 0 else boxes_around(p, seed=22)
    assert_build_equal(prims, kind, 63, skip)


@pytest.mark.parametrize("skip", [0, 1])
@pytest.mark.parametrize("exact", [False, True])
def test_runs_through_the_fallback(exact, skip):
    # runs of 4097 and 6000 elements are too long for one CTA
    p = clustered_points([4097, 6000, 17, 3], 5000, seed=23 + exact, exact=exact)
    assert_build_equal(p, 0, 63, skip)


@pytest.mark.parametrize("skip", [0, 1])
@pytest.mark.parametrize("bits", [33, 45, 63])
def test_other_widths(bits, skip):
    p = clustered_points([2, 5, 20, 300], 20000, seed=25)
    assert_build_equal(p, 0, bits, skip)


@pytest.mark.parametrize("skip", [0, 1])
def test_many_short_runs_over_many_tiles(skip):
    # ~300k points in clusters of 1 to 8 (the mixture's run lengths), several
    # thousand CTAs of the runs kernel
    rng = np.random.default_rng(27)
    sizes = rng.integers(1, 9, size=60000).tolist()
    p = clustered_points(sizes, 30000, seed=28, jitter=1e-5)
    assert_build_equal(p, 0, 63, skip)


@pytest.mark.parametrize("skip", [0, 1])
@pytest.mark.parametrize("n", [1, 2, 3, 127, 128, 129, 255, 256, 257, 4097])
def test_small_sizes(n, skip):
    # index bits 1 .. 13: the first sorted byte holds index bits for most n
    p = inputs.duplicated_points(n, max(1, n // 3), seed=n)
    assert_build_equal(p, 0, 63, skip)


@pytest.mark.parametrize("n", [(1 << 16) + 3, (1 << 17) - 1, 300001])
@pytest.mark.parametrize("bits", [39, 45, 63])
def test_one_byte_fewer_leaves_more_runs(n, bits):
    """One top-bits pass fewer on uniform points: with index bits 17-19 the
    sorted word bits start at 24 instead of at the index's top, i.e. at code
    bit 23. With 39-bit codes 63-99% of the points then share their sorted
    bits with a neighbour (runs of up to 16), with 45-bit codes 2-7% (runs of
    up to 4), with 63-bit codes none: the runs stage puts them in code
    order."""
    p = inputs.uniform_points(n, seed=n % 1000)
    assert_build_equal(p, 0, bits, 1)


def test_sort_alone_at_two_million():
    """Only the permutation, against the oracle's codes and a stable argsort,
    at a size with index bits 21 (the first sorted byte holds index bits 16-20
    beside key bits)."""
    lbvh = L()
    n = (1 << 21) - 12345
    rng = np.random.default_rng(29)
    sizes = rng.integers(1, 6, size=n // 6).tolist()
    p = clustered_points(sizes, n - int(np.sum(sizes)), seed=30, jitter=3e-6)
    codes, _ = oracle.morton_codes(p, oracle.POINTS, 63)
    want = np.argsort(codes, kind="stable").astype(np.uint32)
    for skip in (0, 1):
        t = lbvh.Tree()
        t.set_tuning(skip_choice(skip), -1)
        t.build(p, lbvh.POINTS, 63)
        t.check()
        e = t.export()
        assert np.array_equal(e["perm"], want), skip
        assert np.array_equal(e["sorted"], codes[want]), skip
        t.close()

