"""The allocation-free construct (lbvh_construct_static) against the
allocating entry point (lbvh_build_from_sorted).

Some callers may not let this library allocate device memory (their own pool
owns the heap, or the code path must not call cudaMalloc/cudaFree, which
synchronise the device). lbvh_construct_static serves them: it runs the same
bottom-up pass with its scratch words in a file-scope device array, writing
into buffers the caller allocated. This file is collected last on purpose.
"""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

from paper_2402_00665_gb300 import _build, inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lbvh():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    _build.build()
    from paper_2402_00665_gb300 import lbvh as binding
    binding.load()
    return binding


def _decode(inodes, leaves, n, kind=0):
    """Canonical arrays from the node layout documented in include/lbvh.h."""
    ni = n - 1
    a = inodes.cpu().numpy().reshape(max(ni, 0), 2, 4) if ni > 0 else np.zeros((0, 2, 4), np.float32)
    if kind == 0:
        lv = leaves.cpu().numpy().reshape(n, 4)
        word = lv[:, 3].view(np.uint32)
        leaf_box = np.concatenate([lv[:, :3], lv[:, :3]], axis=1)
    else:
        lv = leaves.cpu().numpy().reshape(n, 2, 4)
        word = lv[:, 0, 3].view(np.uint32)
        leaf_box = np.concatenate([lv[:, 0, :3], lv[:, 1, :3]], axis=1)
    k = np.arange(n)
    skip_leaf = np.where(word & np.uint32(1 << 31), k + 1, ni + k + 1).astype(np.int32)
    skip_leaf[n - 1] = -1
    return {
        "left": a[:, 0, 3].view(np.int32), "skip_internal": a[:, 1, 3].view(np.int32),
        "internal_box": np.concatenate([a[:, 0, :3], a[:, 1, :3]], axis=1),
        "skip_leaf": skip_leaf, "leaf_box": leaf_box,
        "perm": word & np.uint32((1 << 31) - 1),
    }


def _static_call(lbvh, codes, perm, prims, n, kind=0, with_inodes=True):
    lib = lbvh.load()
    dc = torch.as_tensor(codes.view(np.int64)).cuda()
    dp = torch.as_tensor(perm.view(np.int32)).cuda()
    dx = torch.as_tensor(prims).cuda()
    inodes = torch.full((max(n - 1, 0) * 8,), np.nan, dtype=torch.float32, device="cuda")
    leaves = torch.full((n * (4 if kind == 0 else 8),), np.nan, dtype=torch.float32, device="cuda")
    flags = torch.zeros(1, dtype=torch.int32, device="cuda")
    P = lambda t: ctypes.c_void_p(t.data_ptr())
    st = lib.lbvh_construct_static(P(dc), P(dp), P(dx), n, kind, P(inodes) if with_inodes else None, P(leaves),
                                   P(flags), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return st, inodes, leaves, int(flags.item())


def _check_against_allocating(lbvh, codes, perm, prims, n, kind, with_inodes=True):
    st, inodes, leaves, flags = _static_call(lbvh, codes, perm, prims, n, kind, with_inodes)
    assert st == lbvh.OK and flags == 0
    got = _decode(inodes, leaves, n, kind)
    ref = lbvh.Tree().build_from_sorted(codes, perm, prims, kind)
    ref.check()
    want = ref.export()
    for k in ("left", "skip_internal", "skip_leaf", "perm"):
        assert np.array_equal(got[k], want[k]), k
    for k in ("internal_box", "leaf_box"):
        assert np.array_equal(got[k].view(np.uint32), want[k].view(np.uint32)), k
    ref.close()


def test_static_scratch_construct_matches_allocating_entry_point(lbvh):
    rng = np.random.default_rng(41)
    # two calls in a row on the shared scratch array (a larger one, then a smaller one)
    for n in ((1 << 20) + 1, 70001):
        codes = np.sort(rng.integers(0, 1 << 40, size=n, dtype=np.uint64) >> np.uint64(rng.integers(0, 30)))
        perm = rng.permutation(n).astype(np.uint32)
        pts = inputs.uniform_points(n, seed=int(n))
        st, inodes, leaves, flags = _static_call(lbvh, codes, perm, pts, n)
        assert st == lbvh.OK and flags == 0
        got = _decode(inodes, leaves, n)
        ref = lbvh.Tree().build_from_sorted(codes, perm, pts, lbvh.POINTS)
        ref.check()
        want = ref.export()
        for k in ("left", "skip_internal", "skip_leaf", "perm"):
            assert np.array_equal(got[k], want[k]), k
        for k in ("internal_box", "leaf_box"):
            assert np.array_equal(got[k].view(np.uint32), want[k].view(np.uint32)), k


def test_static_scratch_rejects_sizes_beyond_its_maximum(lbvh):
    lib = lbvh.load()
    dummy = ctypes.c_void_p(256)
    assert lib.lbvh_construct_static(dummy, dummy, dummy, (1 << 20) + 2, lbvh.POINTS, dummy, dummy, None,
                                     None) == lbvh.ERR_INVALID
    assert lib.lbvh_construct_static(dummy, dummy, dummy, 0, lbvh.POINTS, dummy, dummy, None,
                                     None) == lbvh.ERR_INVALID


def test_static_scratch_boxes_single_leaf_and_the_largest_size(lbvh):
    """Box leaves (two float4 per leaf), one primitive with no internal-node
    buffer at all, and exactly the largest accepted size."""
    rng = np.random.default_rng(43)
    n = 50001
    codes = np.sort(rng.integers(0, 1 << 30, size=n, dtype=np.uint64))
    perm = rng.permutation(n).astype(np.uint32)
    _check_against_allocating(lbvh, codes, perm, inputs.gaussian_mixture_boxes(n, seed=44), n, lbvh.BOXES)
    one = inputs.uniform_points(1, seed=45)
    _check_against_allocating(lbvh, np.zeros(1, np.uint64), np.zeros(1, np.uint32), one, 1, lbvh.POINTS,
                              with_inodes=False)
    n = (1 << 20) + 1  # LBVH_STATIC_MAX_PRIMS
    codes = np.sort(rng.integers(0, 1 << 62, size=n, dtype=np.uint64))
    perm = rng.permutation(n).astype(np.uint32)
    _check_against_allocating(lbvh, codes, perm, inputs.uniform_points(n, seed=46), n, lbvh.POINTS)
