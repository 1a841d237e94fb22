"""The C-ABI library builds for sm_103a, loads without a GPU, and exports every
function that ``include/lbvh.h`` declares; the binding refuses to run without a
GPU (no CPU fallback)."""
from __future__ import annotations

import ctypes
import os
import re

import pytest

from paper_2402_00665_gb300 import _build, lbvh

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]


def declared_functions():
    names = []
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[\w\s\*]+?\b(lbvh_\w+)\s*\(", text, flags=re.M):
            names.append(m.group(1))
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib_path():
    return _build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("lbvh_build", "lbvh_query", "lbvh_query_into", "lbvh_tree_export",
                     "lbvh_tree_bytes", "lbvh_free", "lbvh_tree_destroy", "lbvh_status_str"):
        assert required in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol():
    assert sorted(lbvh.SIGNATURES) == declared_functions()


def test_library_is_built_for_sm_103a_only():
    assert _build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_status_strings_without_gpu(lib_path):
    lib = lbvh.load()
    assert lib.lbvh_status_str(0) == b"LBVH_OK"
    assert lib.lbvh_status_str(7) == b"LBVH_ERR_CAPACITY"
    assert lib.lbvh_status_str(99) == b"LBVH_ERR_UNKNOWN"


def test_invalid_arguments_rejected_before_any_device_work(lib_path):
    lib = lbvh.load()
    assert lib.lbvh_tree_create(None) == lbvh.ERR_INVALID
    h = ctypes.c_void_p()
    assert lib.lbvh_tree_create(ctypes.byref(h)) == lbvh.OK
    try:
        assert lib.lbvh_build(h, None, 10, 0, 30, None) == lbvh.ERR_INVALID  # null prims
        assert lib.lbvh_build(h, None, -1, 0, 30, None) == lbvh.ERR_INVALID
        assert lib.lbvh_build(h, None, lbvh.MAX_PRIMS + 1, 0, 30, None) == lbvh.ERR_INVALID
        dummy = ctypes.c_void_p(16)
        for bits in (0, 2, 31, 64):
            assert lib.lbvh_build(h, dummy, 10, 0, bits, None) == lbvh.ERR_INVALID
        assert lib.lbvh_build(h, dummy, 10, 7, 30, None) == lbvh.ERR_INVALID  # kind
        # querying a tree that was never built
        off = ctypes.c_void_p(16)
        total = ctypes.c_uint64()
        assert lib.lbvh_query_into(h, dummy, 1, 0, None, 1.0, off, None, 0, ctypes.byref(total),
                                   None) == lbvh.ERR_INVALID
        assert lib.lbvh_query_into_host(h, dummy, 1, 0, None, 1.0, off, None, 0, ctypes.byref(total),
                                        None) == lbvh.ERR_INVALID
        assert lib.lbvh_tree_status(h) == lbvh.ERR_INVALID
        # the host-output chunk setting: 0 (default) to 16
        for chunks, want in ((-1, lbvh.ERR_INVALID), (17, lbvh.ERR_INVALID), (0, lbvh.OK), (1, lbvh.OK),
                             (16, lbvh.OK)):
            assert lib.lbvh_tree_set_host_chunks(h, chunks) == want
        assert lib.lbvh_tree_set_host_chunks(None, 1) == lbvh.ERR_INVALID
        # the construct's jitter test hook: up to 10^6 ns, then off again
        assert lib.lbvh_test_construct_jitter(7, 1000001) == lbvh.ERR_INVALID
        assert lib.lbvh_test_construct_jitter(7, 1000) == lbvh.OK
        assert lib.lbvh_test_construct_jitter(0, 0) == lbvh.OK
        # checkpoint images are validated before any device work
        size = ctypes.c_uint64()
        assert lib.lbvh_tree_save(h, None, 0, ctypes.byref(size)) == lbvh.ERR_INVALID  # never built
        good_header = b"LBVHTREE" + (1).to_bytes(4, "little") + bytes(52)  # n = 0, points
        assert lib.lbvh_tree_load(h, b"NOTATREE" + bytes(56), 64, None) == lbvh.ERR_INVALID
        assert lib.lbvh_tree_load(h, b"LBVHTREE" + (2).to_bytes(4, "little") + bytes(52), 64,
                                  None) == lbvh.ERR_INVALID  # version
        assert lib.lbvh_tree_load(h, good_header, 63, None) == lbvh.ERR_INVALID  # truncated
        assert lib.lbvh_tree_load(h, good_header + bytes(8), 72, None) == lbvh.ERR_INVALID  # size vs n
        bad_kind = b"LBVHTREE" + (1).to_bytes(4, "little") + (5).to_bytes(4, "little") + bytes(48)
        assert lib.lbvh_tree_load(h, bad_kind, 64, None) == lbvh.ERR_INVALID
    finally:
        lib.lbvh_tree_destroy(h)


def test_binding_fails_loudly_without_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(RuntimeError, match="no CUDA device"):
        lbvh.Tree().build([[0.0, 0.0, 0.0]])


def test_tune_cache_file_round_trip_without_a_gpu(lib_path, tmp_path):
    """The tuner's cache file is read and written on the host alone."""
    import json
    lib = lbvh.load(lib_path)
    lib.lbvh_tune_clear()
    good = tmp_path / "tune.json"
    good.write_text(json.dumps({"lbvh_tune_cache": 1, "entries": [
        {"gpu": "NVIDIA GB300", "n_log2": 25, "bits": 63, "kind": 0, "qkind": -1, "instances": 1,
         "sort_variant": 1, "sort_ms": 2.27, "walk_variant": -1, "walk_ms": 0},
        {"gpu": "NVIDIA GB300", "n_log2": 25, "bits": 63, "kind": 0, "qkind": 0, "instances": 1,
         "sort_variant": -1, "sort_ms": 0, "walk_variant": 3, "walk_ms": 15.5},
        {"gpu": 'other "quoted" gpu', "n_log2": 10, "bits": 30, "kind": 1, "qkind": 1, "instances": 4096,
         "sort_variant": 99, "sort_ms": 1.0, "walk_variant": 1, "walk_ms": 0.5}]}))
    assert lib.lbvh_tune_load(os.fsencode(str(good))) == lbvh.OK
    assert lib.lbvh_tune_entries() == 3
    out = tmp_path / "saved.json"
    assert lib.lbvh_tune_save(os.fsencode(str(out))) == lbvh.OK
    saved = json.load(open(out))["entries"]
    by_gpu = {(e["gpu"], e["qkind"]): e for e in saved}
    assert by_gpu[("NVIDIA GB300", -1)]["sort_variant"] == 1
    assert by_gpu[("NVIDIA GB300", 0)]["walk_variant"] == 3
    # a variant index the library does not have is dropped on load
    assert by_gpu[('other "quoted" gpu', 1)]["sort_variant"] == -1
    assert by_gpu[('other "quoted" gpu', 1)]["walk_variant"] == 1
    bad = tmp_path / "bad.json"
    for text in ("", "{", '{"entries": [{"gpu": 3}]}', '{"entries": [{"n_log2": 1}]}', "not json"):
        bad.write_text(text)
        assert lib.lbvh_tune_load(os.fsencode(str(bad))) == lbvh.ERR_INVALID
    assert lib.lbvh_tune_load(os.fsencode(str(tmp_path / "missing.json"))) == lbvh.ERR_INVALID
    assert lib.lbvh_tune_entries() == 3  # a failed load leaves the cache as it was
    lib.lbvh_tune_clear()
    assert lib.lbvh_tune_entries() == 0
