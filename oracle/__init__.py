"""CPU oracle for the linear BVH with skip connections (arXiv 2402.00665).

TEST INFRASTRUCTURE ONLY. This package is the independent reference the CUDA
library is checked against. Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import it; the product path never
does, and the two share no code.

The arithmetic lives in ``lbvh_oracle.c`` (plain C99, ``-O2 -ffp-contract=off``,
single-threaded). This module compiles it with the system C compiler on first
use and wraps it with numpy-friendly functions. What each function computes,
and which passage of the paper it follows, is documented in ``lbvh_oracle.h``
and at the top of ``lbvh_oracle.c``:

* Morton codes - Sec. 3.1 step 1 (encoding fixed by the reading in the C file)
* sort - Sec. 3.1 step 2
* delta, topology - Sec. 3.1 and Sec. 3.2 (XOR, index-augmented keys)
* skips - Sec. 2 and Fig. 1 (pre-order successor past the subtree)
* boxes - Sec. 3.1 step 4
* queries - Algorithm 1, plus all-pairs brute force; predicates: closed ball,
  box overlap, and ray segment (slab test: Sec. 1 names both distance and
  ray range searches)
* refit - boxes (Sec. 3.1 step 4) recomputed on a kept topology
* k nearest neighbours - brute force in the order (squared distance, index),
  the distance being the ball test's d2 (the distance range search of Sec. 1
  asked for its k closest answers)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbvh_oracle.c")
_HDR = os.path.join(_HERE, "lbvh_oracle.h")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liblbvh_oracle.so")

POINTS, BOXES = 0, 1
SPHERE, BOX, RAY = 0, 1, 2
OK, INVALID, NONFINITE = 0, 1, 2

_lock = threading.Lock()
_lib = None


def build_library(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build`` (no-op when up to date)."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= newest:
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build_library())
        P = ctypes.c_void_p
        i64, i32, f32 = ctypes.c_int64, ctypes.c_int, ctypes.c_float
        sig = {
            "oracle_centroids": (i32, [P, i64, i32, P]),
            "oracle_scene_bounds": (i32, [P, i64, P]),
            "oracle_quantize": (ctypes.c_uint32, [f32, f32, f32, i32]),
            "oracle_interleave": (ctypes.c_uint64, [ctypes.c_uint32] * 3 + [i32]),
            "oracle_morton_codes": (i32, [P, i64, i32, i32, P, P]),
            "oracle_sort_codes": (i32, [P, i64, P, P]),
            "oracle_delta": (ctypes.c_int32, [P, i64, i64, i64]),
            "oracle_topology": (i32, [P, i64, P, P, P, P, P]),
            "oracle_skips": (i32, [i64, P, P, P, P, P]),
            "oracle_boxes": (i32, [P, i64, i32, P, P, P, P, P]),
            "oracle_build": (i32, [P, i64, i32, i32] + [P] * 13),
            "oracle_query_traverse": (i64, [i64, P, P, P, P, P, P, P, i64, i32, P, f32, P, P, i64]),
            "oracle_query_bruteforce": (i64, [P, i64, i32, P, i64, i32, P, f32, P, P, i64]),
            "oracle_sphere_box": (i32, [P, f32, P]),
            "oracle_box_box": (i32, [P, P]),
            "oracle_ray_box": (i32, [P, P]),
            "oracle_knn_bruteforce": (i32, [P, i64, i32, P, i64, i32, P, P]),
            "oracle_point_box_d2": (f32, [P, P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _ptr(a):
    return None if a is None else a.ctypes.data


class OracleError(RuntimeError):
    def __init__(self, status):
        super().__init__({INVALID: "invalid argument", NONFINITE: "non-finite input"}.get(status, f"status {status}"))
        self.status = status


def _prims(prims, kind):
    prims = np.ascontiguousarray(prims, dtype=np.float32)
    width = 3 if kind == POINTS else 6
    return prims.reshape(-1, width)


def quantize(c: float, lo: float, hi: float, b: int) -> int:
    return int(_load().oracle_quantize(np.float32(c), np.float32(lo), np.float32(hi), b))


def interleave(qx: int, qy: int, qz: int, b: int) -> int:
    return int(_load().oracle_interleave(qx, qy, qz, b))


def morton_codes(prims, kind=POINTS, bits=30):
    """Morton code per primitive and the scene bounds (Sec. 3.1 step 1)."""
    p = _prims(prims, kind)
    n = p.shape[0]
    codes = np.zeros(n, np.uint64)
    bounds = np.zeros(6, np.float32)
    st = _load().oracle_morton_codes(_ptr(p), n, kind, bits, _ptr(codes), _ptr(bounds))
    if st != OK:
        raise OracleError(st)
    return codes, bounds


def sort_codes(codes):
    codes = np.ascontiguousarray(codes, dtype=np.uint64)
    n = codes.shape[0]
    perm = np.zeros(n, np.uint32)
    sorted_ = np.zeros(n, np.uint64)
    st = _load().oracle_sort_codes(_ptr(codes), n, _ptr(perm), _ptr(sorted_))
    if st != OK:
        raise OracleError(st)
    return perm, sorted_


def delta(sorted_codes, i: int, j: int) -> int:
    s = np.ascontiguousarray(sorted_codes, dtype=np.uint64)
    return int(_load().oracle_delta(_ptr(s), s.shape[0], i, j))


def tree_from_sorted(sorted_codes):
    """Topology and skips for keys already in sorted order (golden tests)."""
    s = np.ascontiguousarray(sorted_codes, dtype=np.uint64)
    n = s.shape[0]
    ni = max(n - 1, 0)
    t = {k: np.zeros(ni, np.int32) for k in ("left", "right", "range_l", "range_r", "split", "skip_internal")}
    t["skip_leaf"] = np.zeros(n, np.int32)
    t["preorder"] = np.zeros(max(2 * n - 1, 0), np.int32)
    lib = _load()
    st = lib.oracle_topology(_ptr(s), n, _ptr(t["left"]), _ptr(t["right"]), _ptr(t["range_l"]),
                             _ptr(t["range_r"]), _ptr(t["split"]))
    if st == OK:
        st = lib.oracle_skips(n, _ptr(t["left"]), _ptr(t["right"]), _ptr(t["skip_internal"]),
                              _ptr(t["skip_leaf"]), _ptr(t["preorder"]))
    if st != OK:
        raise OracleError(st)
    t["n"] = n
    return t


def build(prims, kind=POINTS, bits=30):
    """The whole build; returns a dict of canonical arrays."""
    p = _prims(prims, kind)
    n = p.shape[0]
    ni = max(n - 1, 0)
    t = {
        "n": n, "kind": kind, "bits": bits,
        "codes": np.zeros(n, np.uint64), "bounds": np.zeros(6, np.float32),
        "perm": np.zeros(n, np.uint32), "sorted": np.zeros(n, np.uint64),
        "left": np.zeros(ni, np.int32), "right": np.zeros(ni, np.int32),
        "skip_internal": np.zeros(ni, np.int32), "skip_leaf": np.zeros(n, np.int32),
        "range_l": np.zeros(ni, np.int32), "range_r": np.zeros(ni, np.int32),
        "split": np.zeros(ni, np.int32),
        "leaf_box": np.zeros((n, 6), np.float32), "internal_box": np.zeros((ni, 6), np.float32),
    }
    st = _load().oracle_build(
        _ptr(p), n, kind, bits, _ptr(t["codes"]), _ptr(t["bounds"]), _ptr(t["perm"]),
        _ptr(t["sorted"]), _ptr(t["left"]), _ptr(t["right"]), _ptr(t["skip_internal"]),
        _ptr(t["skip_leaf"]), _ptr(t["range_l"]), _ptr(t["range_r"]), _ptr(t["split"]),
        _ptr(t["leaf_box"]), _ptr(t["internal_box"]))
    if st != OK:
        raise OracleError(st)
    return t


def refit(tree, prims):
    """Refit (box update on a fixed topology): a copy of `tree` whose leaf and
    internal boxes and scene bounds come from `prims` (the same n and kind, the
    same index order), with codes, permutation, children and skips unchanged.
    The boxes are Karras step 4 over the kept topology, by the same post-order
    routine as a build."""
    p = _prims(prims, tree["kind"])
    n = tree["n"]
    if p.shape[0] != n:
        raise OracleError(INVALID)
    t = dict(tree)
    t["leaf_box"] = np.zeros((n, 6), np.float32)
    t["internal_box"] = np.zeros((max(n - 1, 0), 6), np.float32)
    t["bounds"] = np.zeros(6, np.float32)
    lib = _load()
    st = OK
    if n > 0:
        c = np.zeros((n, 3), np.float32)
        st = lib.oracle_centroids(_ptr(p), n, tree["kind"], _ptr(c))
        if st == OK:
            st = lib.oracle_scene_bounds(_ptr(c), n, _ptr(t["bounds"]))
    if st == OK:
        st = lib.oracle_boxes(_ptr(p), n, tree["kind"], _ptr(tree["perm"]), _ptr(tree["left"]),
                              _ptr(tree["right"]), _ptr(t["leaf_box"]), _ptr(t["internal_box"]))
    if st != OK:
        raise OracleError(st)
    return t


def _queries(queries, qkind):
    q = np.ascontiguousarray(queries, dtype=np.float32)
    return q.reshape(-1, {SPHERE: 3, BOX: 6, RAY: 8}[qkind])


def _radii(radii, nq):
    if radii is None:
        return None
    r = np.ascontiguousarray(radii, dtype=np.float32).reshape(-1)
    assert r.shape[0] == nq
    return r


def query(tree, queries, qkind=SPHERE, radius=0.0, radii=None):
    """Algorithm 1 for every query; returns CSR (offsets int64[nq+1], hits uint32)."""
    q = _queries(queries, qkind)
    nq = q.shape[0]
    r = _radii(radii, nq)
    offsets = np.zeros(nq + 1, np.int64)
    lib = _load()
    args = (tree["n"], _ptr(tree["left"]), _ptr(tree["skip_internal"]), _ptr(tree["skip_leaf"]),
            _ptr(tree["leaf_box"]), _ptr(tree["internal_box"]), _ptr(tree["perm"]),
            _ptr(q), nq, qkind, _ptr(r), np.float32(radius))
    total = lib.oracle_query_traverse(*args, _ptr(offsets), None, 0)
    if total < 0:
        raise OracleError(INVALID)
    hits = np.zeros(total, np.uint32)
    total2 = lib.oracle_query_traverse(*args, _ptr(offsets), _ptr(hits), total)
    assert total2 == total
    return offsets, hits


def bruteforce(prims, kind, queries, qkind=SPHERE, radius=0.0, radii=None):
    """All-pairs predicate evaluation; same CSR convention as ``query``."""
    p = _prims(prims, kind)
    q = _queries(queries, qkind)
    nq = q.shape[0]
    r = _radii(radii, nq)
    offsets = np.zeros(nq + 1, np.int64)
    lib = _load()
    args = (_ptr(p), p.shape[0], kind, _ptr(q), nq, qkind, _ptr(r), np.float32(radius))
    total = lib.oracle_query_bruteforce(*args, _ptr(offsets), None, 0)
    if total < 0:
        raise OracleError(INVALID)
    hits = np.zeros(total, np.uint32)
    lib.oracle_query_bruteforce(*args, _ptr(offsets), _ptr(hits), total)
    return offsets, hits


def sphere_box(centre, radius, box6) -> bool:
    c = np.ascontiguousarray(centre, dtype=np.float32)
    b = np.ascontiguousarray(box6, dtype=np.float32)
    return bool(_load().oracle_sphere_box(_ptr(c), np.float32(radius), _ptr(b)))


def ray_box(ray8, box6) -> bool:
    r = np.ascontiguousarray(ray8, np.float32)
    b = np.ascontiguousarray(box6, np.float32)
    return bool(_load().oracle_ray_box(_ptr(r), _ptr(b)))


def box_box(a6, b6) -> bool:
    a = np.ascontiguousarray(a6, dtype=np.float32)
    b = np.ascontiguousarray(b6, dtype=np.float32)
    return bool(_load().oracle_box_box(_ptr(a), _ptr(b)))


def knn(prims, kind, queries, k: int):
    """Brute-force k nearest neighbours: (idx uint32[nq, k], d2 float32[nq, k]),
    each row in the order (squared distance, primitive index), padded with
    0xffffffff / +inf past min(k, n); a query with a non-finite coordinate
    has no neighbours."""
    lib = _load()
    p = _prims(prims, kind)
    q = np.ascontiguousarray(queries, np.float32).reshape(-1, 3)
    nq = q.shape[0]
    idx = np.empty((nq, k), np.uint32)
    d2 = np.empty((nq, k), np.float32)
    st = lib.oracle_knn_bruteforce(_ptr(p), p.shape[0], kind, _ptr(q), nq, int(k), _ptr(idx), _ptr(d2))
    if st != OK:
        raise OracleError(st)
    return idx, d2


def point_box_d2(point, box6) -> float:
    lib = _load()
    c = np.ascontiguousarray(point, np.float32)
    b = np.ascontiguousarray(box6, np.float32)
    return float(lib.oracle_point_box_d2(_ptr(c), _ptr(b)))
