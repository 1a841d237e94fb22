"""Python binding of the C ABI in ``include/lbvh.h`` (ctypes).

Argument marshalling only: every step of the build and the query runs in the
CUDA kernels of ``liblbvh_gb300.so``. PyTorch supplies device memory and the
current stream. There is no CPU fallback: if the library has not been built
(``__graft_entry__.build()`` or ``python -m paper_2402_00665_gb300._build``)
or no GPU is present, the calls raise.

The names follow the C functions: ``Tree.build`` = ``lbvh_build``,
``Tree.query`` = ``lbvh_query_into`` and so on.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import _build

POINTS, BOXES = 0, 1
SPHERE, BOX, RAY = 0, 1, 2
MAX_PRIMS = (1 << 30) - 1
MAX_BATCH = 1 << 20
KNN_MAX_K = 256
SERVER_PHASES = 4
BUILD_MODIFIED_APETREI, BUILD_KARRAS, BUILD_APETREI = 0, 1, 2
_QDIM = {SPHERE: 3, BOX: 6, RAY: 8}
STAGE_COUNT = 18

STATUS = {0: "LBVH_OK", 1: "LBVH_ERR_INVALID", 2: "LBVH_ERR_NONFINITE", 3: "LBVH_ERR_OOM",
          4: "LBVH_ERR_CUDA", 5: "LBVH_ERR_TIMEOUT", 6: "LBVH_ERR_CORRUPT", 7: "LBVH_ERR_CAPACITY"}
OK, ERR_INVALID, ERR_NONFINITE, ERR_OOM, ERR_CUDA, ERR_TIMEOUT, ERR_CORRUPT, ERR_CAPACITY = range(8)

# every function declared in include/lbvh.h, with its ctypes signature
_P = ctypes.c_void_p
_I64, _U64, _I32, _F32 = ctypes.c_int64, ctypes.c_uint64, ctypes.c_int, ctypes.c_float
SIGNATURES = {
    "lbvh_tree_create": (_I32, [_P]),
    "lbvh_tree_destroy": (None, [_P]),
    "lbvh_build": (_I32, [_P, _P, _I64, _I32, _I32, _P]),
    "lbvh_build_from_sorted": (_I32, [_P, _P, _P, _P, _I64, _I32, _P]),
    "lbvh_tree_status": (_I32, [_P]),
    "lbvh_tree_size": (_I32, [_P, _P]),
    "lbvh_tree_bytes": (_I32, [_P, _P]),
    "lbvh_tree_export": (_I32, [_P] * 9),
    "lbvh_query_into": (_I32, [_P, _P, _I64, _I32, _P, _F32, _P, _P, _U64, _P, _P]),
    "lbvh_query_into_host": (_I32, [_P, _P, _I64, _I32, _P, _F32, _P, _P, _U64, _P, _P]),
    "lbvh_query": (_I32, [_P, _P, _I64, _I32, _P, _F32, _P, _P, _P, _P]),
    "lbvh_free": (None, [_P]),
    "lbvh_knn": (_I32, [_P, _P, _I64, _I32, _P, _P, _P]),
    "lbvh_tree_walk_visits": (_I32, [_P, _P, _I64, _I32, _P, _F32, _P, _P, _P]),
    "lbvh_morton_codes": (_I32, [_P, _I64, _I32, _I32, _P, _P, _P]),
    "lbvh_sort_pairs": (_I32, [_P, _P, _I64, _I32, _P, _P, _P]),
    "lbvh_batch_create": (_I32, [_P]),
    "lbvh_batch_destroy": (None, [_P]),
    "lbvh_batch_build_query": (_I32, [_P, _P, _P, _I64, _I32, _I32, _P, _P, _I32, _P, _F32, _P, _P, _U64, _P, _P]),
    "lbvh_batch_export": (_I32, [_P, _I64] + [_P] * 8),
    "lbvh_batch_sort_variant": (_I32, [_P, _P]),
    "lbvh_server_create": (_I32, [_U64, _I32, _I32, _P]),
    "lbvh_server_submit": (_I32, [_P, _P, _P]),
    "lbvh_server_wait": (_I32, [_P, _U64, _P]),
    "lbvh_server_stats": (_I32, [_P, _P, _P, _P, _P]),
    "lbvh_server_phase_seconds": (_I32, [_P, _P]),
    "lbvh_server_device_spans": (_I32, [_P, _P, _U64, _P]),
    "lbvh_server_latency": (_I32, [_P, _P, _P, _P]),
    "lbvh_release_cached_memory": (_I32, []),
    "lbvh_refit": (_I32, [_P, _P, _P]),
    "lbvh_test_hold_sort_tile": (_I32, [_I64]),
    "lbvh_test_construct_jitter": (_I32, [ctypes.c_uint64, ctypes.c_uint32]),
    "lbvh_tree_save": (_I32, [_P, _P, _U64, _P]),
    "lbvh_tree_load": (_I32, [_P, _P, _U64, _P]),
    "lbvh_build_variant": (_I32, [_P, _P, _I64, _I32, _I32, _I32, _P]),
    "lbvh_server_destroy": (None, [_P]),
    "lbvh_construct_static": (_I32, [_P, _P, _P, _I64, _I32, _P, _P, _P, _P]),
    "lbvh_tree_set_profiling": (_I32, [_P, _I32]),
    "lbvh_sort_variant_count": (_I32, []),
    "lbvh_walk_variant_count": (_I32, []),
    "lbvh_tree_autotune": (_I32, [_P, _P, _I64, _I32, _I32, _P, _I64, _I32, _P, _F32, _P, _P, _P]),
    "lbvh_tree_set_tuning": (_I32, [_P, _I32, _I32]),
    "lbvh_tree_set_host_chunks": (_I32, [_P, _I32]),
    "lbvh_tune_save": (_I32, [ctypes.c_char_p]),
    "lbvh_tune_load": (_I32, [ctypes.c_char_p]),
    "lbvh_tune_clear": (None, []),
    "lbvh_tune_entries": (_I32, []),
    "lbvh_tree_stage_times": (_I32, [_P, _P]),
    "lbvh_stage_name": (ctypes.c_char_p, [_I32]),
    "lbvh_kernel_launches": (_U64, []),
    "lbvh_status_str": (ctypes.c_char_p, [_I32]),
    "lbvh_last_cuda_error": (ctypes.c_char_p, []),
}

_lock = threading.Lock()
_lib = None


class LbvhError(RuntimeError):
    def __init__(self, status: int, where: str = ""):
        msg = f"{where}: {STATUS.get(status, status)}"
        if status == ERR_CUDA and _lib is not None:
            msg += f" ({_lib.lbvh_last_cuda_error().decode()})"
        super().__init__(msg)
        self.status = status


def library_path() -> str:
    return _build.LIB


def load(path: str | None = None):
    """Load the CUDA library (it must have been built); raises if missing."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = path or library_path()
        if not os.path.exists(path):
            raise RuntimeError(
                f"CUDA library not built ({path} missing); run __graft_entry__.build() first")
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _check(status: int, where: str):
    if status != OK:
        raise LbvhError(status, where)


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("no CUDA device: the LBVH library runs on the GPU only")
    return torch


def _stream(stream=None):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dev(t, dtype, width=None):
    torch = _torch()
    if not isinstance(t, torch.Tensor):
        t = torch.as_tensor(np.ascontiguousarray(t))
    t = t.to(device="cuda", dtype=dtype).contiguous()
    if width is not None:
        t = t.reshape(-1, width)
    return t


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None and t.numel() > 0 else ctypes.c_void_p(0)


class Tree:
    """A device-resident LBVH (handle of ``lbvh_tree_t``)."""

    def __init__(self):
        self._lib = load()
        h = ctypes.c_void_p()
        _check(self._lib.lbvh_tree_create(ctypes.byref(h)), "lbvh_tree_create")
        self._h = h
        self._keep = None
        self.kind = POINTS

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._lib.lbvh_tree_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def build(self, prims, kind: int = POINTS, morton_bits: int = 30, stream=None,
              algorithm: int | None = None) -> "Tree":
        """lbvh_build, or lbvh_build_variant when `algorithm` is given."""
        torch = _torch()
        p = _dev(prims, torch.float32, 3 if kind == POINTS else 6)
        if algorithm is None:
            _check(self._lib.lbvh_build(self._h, _ptr(p), p.shape[0], kind, morton_bits, _stream(stream)),
                   "lbvh_build")
        else:
            _check(self._lib.lbvh_build_variant(self._h, _ptr(p), p.shape[0], kind, morton_bits, algorithm,
                                                _stream(stream)), "lbvh_build_variant")
        self._keep = p  # the kernels read it asynchronously
        self.kind = kind
        return self

    def save(self) -> bytes:
        """lbvh_tree_save: the tree as one flat byte image."""
        size = ctypes.c_uint64()
        _check(self._lib.lbvh_tree_save(self._h, None, 0, ctypes.byref(size)), "lbvh_tree_save")
        buf = ctypes.create_string_buffer(size.value)
        _check(self._lib.lbvh_tree_save(self._h, buf, size.value, ctypes.byref(size)), "lbvh_tree_save")
        return buf.raw

    def load(self, image: bytes, stream=None) -> "Tree":
        """lbvh_tree_load: replace this tree with a saved image."""
        _check(self._lib.lbvh_tree_load(self._h, image, len(image), _stream(stream)), "lbvh_tree_load")
        self.kind = int.from_bytes(image[12:16], "little")
        return self

    def refit(self, prims, stream=None) -> "Tree":
        """lbvh_refit: new boxes from moved primitives, same topology."""
        torch = _torch()
        p = _dev(prims, torch.float32, 3 if self.kind == POINTS else 6)
        _check(self._lib.lbvh_refit(self._h, _ptr(p), _stream(stream)), "lbvh_refit")
        self._keep = p
        return self

    def build_from_sorted(self, sorted_codes, perm, prims, kind: int = POINTS, stream=None) -> "Tree":
        torch = _torch()
        c = _dev(np.asarray(sorted_codes, np.uint64).view(np.int64), torch.int64)
        pm = _dev(np.asarray(perm, np.uint32).view(np.int32), torch.int32)
        p = _dev(prims, torch.float32, 3 if kind == POINTS else 6)
        _check(self._lib.lbvh_build_from_sorted(self._h, _ptr(c), _ptr(pm), _ptr(p), c.shape[0], kind,
                                                _stream(stream)), "lbvh_build_from_sorted")
        self._keep = (c, pm, p)
        self.kind = kind
        return self

    def status(self) -> int:
        return self._lib.lbvh_tree_status(self._h)

    def check(self):
        _check(self.status(), "lbvh_tree_status")

    def size(self) -> int:
        n = ctypes.c_int64()
        _check(self._lib.lbvh_tree_size(self._h, ctypes.byref(n)), "lbvh_tree_size")
        return n.value

    def device_bytes(self) -> int:
        b = ctypes.c_uint64()
        _check(self._lib.lbvh_tree_bytes(self._h, ctypes.byref(b)), "lbvh_tree_bytes")
        return b.value

    def autotune(self, prims, kind: int = POINTS, morton_bits: int = 30, queries=None, qkind: int = SPHERE,
                 radius: float = 0.0, radii=None, stream=None) -> tuple:
        """lbvh_tree_autotune: times every sort (and, with queries, every walk)
        variant on these inputs, caches the fastest; returns (sort, walk)."""
        torch = _torch()
        p = _dev(prims, torch.float32, 3 if kind == POINTS else 6)
        q, nq, r = None, 0, None
        if queries is not None:
            q = _dev(queries, torch.float32, _QDIM[qkind])
            nq = q.shape[0]
            r = _dev(radii, torch.float32) if radii is not None else None
        sv, wv = ctypes.c_int(), ctypes.c_int()
        _check(self._lib.lbvh_tree_autotune(self._h, _ptr(p), p.shape[0], kind, morton_bits,
                                            _ptr(q) if q is not None else None, nq, qkind,
                                            _ptr(r) if r is not None else None, float(radius), _stream(stream),
                                            ctypes.byref(sv), ctypes.byref(wv)), "lbvh_tree_autotune")
        self._keep = (p, q, r)
        self.kind = kind
        return sv.value, wv.value

    def set_tuning(self, sort_variant: int = -1, walk_variant: int = -1):
        """lbvh_tree_set_tuning: fix this tree's variants (-1: the cache's choice)."""
        _check(self._lib.lbvh_tree_set_tuning(self._h, int(sort_variant), int(walk_variant)),
               "lbvh_tree_set_tuning")

    def set_host_chunks(self, max_chunks: int = 0):
        """lbvh_tree_set_host_chunks: the most chunks query_into_host cuts the queries into (0: default)."""
        _check(self._lib.lbvh_tree_set_host_chunks(self._h, int(max_chunks)), "lbvh_tree_set_host_chunks")

    def set_profiling(self, on: bool = True):
        _check(self._lib.lbvh_tree_set_profiling(self._h, int(bool(on))), "lbvh_tree_set_profiling")

    def stage_times(self) -> dict:
        """{stage name: device ms} of the last build and query (timed stages only)."""
        ms = (ctypes.c_float * STAGE_COUNT)()
        _check(self._lib.lbvh_tree_stage_times(self._h, ms), "lbvh_tree_stage_times")
        out = {}
        for k in range(STAGE_COUNT):
            if ms[k] == ms[k]:  # not NaN
                out[self._lib.lbvh_stage_name(k).decode()] = float(ms[k])
        return out

    def export(self) -> dict:
        """Canonical arrays of the last build, copied to host numpy arrays."""
        n = self.size()
        ni = max(n - 1, 0)
        out = {
            "n": n,
            "perm": np.zeros(n, np.uint32), "sorted": np.zeros(n, np.uint64),
            "left": np.zeros(ni, np.int32), "skip_internal": np.zeros(ni, np.int32),
            "skip_leaf": np.zeros(n, np.int32), "internal_box": np.zeros((ni, 6), np.float32),
            "leaf_box": np.zeros((n, 6), np.float32), "bounds": np.zeros(6, np.float32),
        }
        a = [ctypes.c_void_p(out[k].ctypes.data) for k in
             ("perm", "sorted", "left", "skip_internal", "skip_leaf", "internal_box", "leaf_box", "bounds")]
        _check(self._lib.lbvh_tree_export(self._h, *a), "lbvh_tree_export")
        return out

    def query_into(self, queries, qkind, offsets, hits, radius: float = 0.0, radii=None, stream=None):
        """lbvh_query_into with caller tensors; returns (status, total)."""
        torch = _torch()
        q = _dev(queries, torch.float32, _QDIM[qkind])
        r = None if radii is None else _dev(radii, torch.float32).reshape(-1)
        total = ctypes.c_uint64()
        cap = 0 if hits is None else hits.numel()
        st = self._lib.lbvh_query_into(self._h, _ptr(q), q.shape[0], qkind, _ptr(r), float(radius),
                                       _ptr(offsets), _ptr(hits), cap, ctypes.byref(total),
                                       _stream(stream))
        return st, total.value

    def query_into_host(self, queries, qkind, offsets, hits, radius: float = 0.0, radii=None, stream=None):
        """lbvh_query_into_host: the CSR into page-locked host tensors
        (``pin_memory()``), chunk copies overlapped with the next chunk's walk;
        complete once the stream is synchronised. Returns (status, total)."""
        torch = _torch()
        q = _dev(queries, torch.float32, _QDIM[qkind])
        r = None if radii is None else _dev(radii, torch.float32).reshape(-1)
        total = ctypes.c_uint64()
        cap = 0 if hits is None else hits.numel()
        st = self._lib.lbvh_query_into_host(self._h, _ptr(q), q.shape[0], qkind, _ptr(r), float(radius),
                                            _ptr(offsets), _ptr(hits), cap, ctypes.byref(total),
                                            _stream(stream))
        return st, total.value

    def walk_visits(self, queries, qkind: int = SPHERE, radius: float = 0.0, radii=None, stream=None) -> tuple:
        """lbvh_tree_walk_visits: (leaf visits, internal-node visits) of Algorithm 1 over these queries."""
        torch = _torch()
        q = _dev(queries, torch.float32, _QDIM[qkind])
        r = None if radii is None else _dev(radii, torch.float32).reshape(-1)
        lv, iv = ctypes.c_uint64(), ctypes.c_uint64()
        _check(self._lib.lbvh_tree_walk_visits(self._h, _ptr(q), q.shape[0], qkind, _ptr(r), float(radius),
                                               ctypes.byref(lv), ctypes.byref(iv), _stream(stream)),
               "lbvh_tree_walk_visits")
        return lv.value, iv.value

    def knn(self, queries, k: int, stream=None, distances: bool = True):
        """lbvh_knn: the k nearest primitives of each query point; returns
        (idx int32[nq, k] view of uint32, d2 float32[nq, k] or None), rows in
        the order (squared distance, index), padded with 0xffffffff / +inf."""
        torch = _torch()
        q = _dev(queries, torch.float32, 3)
        nq = q.shape[0]
        idx = torch.empty((nq, k), dtype=torch.int32, device=q.device)
        d2 = torch.empty((nq, k), dtype=torch.float32, device=q.device) if distances else None
        _check(self._lib.lbvh_knn(self._h, _ptr(q), nq, int(k), _ptr(idx), _ptr(d2) if d2 is not None else None,
                                  _stream(stream)), "lbvh_knn")
        return idx, d2

    def query(self, queries, qkind: int = SPHERE, radius: float = 0.0, radii=None, capacity=None,
              stream=None):
        """Stackless range query (Algorithm 1): returns CSR (offsets int64[nq+1], hits int32 view of uint32)."""
        torch = _torch()
        q = _dev(queries, torch.float32, _QDIM[qkind])
        nq = q.shape[0]
        offsets = torch.empty(nq + 1, dtype=torch.int64, device="cuda")
        cap = int(capacity) if capacity is not None else max(16 * nq, 1)
        hits = torch.empty(cap, dtype=torch.int32, device="cuda")
        st, total = self.query_into(q, qkind, offsets, hits, radius, radii, stream)
        if st == ERR_CAPACITY:
            hits = torch.empty(max(total, 1), dtype=torch.int32, device="cuda")
            st, total = self.query_into(q, qkind, offsets, hits, radius, radii, stream)
        _check(st, "lbvh_query_into")
        return offsets, hits[:total]


class Batch:
    """Many independent trees built and queried in one pass (``lbvh_batch_*``).

    Pass the same tensors on every call to replay the recorded CUDA graph.
    """

    def __init__(self):
        self._lib = load()
        h = ctypes.c_void_p()
        _check(self._lib.lbvh_batch_create(ctypes.byref(h)), "lbvh_batch_create")
        self._h = h
        self._keep = None
        self._out = None
        self.kind = POINTS
        self.count = 0

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._lib.lbvh_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def build_query(self, prims, prim_offsets, kind: int = POINTS, morton_bits: int = 30, queries=None,
                    query_offsets=None, qkind: int = SPHERE, radius: float = 0.0, radii=None,
                    offsets=None, hits=None, capacity=None, stream=None):
        """Returns (offsets int64[nq+1], hits int32 view of uint32 local ids, total, status)."""
        torch = _torch()
        p = prims if isinstance(prims, torch.Tensor) and prims.is_cuda else _dev(prims, torch.float32)
        q = p if queries is None else (queries if isinstance(queries, torch.Tensor) and queries.is_cuda
                                       else _dev(queries, torch.float32))
        po = np.ascontiguousarray(prim_offsets, dtype=np.int64)
        qo = po if query_offsets is None else np.ascontiguousarray(query_offsets, dtype=np.int64)
        count = po.size - 1
        nq = int(qo[-1])
        r = None
        if radii is not None:
            r = radii if isinstance(radii, torch.Tensor) and radii.is_cuda else _dev(radii, torch.float32).reshape(-1)
        if offsets is None:
            if self._out is None or self._out[0].numel() != nq + 1:
                self._out = (torch.empty(nq + 1, dtype=torch.int64, device="cuda"), None)
            offsets = self._out[0]
        if hits is None:
            cap = int(capacity) if capacity is not None else max(20 * nq, 1)
            if self._out[1] is None or self._out[1].numel() != cap:
                self._out = (offsets, torch.empty(cap, dtype=torch.int32, device="cuda"))
            hits = self._out[1]
        total = ctypes.c_uint64()
        st = self._lib.lbvh_batch_build_query(
            self._h, _ptr(p), ctypes.c_void_p(po.ctypes.data), count, kind, morton_bits, _ptr(q),
            ctypes.c_void_p(qo.ctypes.data), qkind, _ptr(r), float(radius), _ptr(offsets), _ptr(hits),
            hits.numel(), ctypes.byref(total), _stream(stream))
        self._keep = (p, q, r)
        self.kind, self.count, self._po = kind, count, po
        return offsets, hits, total.value, st

    def export(self, instance: int) -> dict:
        n = int(self._po[instance + 1] - self._po[instance])
        ni = max(n - 1, 0)
        out = {
            "n": n,
            "perm": np.zeros(n, np.uint32), "sorted": np.zeros(n, np.uint64),
            "left": np.zeros(ni, np.int32), "skip_internal": np.zeros(ni, np.int32),
            "skip_leaf": np.zeros(n, np.int32), "internal_box": np.zeros((ni, 6), np.float32),
            "leaf_box": np.zeros((n, 6), np.float32), "bounds": np.zeros(6, np.float32),
        }
        a = [ctypes.c_void_p(out[k].ctypes.data) for k in
             ("perm", "sorted", "left", "skip_internal", "skip_leaf", "internal_box", "leaf_box", "bounds")]
        _check(self._lib.lbvh_batch_export(self._h, instance, *a), "lbvh_batch_export")
        return out

    def sort_variant(self) -> int:
        v = ctypes.c_int()
        _check(self._lib.lbvh_batch_sort_variant(self._h, ctypes.byref(v)), "lbvh_batch_sort_variant")
        return v.value


class _Request(ctypes.Structure):
    _fields_ = [("d_prims", ctypes.c_void_p), ("n", ctypes.c_int64), ("kind", ctypes.c_int),
                ("morton_bits", ctypes.c_int), ("d_queries", ctypes.c_void_p), ("nq", ctypes.c_int64),
                ("qkind", ctypes.c_int), ("radius", ctypes.c_float), ("d_radii", ctypes.c_void_p),
                ("d_offsets", ctypes.c_void_p), ("d_hits", ctypes.c_void_p), ("capacity", ctypes.c_uint64),
                ("key", ctypes.c_uint64)]


class _Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("total", ctypes.c_uint64), ("queued_s", ctypes.c_double),
                ("service_s", ctypes.c_double), ("latency_s", ctypes.c_double), ("batch_size", ctypes.c_int)]


class Server:
    """Request server (``lbvh_server_*``): build + query requests batched as
    they arrive, trees kept resident under an HBM byte budget."""

    def __init__(self, budget_bytes: int, slots: int = 2, max_batch: int = 64):
        self._lib = load()
        h = ctypes.c_void_p()
        _check(self._lib.lbvh_server_create(int(budget_bytes), slots, max_batch, ctypes.byref(h)),
               "lbvh_server_create")
        self._h = h
        self._live = {}

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._lib.lbvh_server_destroy(self._h)
            self._h = ctypes.c_void_p()
            self._live.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, prims=None, kind: int = POINTS, morton_bits: int = 30, queries=None, qkind: int = SPHERE,
               radius: float = 0.0, radii=None, capacity: int | None = None, key: int = 0) -> int:
        """Queue a request; ``prims=None`` queries the resident tree ``key``.
        ``queries=None`` queries the primitives themselves."""
        torch = _torch()
        p = None if prims is None else (prims if isinstance(prims, torch.Tensor) and prims.is_cuda
                                        else _dev(prims, torch.float32))
        q = p if queries is None else (queries if isinstance(queries, torch.Tensor) and queries.is_cuda
                                       else _dev(queries, torch.float32))
        if q is None:
            raise ValueError("a query-only request needs queries")
        n = 0 if p is None else p.numel() // (3 if kind == POINTS else 6)
        nq = q.numel() // _QDIM[qkind]
        r = None
        if radii is not None:
            r = radii if isinstance(radii, torch.Tensor) and radii.is_cuda else _dev(radii, torch.float32).reshape(-1)
        cap = int(capacity) if capacity is not None else max(32 * nq, 64)
        offsets = torch.empty(nq + 1, dtype=torch.int64, device="cuda")
        hits = torch.empty(max(cap, 1), dtype=torch.int32, device="cuda")
        req = _Request(_ptr(p), n, kind, morton_bits, _ptr(q), nq, qkind, float(radius), _ptr(r),
                       _ptr(offsets), _ptr(hits), cap, int(key))
        ticket = ctypes.c_uint64()
        torch.cuda.current_stream().synchronize()  # inputs written on the caller's stream are complete
        _check(self._lib.lbvh_server_submit(self._h, ctypes.byref(req), ctypes.byref(ticket)), "lbvh_server_submit")
        self._live[ticket.value] = (p, q, r, offsets, hits)
        return ticket.value

    def wait(self, ticket: int):
        """Block until done: (offsets, hits[:total], result dict)."""
        res = _Result()
        _check(self._lib.lbvh_server_wait(self._h, ticket, ctypes.byref(res)), "lbvh_server_wait")
        _, _, _, offsets, hits = self._live.pop(ticket)
        info = {"status": res.status, "total": res.total, "queued_s": res.queued_s,
                "service_s": res.service_s, "latency_s": res.latency_s, "batch_size": res.batch_size}
        return offsets, hits[:res.total] if res.status == OK else hits[:0], info

    def stats(self) -> dict:
        v = [ctypes.c_uint64() for _ in range(4)]
        _check(self._lib.lbvh_server_stats(self._h, *[ctypes.byref(x) for x in v]), "lbvh_server_stats")
        return dict(zip(("resident_bytes", "resident_trees", "evictions", "batches"), (x.value for x in v)))

    def latency(self) -> dict:
        """lbvh_server_latency: p50 / p99 (seconds) and count of answered requests."""
        p50, p99, cnt = ctypes.c_double(), ctypes.c_double(), ctypes.c_uint64()
        _check(self._lib.lbvh_server_latency(self._h, ctypes.byref(p50), ctypes.byref(p99), ctypes.byref(cnt)),
               "lbvh_server_latency")
        return {"p50_s": p50.value, "p99_s": p99.value, "count": cnt.value}

    def device_spans(self) -> np.ndarray:
        """lbvh_server_device_spans: float64[jobs, 3] rows (slot, begin s, end s)."""
        count = ctypes.c_uint64()
        _check(self._lib.lbvh_server_device_spans(self._h, None, 0, ctypes.byref(count)), "lbvh_server_device_spans")
        out = np.zeros((count.value, 3), np.float64)
        if count.value:
            _check(self._lib.lbvh_server_device_spans(self._h, ctypes.c_void_p(out.ctypes.data), count.value,
                                                      ctypes.byref(count)), "lbvh_server_device_spans")
        return out

    def phase_seconds(self) -> dict:
        """lbvh_server_phase_seconds: worker time per phase, summed over batches."""
        v = (ctypes.c_double * SERVER_PHASES)()
        _check(self._lib.lbvh_server_phase_seconds(self._h, v), "lbvh_server_phase_seconds")
        return dict(zip(("stage", "batch", "deliver", "query_only"), list(v)))


def morton_codes(prims, kind: int = POINTS, morton_bits: int = 30, stream=None):
    """lbvh_morton_codes: (codes as int64 tensor holding the uint64 bits, bounds float[6])."""
    lib = load()
    torch = _torch()
    p = _dev(prims, torch.float32, 3 if kind == POINTS else 6)
    n = p.shape[0]
    codes = torch.empty(n, dtype=torch.int64, device="cuda")
    bounds = torch.empty(6, dtype=torch.float32, device="cuda")
    _check(lib.lbvh_morton_codes(_ptr(p), n, kind, morton_bits, _ptr(codes), _ptr(bounds), _stream(stream)),
           "lbvh_morton_codes")
    return codes, bounds


def sort_pairs(keys, vals=None, key_bits: int = 64, stream=None):
    """lbvh_sort_pairs on int64-held uint64 keys; vals None = primitive index."""
    lib = load()
    torch = _torch()
    k = keys if isinstance(keys, torch.Tensor) else torch.as_tensor(np.asarray(keys, np.uint64).view(np.int64))
    k = k.to(device="cuda", dtype=torch.int64).contiguous()
    v = None
    if vals is not None:
        v = vals if isinstance(vals, torch.Tensor) else torch.as_tensor(np.asarray(vals, np.uint32).view(np.int32))
        v = v.to(device="cuda", dtype=torch.int32).contiguous()
    n = k.numel()
    ko = torch.empty_like(k)
    vo = torch.empty(n, dtype=torch.int32, device="cuda")
    _check(lib.lbvh_sort_pairs(_ptr(k), _ptr(v), n, key_bits, _ptr(ko), _ptr(vo), _stream(stream)),
           "lbvh_sort_pairs")
    return ko, vo


def sort_variant_count() -> int:
    return load().lbvh_sort_variant_count()


def walk_variant_count() -> int:
    return load().lbvh_walk_variant_count()


def tune_save(path: str) -> None:
    """lbvh_tune_save: the tuner's cache to a JSON file."""
    _check(load().lbvh_tune_save(os.fsencode(path)), "lbvh_tune_save")


def tune_load(path: str) -> None:
    """lbvh_tune_load: merge a saved cache file into the tuner's cache."""
    _check(load().lbvh_tune_load(os.fsencode(path)), "lbvh_tune_load")


def tune_clear() -> None:
    load().lbvh_tune_clear()


def tune_entries() -> int:
    return load().lbvh_tune_entries()


def release_cached_memory() -> None:
    """lbvh_release_cached_memory: hand the library pool's unused blocks back."""
    _check(load().lbvh_release_cached_memory(), "lbvh_release_cached_memory")


def kernel_launches() -> int:
    """Kernels launched by the library so far in this process."""
    return int(load().lbvh_kernel_launches())


def to_u64(t) -> np.ndarray:
    return t.cpu().numpy().view(np.uint64)


def to_u32(t) -> np.ndarray:
    return t.cpu().numpy().view(np.uint32)
