"""ctypes binding of the R-tree CUDA library (``include/rtree.h``).

Argument marshalling only: every step of build, select and join runs in the
library's CUDA kernels.  Functions carry the C names (``rtree_build``,
``rtree_range_select``, ``rtree_join``, ...); :class:`RTree` and
:class:`Result` wrap them with ownership.  If ``librtree.so`` has not been
built this module raises; there is no CPU fallback.

Arrays may be NumPy arrays (host memory) or torch tensors (host or CUDA);
the library copies host inputs to the device itself.  Streams: ``None``
means torch's current CUDA stream (or the legacy default stream when torch
has no CUDA), an ``int`` is a raw ``cudaStream_t``, and a
``torch.cuda.Stream`` is used as is.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "librtree.so")

(RTREE_OK, RTREE_EINVAL, RTREE_ENOMEM, RTREE_ECUDA, RTREE_ETIMEOUT, RTREE_EOVERFLOW, RTREE_EINTERNAL,
 RTREE_EIO) = range(8)
STATUS_NAMES = {0: "RTREE_OK", 1: "RTREE_EINVAL", 2: "RTREE_ENOMEM", 3: "RTREE_ECUDA",
                4: "RTREE_ETIMEOUT", 5: "RTREE_EOVERFLOW", 6: "RTREE_EINTERNAL", 7: "RTREE_EIO"}
LAYOUTS = {"soa": 0, "aos": 1, "lohi": 2}
MAPPINGS = {"auto": 0, "warp_per_query": 1, "work_queue": 2}
PRUNES = {"auto": 0, "off": 1, "on": 2}
TRAVERSALS = {"auto": 0, "levels": 1, "queue": 2}
ORDERS = {"input": 0, "hilbert": 1}


class RTreeError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class rtree_config_t(C.Structure):
    _fields_ = [("fanout", C.c_int32), ("layout", C.c_int32), ("sort_children", C.c_int32),
                ("reserved", C.c_int32 * 5)]


class rtree_join_opts_t(C.Structure):
    _fields_ = [("prune", C.c_int32), ("traversal", C.c_int32), ("reserved", C.c_int32 * 6)]


class rtree_select_opts_t(C.Structure):
    _fields_ = [("unsorted", C.c_int32), ("mapping", C.c_int32), ("order", C.c_int32),
                ("reserved", C.c_int32 * 5)]


class rtree_server_config_t(C.Structure):
    _fields_ = [("workers", C.c_int32), ("max_batch_queries", C.c_int32),
                ("max_batch_ids", C.c_int64), ("mapping", C.c_int32), ("reserved", C.c_int32 * 5)]


class rtree_reply_t(C.Structure):
    _fields_ = [("kind", C.c_int32), ("reserved", C.c_int32), ("rows", C.c_int64),
                ("total", C.c_int64), ("offsets", C.POINTER(C.c_int64)),
                ("ids", C.POINTER(C.c_int32)), ("latency_us", C.c_double)]


class rtree_server_stats_t(C.Structure):
    _fields_ = [("completed", C.c_int64), ("batches", C.c_int64), ("batch_queries", C.c_int64),
                ("splits", C.c_int64), ("fallbacks", C.c_int64), ("pending", C.c_int64),
                ("p50_us", C.c_double), ("p99_us", C.c_double), ("max_us", C.c_double),
                ("elapsed_s", C.c_double)]


RTREE_REQ_SELECT, RTREE_REQ_PROBE_JOIN = 0, 1
RTREE_TUNE_INCLUDE_BUILD = 1
RTREE_TUNE_ORDERS = 2


class rtree_tune_result_t(C.Structure):
    _fields_ = [("fanout", C.c_int32), ("layout", C.c_int32), ("mapping", C.c_int32),
                ("order", C.c_int32), ("tried", C.c_int32), ("reserved", C.c_int32),
                ("ms", C.c_double), ("ms_all", C.c_double * 64),
                ("fanout_all", C.c_int32 * 64), ("layout_all", C.c_int32 * 64),
                ("mapping_all", C.c_int32 * 64), ("order_all", C.c_int32 * 64)]


class rtree_info_t(C.Structure):
    _fields_ = [("n", C.c_int64), ("nodes", C.c_int64), ("levels", C.c_int32),
                ("fanout", C.c_int32), ("layout", C.c_int32), ("device", C.c_int32),
                ("device_bytes", C.c_int64), ("root_mbr", C.c_float * 4),
                ("sort_children", C.c_int32), ("reserved", C.c_int32 * 3)]


# device-memory hook (rtree_allocator_t): alloc(bytes, stream, ctx) -> pointer,
# free(pointer, stream, ctx)
ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)


class rtree_allocator_t(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", C.c_void_p)]


class Allocator:
    """A device-memory hook for rtree_build: every device buffer the library
    allocates for the tree (the tree, the scratch of calls on it, their
    results) comes from ``alloc(nbytes, stream) -> int`` (0 on failure) and
    goes back through ``free(ptr, stream)``; ``stream`` is the raw
    cudaStream_t of the call (0 = legacy default stream).  The callbacks run
    on whichever host thread calls into the library, with the GIL taken.
    Keep the object alive as long as the tree and its results (RTree and
    Result objects hold a reference).  Counts calls and live bytes."""

    def __init__(self, alloc, free):
        self._alloc, self._free = alloc, free
        self.allocs = self.frees = 0
        self.live = {}

        def c_alloc(nbytes, stream, _ctx):
            try:
                p = int(self._alloc(int(nbytes), int(stream or 0)) or 0)
            except Exception:  # an exception must not cross into C
                p = 0
            if p:
                self.allocs += 1
                self.live[p] = int(nbytes)
            return p

        def c_free(ptr, stream, _ctx):
            try:
                if ptr:
                    self.frees += 1
                    self.live.pop(int(ptr), None)
                    self._free(int(ptr), int(stream or 0))
            except Exception:
                pass

        self._c_alloc, self._c_free = ALLOC_FN(c_alloc), FREE_FN(c_free)
        self.struct = rtree_allocator_t(self._c_alloc, self._c_free, None)


class TorchAllocator(Allocator):
    """Takes the library's device memory from PyTorch's caching allocator
    (torch.cuda.caching_allocator_alloc / caching_allocator_delete), on the
    stream of each call, so the library shares one pool with the tensors
    around it.  Each allocation is a call into Python: use the default pool
    (no allocator) where many small calls run concurrently with busy Python
    threads (e.g. a serving loop whose client spins on the GIL)."""

    def __init__(self):
        import torch

        def alloc(nbytes, stream):
            return torch.cuda.caching_allocator_alloc(max(1, nbytes), None, stream)

        def free(ptr, _stream):
            torch.cuda.caching_allocator_delete(ptr)

        super().__init__(alloc, free)


_lock = threading.Lock()
_lib = None


def _bind(lib):
    vp, i64, i32 = C.c_void_p, C.c_int64, C.c_int32
    sigs = {
        "rtree_build": (C.c_int, [vp, vp, i64, C.POINTER(rtree_config_t), vp, vp, C.POINTER(vp)]),
        "rtree_free": (None, [vp]),
        "rtree_free_async": (None, [vp, vp]),
        "rtree_get_info": (C.c_int, [vp, C.POINTER(rtree_info_t)]),
        "rtree_export": (C.c_int, [vp, vp, vp, vp, vp, vp]),
        "rtree_range_select": (C.c_int, [vp, vp, i64, C.POINTER(rtree_select_opts_t), vp, C.POINTER(vp)]),
        "rtree_join": (C.c_int, [vp, vp, vp, C.POINTER(vp)]),
        "rtree_join_ex": (C.c_int, [vp, vp, vp, vp, C.POINTER(vp)]),
        "rtree_join_stats": (C.c_int, [vp, vp, vp, vp, C.POINTER(C.c_int64)]),
        "rtree_save": (C.c_int, [vp, C.c_char_p, vp]),
        "rtree_range_select_host": (C.c_int, [vp, vp, C.c_int64, vp, vp, vp, vp, C.c_int64,
                                              C.POINTER(C.c_int64)]),
        "rtree_range_select_host_async": (C.c_int, [vp, vp, C.c_int64, vp, vp, vp, vp, C.c_int64,
                                                    C.POINTER(C.c_int64), C.POINTER(vp)]),
        "rtree_pending_wait": (C.c_int, [vp]),
        "rtree_load": (C.c_int, [C.c_char_p, C.c_int, vp, C.POINTER(vp)]),
        "rtree_range_select_stats": (C.c_int, [vp, vp, i64, vp, C.POINTER(C.c_int64)]),
        "rtree_range_select_noalloc": (C.c_int, [vp, vp, i64, vp, vp, i64, C.POINTER(C.c_int64), vp]),
        "rtree_result_total": (i64, [vp]),
        "rtree_result_rows": (i64, [vp]),
        "rtree_result_offsets": (vp, [vp]),
        "rtree_result_ids": (vp, [vp]),
        "rtree_result_copy_to_host": (C.c_int, [vp, vp, vp, vp]),
        "rtree_result_free": (None, [vp]),
        "rtree_result_free_async": (None, [vp, vp]),
        "rtree_result_wait": (C.c_int, [vp]),
        "rtree_last_error": (C.c_char_p, []),
        "rtree_version": (C.c_char_p, []),
        "rtree_debug_fail_alloc_after": (None, [C.c_longlong]),
        "rtree_debug_wq_wait": (None, [C.c_longlong, C.c_int]),
        "rtree_plan_create": (C.c_int, [vp, i64, i64, C.POINTER(rtree_select_opts_t), C.POINTER(vp)]),
        "rtree_plan_run": (C.c_int, [vp, vp, i64, vp, C.POINTER(C.c_int64)]),
        "rtree_plan_offsets": (vp, [vp]),
        "rtree_plan_ids": (vp, [vp]),
        "rtree_plan_free": (None, [vp]),
        "rtree_server_start": (C.c_int, [vp, C.POINTER(rtree_server_config_t), C.POINTER(vp)]),
        "rtree_server_submit": (C.c_int, [vp, vp, i64, C.c_int32, C.POINTER(C.c_uint64)]),
        "rtree_server_wait": (C.c_int, [vp, C.c_uint64, i64, C.POINTER(rtree_reply_t)]),
        "rtree_reply_free": (None, [C.POINTER(rtree_reply_t)]),
        "rtree_server_get_stats": (C.c_int, [vp, C.POINTER(rtree_server_stats_t)]),
        "rtree_server_reset_stats": (C.c_int, [vp]),
        "rtree_server_stop": (None, [vp]),
        "rtree_autotune": (C.c_int, [vp, vp, i64, vp, i64, vp, C.c_int32, C.c_int32, vp,
                                     C.POINTER(rtree_tune_result_t)]),
        "rtree_timing_enable": (None, [C.c_int]),
        "rtree_timing_reset": (None, []),
        "rtree_timing_get": (C.c_int, [C.c_int, C.POINTER(C.c_char_p), C.POINTER(C.c_longlong),
                                       C.POINTER(C.c_double)]),
        "rtree_launch_count": (C.c_longlong, []),
    }
    for name, (res, args) in sigs.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


def load_library(path: str | None = None):
    """Loads ``librtree.so``; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is not None and path is None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(
                f"CUDA library not built ({p} missing); run "
                "`python -c 'import __graft_entry__ as g; g.build()'`")
        lib = _bind(C.CDLL(p))
        if path is None:
            _lib = lib
        return lib


def _check(status: int, lib=None):
    if status != RTREE_OK:
        lib = lib or load_library()
        raise RTreeError(status, (lib.rtree_last_error() or b"").decode())


# ------------------------------------------------------------- marshalling
def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _as_rows(x, what: str):
    """Returns (pointer, rows, keepalive) for an [n, 4] float32 array."""
    if x is None:
        return None, 0, None
    if _is_torch(x):
        import torch
        if x.dtype != torch.float32:
            raise TypeError(f"{what} must be float32")
        x = x.reshape(-1, 4)
        if not x.is_contiguous():
            x = x.contiguous()
        return x.data_ptr() or None, x.shape[0], x
    a = np.ascontiguousarray(x, dtype=np.float32).reshape(-1, 4)
    return a.ctypes.data or None, a.shape[0], a


def _as_ids(x, n: int):
    if x is None:
        return None, None
    if _is_torch(x):
        import torch
        if x.dtype != torch.int32:
            raise TypeError("ids must be int32")
        x = x.reshape(-1).contiguous()
        if x.numel() != n:
            raise ValueError("ids must have one entry per rectangle")
        return x.data_ptr() or None, x
    a = np.ascontiguousarray(x, dtype=np.int32).reshape(-1)
    if a.size != n:
        raise ValueError("ids must have one entry per rectangle")
    return a.ctypes.data or None, a


def _stream(stream) -> int:
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available() and torch.cuda.is_initialized():
                return torch.cuda.current_stream().cuda_stream
        except Exception:
            pass
        return 0
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


# ------------------------------------------------- C names, thin wrappers
def rtree_build(rects, ids=None, fanout: int = 16, layout: str | int = "soa", stream=None,
                sort_children: bool = False, allocator: Allocator | None = None) -> int:
    """Builds a tree; returns the opaque handle (free with rtree_free).
    ``allocator`` (an :class:`Allocator`) supplies the tree's device memory;
    None selects the library's default pool."""
    lib = load_library()
    rp, n, keep_r = _as_rows(rects, "rects")
    ip, keep_i = _as_ids(ids, n)
    cfg = rtree_config_t()
    cfg.fanout = int(fanout)
    cfg.layout = LAYOUTS[layout] if isinstance(layout, str) else int(layout)
    cfg.sort_children = 1 if sort_children else 0
    out = C.c_void_p()
    ap = C.byref(allocator.struct) if allocator is not None else None
    _check(lib.rtree_build(rp, ip, n, C.byref(cfg), ap, _stream(stream), C.byref(out)), lib)
    del keep_r, keep_i
    return out.value


def rtree_save(handle: int, path: str, stream=None) -> None:
    """Writes the tree to ``path`` (atomically; see the C header)."""
    lib = load_library()
    _check(lib.rtree_save(handle, os.fsencode(path), _stream(stream)), lib)


def rtree_load(path: str, device: int = -1, stream=None) -> int:
    """Loads a tree saved by rtree_save; returns the handle."""
    lib = load_library()
    out = C.c_void_p()
    _check(lib.rtree_load(os.fsencode(path), int(device), _stream(stream), C.byref(out)), lib)
    return out.value


def rtree_free(handle: int, stream=None) -> None:
    """Frees a tree.  With ``stream`` the release is ordered on that stream
    (rtree_free_async) and does not wait for work on other streams."""
    if handle:
        if stream is None:
            load_library().rtree_free(handle)
        else:
            load_library().rtree_free_async(handle, _stream(stream))


def rtree_get_info(handle: int) -> dict:
    lib = load_library()
    info = rtree_info_t()
    _check(lib.rtree_get_info(handle, C.byref(info)), lib)
    return {"n": info.n, "nodes": info.nodes, "levels": info.levels, "fanout": info.fanout,
            "layout": info.layout, "device": info.device, "device_bytes": info.device_bytes,
            "root_mbr": np.array(info.root_mbr[:], dtype=np.float32),
            "sort_children": info.sort_children}


def rtree_export(handle: int, stream=None) -> dict:
    lib = load_library()
    info = rtree_get_info(handle)
    L, M, F, n = info["levels"], info["nodes"], info["fanout"], info["n"]
    level_nodes = np.zeros(L, np.int64)
    counts = np.zeros(M, np.int32)
    mbrs = np.zeros((M, F, 4), np.float32)
    leaf_ids = np.zeros(n, np.int32)
    if L:
        _check(lib.rtree_export(handle, level_nodes.ctypes.data, counts.ctypes.data,
                                mbrs.ctypes.data, leaf_ids.ctypes.data, _stream(stream)), lib)
    return {"level_nodes": level_nodes, "counts": counts, "mbrs": mbrs, "leaf_ids": leaf_ids}


def rtree_range_select(handle: int, queries, unsorted: bool = False, mapping: str | int = "auto",
                       stream=None, order: str | int = "input") -> int:
    """Runs a batched range select; returns the result handle."""
    lib = load_library()
    qp, q, keep = _as_rows(queries, "queries")
    opts = rtree_select_opts_t()
    opts.unsorted = 1 if unsorted else 0
    opts.mapping = MAPPINGS[mapping] if isinstance(mapping, str) else int(mapping)
    opts.order = ORDERS[order] if isinstance(order, str) else int(order)
    out = C.c_void_p()
    _check(lib.rtree_range_select(handle, qp, q, C.byref(opts), _stream(stream), C.byref(out)), lib)
    del keep
    return out.value


def _host_select_args(queries, offsets, ids, unsorted, mapping, order):
    qp, q, keep = _as_rows(queries, "queries")
    opts = rtree_select_opts_t()
    opts.unsorted = 1 if unsorted else 0
    opts.mapping = MAPPINGS[mapping] if isinstance(mapping, str) else int(mapping)
    opts.order = ORDERS[order] if isinstance(order, str) else int(order)

    def host_ptr(a, dtype, name):
        if _is_torch(a):
            assert not a.is_cuda and a.is_contiguous(), f"{name} must be a contiguous CPU tensor"
            return a.data_ptr(), a.numel()
        assert a.dtype == dtype and a.flags["C_CONTIGUOUS"], f"{name} must be contiguous {dtype}"
        return a.ctypes.data, a.size
    op, on = host_ptr(offsets, np.int64, "offsets")
    ip, cap = host_ptr(ids, np.int32, "ids")
    assert on >= q + 1, "offsets needs q+1 entries"
    return qp, q, keep, opts, op, ip, cap


def rtree_range_select_host(handle: int, queries, offsets, ids, unsorted: bool = False,
                            mapping: str | int = "auto", order: str | int = "input", stream=None) -> int:
    """Select into host arrays (NumPy or CPU tensors; pinned memory overlaps
    the copies with the work).  ``offsets`` int64[q+1], ``ids`` int32
    [capacity].  Returns the total; raises RTreeError (RTREE_EOVERFLOW) when
    ids is too small, after offsets have been written."""
    lib = load_library()
    qp, q, keep, opts, op, ip, cap = _host_select_args(queries, offsets, ids, unsorted, mapping, order)
    total = C.c_int64()
    rc = lib.rtree_range_select_host(handle, qp, q, C.byref(opts), _stream(stream), op, ip if cap else None,
                                     cap, C.byref(total))
    del keep
    _check(rc, lib)
    return total.value


class PendingSelect:
    """A host-result select in flight (rtree_range_select_host_async).
    ``total`` is known at once; ``wait()`` returns it once the offsets and
    ids are in host memory.  Every pending select must be waited for."""

    def __init__(self, handle, total, keep):
        self._h = handle
        self.total = total
        self._keep = keep  # inputs the enqueued copies may still read

    def wait(self) -> int:
        if self._h is not None:
            lib = load_library()
            h, self._h = self._h, None
            rc = lib.rtree_pending_wait(h)
            self._keep = None
            _check(rc, lib)
        return self.total

    def __del__(self):
        if getattr(self, "_h", None):
            try:
                self.wait()
            except Exception:
                pass


def rtree_range_select_host_async(handle: int, queries, offsets, ids, unsorted: bool = False,
                                  mapping: str | int = "auto", order: str | int = "input",
                                  stream=None) -> PendingSelect:
    """rtree_range_select_host that returns once its work and copies are
    enqueued; the result is in ``offsets``/``ids`` after ``wait()``.  The
    next call (or tree build) may be started meanwhile."""
    lib = load_library()
    qp, q, keep, opts, op, ip, cap = _host_select_args(queries, offsets, ids, unsorted, mapping, order)
    total = C.c_int64()
    pend = C.c_void_p()
    rc = lib.rtree_range_select_host_async(handle, qp, q, C.byref(opts), _stream(stream), op,
                                           ip if cap else None, cap, C.byref(total), C.byref(pend))
    _check(rc, lib)
    return PendingSelect(pend.value, total.value, (keep, queries, offsets, ids))


def rtree_range_select_noalloc(handle: int, queries, offsets, ids, stream=None) -> int:
    """Range select into caller-owned device tensors without any device
    allocation (for callers that cannot allocate while running; see the C
    header).  ``queries`` float32 [q, 4] (q <= 65536), ``offsets`` int64
    [q+1], ``ids`` int32 [capacity], all CUDA tensors.  Returns the total;
    raises RTreeError (RTREE_EOVERFLOW) when ids is too small, after
    offsets have been written.  Ids come in traversal order."""
    lib = load_library()
    qp, q, keep = _as_rows(queries, "queries")
    total = C.c_int64()
    rc = lib.rtree_range_select_noalloc(handle, qp, q, offsets.data_ptr(), ids.data_ptr(),
                                        ids.numel(), C.byref(total), _stream(stream))
    del keep
    _check(rc, lib)
    return total.value


def rtree_range_select_stats(handle: int, queries, stream=None) -> dict:
    """Traversal counters of one count pass (no output produced)."""
    lib = load_library()
    qp, q, keep = _as_rows(queries, "queries")
    st = (C.c_int64 * 8)()
    _check(lib.rtree_range_select_stats(handle, qp, q, _stream(stream), st), lib)
    del keep
    keys = ("queries", "nodes_visited", "leaves_visited", "whole_children", "ids", "ids_from_whole")
    return {k: int(st[i]) for i, k in enumerate(keys)}


def rtree_join(r_handle: int, s_handle: int, stream=None) -> int:
    lib = load_library()
    out = C.c_void_p()
    _check(lib.rtree_join(r_handle, s_handle, _stream(stream), C.byref(out)), lib)
    return out.value


def rtree_join_ex(r_handle: int, s_handle: int, prune: str | int = "auto", stream=None,
                  traversal: str | int = "auto") -> int:
    """rtree_join with the sorted-node prunings ("auto", "off" or "on") and the
    traversal schedule ("auto", "levels" or "queue")."""
    lib = load_library()
    opts = rtree_join_opts_t()
    opts.prune = PRUNES[prune] if isinstance(prune, str) else int(prune)
    opts.traversal = TRAVERSALS[traversal] if isinstance(traversal, str) else int(traversal)
    out = C.c_void_p()
    _check(lib.rtree_join_ex(r_handle, s_handle, C.byref(opts), _stream(stream), C.byref(out)), lib)
    return out.value


def rtree_join_stats(r_handle: int, s_handle: int, prune: str | int = "auto", stream=None) -> dict:
    """Traversal counters of one join (the pairs themselves are dropped)."""
    lib = load_library()
    opts = rtree_join_opts_t()
    opts.prune = PRUNES[prune] if isinstance(prune, str) else int(prune)
    st = (C.c_int64 * 8)()
    _check(lib.rtree_join_stats(r_handle, s_handle, C.byref(opts), _stream(stream), st), lib)
    keys = ("pairs_equal_internal", "pairs_r_descends", "pairs_s_descends", "pairs_leaf", "pairs_found")
    return {k: int(st[i]) for i, k in enumerate(keys)}


def rtree_result_total(res: int) -> int:
    return load_library().rtree_result_total(res)


def rtree_result_rows(res: int) -> int:
    return load_library().rtree_result_rows(res)


def rtree_result_offsets(res: int) -> int:
    return load_library().rtree_result_offsets(res) or 0


def rtree_result_ids(res: int) -> int:
    return load_library().rtree_result_ids(res) or 0


def rtree_result_copy_to_host(res: int, stream=None):
    """Returns (offsets int64[rows+1] or None, ids int32[...]) as NumPy arrays."""
    lib = load_library()
    total, rows = lib.rtree_result_total(res), lib.rtree_result_rows(res)
    is_join = not lib.rtree_result_offsets(res)
    offsets = None if is_join else np.zeros(rows + 1, np.int64)
    ids = np.zeros(2 * total if is_join else total, np.int32)
    _check(lib.rtree_result_copy_to_host(res, None if offsets is None else offsets.ctypes.data,
                                         ids.ctypes.data if ids.size else None, _stream(stream)), lib)
    return offsets, (ids.reshape(-1, 2) if is_join else ids)


def rtree_result_free(res: int) -> None:
    if res:
        load_library().rtree_result_free(res)


def rtree_result_wait(res: int) -> None:
    """Waits for the work producing the result; raises on a device-side error."""
    lib = load_library()
    _check(lib.rtree_result_wait(res), lib)


def rtree_last_error() -> str:
    return (load_library().rtree_last_error() or b"").decode()


def rtree_version() -> str:
    return load_library().rtree_version().decode()


def rtree_debug_fail_alloc_after(k: int) -> None:
    load_library().rtree_debug_fail_alloc_after(int(k))


def rtree_debug_wq_wait(cycles: int, hold: bool = True) -> None:
    load_library().rtree_debug_wq_wait(int(cycles), 1 if hold else 0)


def rtree_plan_create(handle: int, max_queries: int, max_ids: int, mapping: str | int = "auto") -> int:
    """Creates a graph-captured batched select plan (see the C header)."""
    lib = load_library()
    opts = rtree_select_opts_t()
    opts.mapping = MAPPINGS[mapping] if isinstance(mapping, str) else int(mapping)
    out = C.c_void_p()
    _check(lib.rtree_plan_create(handle, int(max_queries), int(max_ids), C.byref(opts), C.byref(out)), lib)
    return out.value


def rtree_plan_run(plan: int, queries, stream=None) -> int:
    """Runs one batch; returns the number of ids (results stay in the plan)."""
    lib = load_library()
    qp, q, keep = _as_rows(queries, "queries")
    total = C.c_int64()
    rc = lib.rtree_plan_run(plan, qp, q, _stream(stream), C.byref(total))
    del keep
    _check(rc, lib)
    return total.value


def rtree_plan_offsets(plan: int) -> int:
    return load_library().rtree_plan_offsets(plan) or 0


def rtree_plan_ids(plan: int) -> int:
    return load_library().rtree_plan_ids(plan) or 0


def rtree_plan_free(plan: int) -> None:
    if plan:
        load_library().rtree_plan_free(plan)


def rtree_server_start(handle: int, workers: int = 2, max_batch_queries: int = 16384,
                       max_batch_ids: int = 16 << 20, mapping: str | int = "auto") -> int:
    lib = load_library()
    cfg = rtree_server_config_t()
    cfg.workers, cfg.max_batch_queries, cfg.max_batch_ids = workers, max_batch_queries, max_batch_ids
    cfg.mapping = MAPPINGS[mapping] if isinstance(mapping, str) else int(mapping)
    out = C.c_void_p()
    _check(lib.rtree_server_start(handle, C.byref(cfg), C.byref(out)), lib)
    return out.value


def rtree_server_submit(server: int, rects, kind: int = RTREE_REQ_SELECT) -> int:
    lib = load_library()
    a = np.ascontiguousarray(rects, dtype=np.float32).reshape(-1, 4)
    t = C.c_uint64()
    _check(lib.rtree_server_submit(server, a.ctypes.data or None, a.shape[0], int(kind), C.byref(t)), lib)
    return t.value


def rtree_server_wait(server: int, ticket: int, timeout_us: int = -1):
    """Returns (offsets int64[rows+1], ids int32[total], latency_us)."""
    lib = load_library()
    r = rtree_reply_t()
    _check(lib.rtree_server_wait(server, int(ticket), int(timeout_us), C.byref(r)), lib)
    try:
        off = np.ctypeslib.as_array(r.offsets, shape=(r.rows + 1,)).copy()
        ids = np.ctypeslib.as_array(r.ids, shape=(r.total,)).copy() if r.total else np.zeros(0, np.int32)
        return off, ids, r.latency_us
    finally:
        lib.rtree_reply_free(C.byref(r))


def rtree_server_get_stats(server: int) -> dict:
    lib = load_library()
    st = rtree_server_stats_t()
    _check(lib.rtree_server_get_stats(server, C.byref(st)), lib)
    return {k: getattr(st, k) for k, _ in rtree_server_stats_t._fields_}


def rtree_server_reset_stats(server: int) -> None:
    lib = load_library()
    _check(lib.rtree_server_reset_stats(server), lib)


def rtree_server_stop(server: int) -> None:
    if server:
        load_library().rtree_server_stop(server)


def rtree_autotune(rects, queries, ids=None, fanouts=(16, 32, 64, 128), include_build: bool = True,
                   stream=None, orders: bool = False) -> dict:
    """Times every fanout x layout x mapping (x traversal order with
    ``orders``) on the given sample and returns the fastest configuration
    plus all times (see the C header)."""
    lib = load_library()
    rp, n, keep_r = _as_rows(rects, "rects")
    ip, keep_i = _as_ids(ids, n)
    qp, q, keep_q = _as_rows(queries, "queries")
    fo = (C.c_int32 * len(fanouts))(*fanouts)
    out = rtree_tune_result_t()
    _check(lib.rtree_autotune(rp, ip, n, qp, q, fo, len(fanouts),
                              (RTREE_TUNE_INCLUDE_BUILD if include_build else 0) |
                              (RTREE_TUNE_ORDERS if orders else 0), _stream(stream),
                              C.byref(out)), lib)
    del keep_r, keep_i, keep_q
    names = {v: k for k, v in MAPPINGS.items()}
    lays = {v: k for k, v in LAYOUTS.items()}
    ords = {v: k for k, v in ORDERS.items()}

    def key(f, l, m, o):
        return f"F{f}_{lays[l]}_{names[m]}" + ("_hilbert" if o else "")
    return {"fanout": out.fanout, "layout": lays[out.layout], "mapping": names[out.mapping],
            "order": ords[out.order], "ms": out.ms,
            "all": {key(out.fanout_all[i], out.layout_all[i], out.mapping_all[i], out.order_all[i]):
                    round(out.ms_all[i], 3) for i in range(out.tried)}}


def rtree_timing_enable(on: bool = True) -> None:
    load_library().rtree_timing_enable(1 if on else 0)


def rtree_timing_reset() -> None:
    load_library().rtree_timing_reset()


def rtree_timing_get() -> dict:
    """{kernel name: (launches, total device ms)} since the last reset."""
    lib = load_library()
    out, i = {}, 0
    name, launches, ms = C.c_char_p(), C.c_longlong(), C.c_double()
    while lib.rtree_timing_get(i, C.byref(name), C.byref(launches), C.byref(ms)):
        out[name.value.decode()] = (launches.value, ms.value)
        i += 1
    return out


def rtree_launch_count() -> int:
    return load_library().rtree_launch_count()


# ------------------------------------------------------------ convenience
class _DeviceArray:
    """Exposes a library-owned device array through __cuda_array_interface__."""

    def __init__(self, owner, ptr: int, shape: tuple, typestr: str):
        self._owner = owner
        self.__cuda_array_interface__ = {"shape": shape, "typestr": typestr,
                                         "data": (int(ptr), False), "version": 3, "strides": None}


class Result:
    """A select (CSR) or join (pairs) result resident on the device.  A select
    returns while its last kernels still run on the call's stream: ``total``
    is valid at once; the arrays once that stream has reached them
    (``wait()``, ``to_numpy()``, or work and tensors on the same stream)."""

    def __init__(self, handle: int, owner=None):
        self.handle = handle
        self._owner = owner  # keeps the tree's allocator alive until the result is freed

    def __del__(self):
        self.close()

    def close(self, stream=None):
        """Frees the result; with ``stream`` in that stream's order
        (rtree_result_free_async), without waiting for the device."""
        h, self.handle = getattr(self, "handle", None), None
        if h:
            if stream is None:
                rtree_result_free(h)
            else:
                load_library().rtree_result_free_async(h, _stream(stream))

    @property
    def total(self) -> int:
        return rtree_result_total(self.handle)

    @property
    def rows(self) -> int:
        return rtree_result_rows(self.handle)

    @property
    def is_join(self) -> bool:
        return rtree_result_offsets(self.handle) == 0

    def wait(self) -> "Result":
        """Waits for the device work that produces this result (raises
        RTreeError on a device-side error)."""
        rtree_result_wait(self.handle)
        return self

    def to_numpy(self, stream=None):
        """(offsets, ids) for select; (None, pairs[total, 2]) for join."""
        return rtree_result_copy_to_host(self.handle, stream)

    def offsets_tensor(self):
        """Zero-copy torch view of the offsets (keeps this result alive)."""
        import torch
        self.wait()
        ptr = rtree_result_offsets(self.handle)
        return torch.as_tensor(_DeviceArray(self, ptr, (self.rows + 1,), "<i8"), device="cuda")

    def ids_tensor(self):
        """Zero-copy torch view of the ids (select) or pairs (join)."""
        import torch
        self.wait()
        ptr = rtree_result_ids(self.handle)
        shape = (self.total, 2) if self.is_join else (self.total,)
        if self.total == 0:
            return torch.zeros(shape, dtype=torch.int32, device="cuda")
        return torch.as_tensor(_DeviceArray(self, ptr, shape, "<i4"), device="cuda")


class Plan:
    """A graph-captured batched select over one tree (keeps the tree alive)."""

    def __init__(self, tree: "RTree", max_queries: int, max_ids: int, mapping="auto"):
        self.tree = tree
        self.handle = None
        self.handle = rtree_plan_create(tree.handle, max_queries, max_ids, mapping)
        self.q = 0
        self.total = 0

    def __del__(self):
        self.close()

    def close(self):
        h, self.handle = getattr(self, "handle", None), None
        if h:
            rtree_plan_free(h)

    def run(self, queries, stream=None) -> int:
        self.q = int(queries.shape[0])
        self.total = rtree_plan_run(self.handle, queries, stream)
        return self.total

    def offsets_tensor(self):
        import torch
        ptr = rtree_plan_offsets(self.handle)
        return torch.as_tensor(_DeviceArray(self, ptr, (self.q + 1,), "<i8"), device="cuda")

    def ids_tensor(self):
        import torch
        if self.total == 0:
            return torch.zeros(0, dtype=torch.int32, device="cuda")
        ptr = rtree_plan_ids(self.handle)
        return torch.as_tensor(_DeviceArray(self, ptr, (self.total,), "<i4"), device="cuda")

    def to_numpy(self):
        return self.offsets_tensor().cpu().numpy(), self.ids_tensor().cpu().numpy()


class Server:
    """Continuous-batching request loop over a resident tree (keeps it alive)."""

    def __init__(self, tree: "RTree", workers: int = 2, max_batch_queries: int = 16384,
                 max_batch_ids: int = 16 << 20, mapping="auto"):
        self.tree = tree
        self.handle = None
        self.handle = rtree_server_start(tree.handle, workers, max_batch_queries, max_batch_ids, mapping)

    def submit(self, rects, kind: int = RTREE_REQ_SELECT) -> int:
        return rtree_server_submit(self.handle, rects, kind)

    def wait(self, ticket: int, timeout_us: int = -1):
        return rtree_server_wait(self.handle, ticket, timeout_us)

    def stats(self) -> dict:
        return rtree_server_get_stats(self.handle)

    def reset_stats(self) -> None:
        rtree_server_reset_stats(self.handle)

    def stop(self):
        h, self.handle = getattr(self, "handle", None), None
        if h:
            rtree_server_stop(h)

    def __del__(self):
        self.stop()


class RTree:
    """An R-tree on the GPU: build, range select, join."""

    def __init__(self, rects, ids=None, fanout: int = 16, layout: str | int = "soa", stream=None,
                 sort_children: bool = False, allocator: Allocator | None = None):
        self.handle = None
        self.allocator = allocator
        self.handle = rtree_build(rects, ids, fanout, layout, stream, sort_children, allocator)

    def __del__(self):
        self.close()

    def close(self, stream=None):
        """Frees the tree; with ``stream`` in that stream's order
        (rtree_free_async), without waiting for the device."""
        h, self.handle = getattr(self, "handle", None), None
        if h:
            rtree_free(h, stream)

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def info(self) -> dict:
        return rtree_get_info(self.handle)

    def save(self, path: str, stream=None) -> None:
        rtree_save(self.handle, path, stream)

    @classmethod
    def load(cls, path: str, device: int = -1, stream=None) -> "RTree":
        t = cls.__new__(cls)
        t.handle = None
        t.allocator = None
        t.handle = rtree_load(path, device, stream)
        return t

    def export(self, stream=None) -> dict:
        return rtree_export(self.handle, stream)

    def range_select(self, queries, unsorted: bool = False, mapping="auto", stream=None,
                     order="input") -> Result:
        return Result(rtree_range_select(self.handle, queries, unsorted, mapping, stream, order),
                      self.allocator)

    def select_stats(self, queries, stream=None) -> dict:
        return rtree_range_select_stats(self.handle, queries, stream)

    def join(self, other: "RTree", stream=None, prune: str | int | None = None,
             traversal: str | int | None = None) -> Result:
        if prune is None and traversal is None:
            return Result(rtree_join(self.handle, other.handle, stream), self.allocator)
        return Result(rtree_join_ex(self.handle, other.handle, prune or "auto", stream, traversal or "auto"),
                      self.allocator)

    def join_stats(self, other: "RTree", stream=None, prune: str | int = "auto") -> dict:
        return rtree_join_stats(self.handle, other.handle, prune, stream)
