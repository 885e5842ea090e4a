"""CPU oracle for R-tree range select and join (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package.  The CUDA library never links or calls it.

The arithmetic lives in ``rtree_oracle.c`` (plain scalar C, compiled with
``-O2 -fno-fast-math -ffp-contract=off`` so float32 behaves as IEEE 754).
This module only compiles it and marshals NumPy arrays through ctypes.

Parity status: every function here is pinned by the non-GPU tests
(hand-written golden cases, closed forms, invariants, brute force on small
inputs and an independent plane-sweep join); none is "parity unpinned".
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rtree_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
CFLAGS = ["-O2", "-fno-fast-math", "-ffp-contract=off", "-fPIC", "-shared", "-std=c11", "-pthread"]

_lock = threading.Lock()
_lib = None


def build_oracle(src: str = _SRC, out: str = _LIB_PATH, force: bool = False) -> str:
    """Compile the oracle's C source into a shared library; returns its path."""
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(src):
        return out
    os.makedirs(os.path.dirname(out), exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    subprocess.run(["gcc", *CFLAGS, "-o", tmp, src, "-lm", "-lpthread"], check=True)
    os.replace(tmp, out)
    return out


def _bind(lib):
    i64, i32p, f32p, i64p = C.c_int64, C.POINTER(C.c_int32), C.POINTER(C.c_float), C.POINTER(C.c_int64)
    lib.orc_tree_build.restype = C.c_void_p
    lib.orc_tree_build.argtypes = [f32p, i32p, i64, C.c_int]
    lib.orc_tree_build2.restype = C.c_void_p
    lib.orc_tree_build2.argtypes = [f32p, i32p, i64, C.c_int, C.c_int]
    lib.orc_join_pruned.restype = i64
    lib.orc_join_pruned.argtypes = [C.c_void_p, C.c_void_p, C.POINTER(i32p), i64p]
    lib.orc_join_tests.restype = i64
    lib.orc_join_tests.argtypes = [C.c_void_p, C.c_void_p]
    lib.orc_o5_bounds.restype = C.c_int
    lib.orc_o5_bounds.argtypes = [f32p, C.c_int, f32p, C.c_int, i32p, i32p, i32p]
    lib.orc_tree_free.restype = None
    lib.orc_tree_free.argtypes = [C.c_void_p]
    lib.orc_tree_levels.restype = C.c_int
    lib.orc_tree_levels.argtypes = [C.c_void_p]
    lib.orc_tree_nodes.restype = i64
    lib.orc_tree_nodes.argtypes = [C.c_void_p]
    lib.orc_tree_export.restype = C.c_int
    lib.orc_tree_export.argtypes = [C.c_void_p, i64p, i32p, f32p, i32p]
    lib.orc_select.restype = i64
    lib.orc_select.argtypes = [C.c_void_p, f32p, i64, i64p, C.POINTER(i32p)]
    lib.orc_brute_select.restype = i64
    lib.orc_brute_select.argtypes = [f32p, i32p, i64, f32p, i64, i64p, C.POINTER(i32p)]
    lib.orc_join.restype = i64
    lib.orc_join.argtypes = [C.c_void_p, C.c_void_p, C.POINTER(i32p)]
    lib.orc_select_mt.restype = i64
    lib.orc_select_mt.argtypes = [C.c_void_p, f32p, i64, i64p, C.POINTER(i32p), C.c_int]
    lib.orc_join_mt.restype = i64
    lib.orc_join_mt.argtypes = [C.c_void_p, C.c_void_p, C.POINTER(i32p), C.c_int]
    lib.orc_brute_join.restype = i64
    lib.orc_brute_join.argtypes = [f32p, i32p, i64, f32p, i32p, i64, C.POINTER(i32p)]
    lib.orc_free.restype = None
    lib.orc_free.argtypes = [C.c_void_p]
    return lib


def load(path: str | None = None):
    """Load (building if needed) the oracle library.  ``path`` loads a variant."""
    global _lib
    if path is not None:
        return _bind(C.CDLL(path))
    with _lock:
        if _lib is None:
            _lib = _bind(C.CDLL(build_oracle()))
        return _lib


def _rects(a) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float32)
    if a.ndim != 2 or a.shape[1] != 4:
        a = a.reshape(-1, 4)
    return a


def _ids(a, n) -> np.ndarray:
    if a is None:
        return np.arange(n, dtype=np.int32)
    a = np.ascontiguousarray(a, dtype=np.int32)
    assert a.shape == (n,)
    return a


def _f(a):
    return a.ctypes.data_as(C.POINTER(C.c_float))


def _i(a):
    return a.ctypes.data_as(C.POINTER(C.c_int32))


def _l(a):
    return a.ctypes.data_as(C.POINTER(C.c_int64))


def _take_i32(lib, ptr, count) -> np.ndarray:
    if count == 0:
        out = np.empty(0, dtype=np.int32)
    else:
        out = np.ctypeslib.as_array(ptr, shape=(count,)).copy()
    lib.orc_free(C.cast(ptr, C.c_void_p))
    return out


class Tree:
    """Oracle R-tree: STR bulk load, recursive select, synchronized join.

    ``sort_children`` orders every node's entries by ascending lx (stable),
    as the join pruning of Section 4.2 assumes."""

    def __init__(self, rects, ids=None, fanout: int = 16, lib=None, sort_children: bool = False):
        self._lib = lib or load()
        self.rects = _rects(rects)
        self.n = self.rects.shape[0]
        self.ids = _ids(ids, self.n)
        self.fanout = int(fanout)
        self.sort_children = bool(sort_children)
        h = self._lib.orc_tree_build2(_f(self.rects), _i(self.ids), self.n, self.fanout,
                                      1 if self.sort_children else 0)
        if not h:
            raise MemoryError("oracle tree build failed")
        self._h = h

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.orc_tree_free(h)
            self._h = None

    @property
    def levels(self) -> int:
        return self._lib.orc_tree_levels(self._h)

    @property
    def n_nodes(self) -> int:
        return self._lib.orc_tree_nodes(self._h)

    def select(self, queries, threads: int = 1):
        """Returns (offsets int64[Q+1], ids int32[total]) with sorted segments.
        ``threads`` > 1 runs the same select on that many POSIX threads, each
        on a contiguous run of the queries (orc_select_mt)."""
        q = _rects(queries)
        off = np.zeros(q.shape[0] + 1, dtype=np.int64)
        ptr = C.POINTER(C.c_int32)()
        if threads > 1:
            total = self._lib.orc_select_mt(self._h, _f(q), q.shape[0], _l(off), C.byref(ptr), int(threads))
        else:
            total = self._lib.orc_select(self._h, _f(q), q.shape[0], _l(off), C.byref(ptr))
        if total < 0:
            raise MemoryError("oracle select failed")
        return off, _take_i32(self._lib, ptr, total)

    def join(self, other: "Tree", threads: int = 1) -> np.ndarray:
        """Returns int32[total, 2] (r_id, s_id) pairs, sorted lexicographically.
        ``threads`` > 1 splits the traversal's top-level node pairs over that
        many POSIX threads (orc_join_mt)."""
        ptr = C.POINTER(C.c_int32)()
        if threads > 1:
            total = self._lib.orc_join_mt(self._h, other._h, C.byref(ptr), int(threads))
        else:
            total = self._lib.orc_join(self._h, other._h, C.byref(ptr))
        if total < 0:
            raise MemoryError("oracle join failed")
        return _take_i32(self._lib, ptr, 2 * total).reshape(-1, 2)

    def join_pruned(self, other: "Tree"):
        """Join with the O3/O4 prunings (both trees built with sort_children).
        Returns (pairs int32[total, 2] sorted, predicate evaluations)."""
        ptr = C.POINTER(C.c_int32)()
        tests = C.c_int64()
        total = self._lib.orc_join_pruned(self._h, other._h, C.byref(ptr), C.byref(tests))
        if total < 0:
            raise ValueError("oracle pruned join needs two trees built with sort_children")
        return _take_i32(self._lib, ptr, 2 * total).reshape(-1, 2), tests.value

    def join_tests(self, other: "Tree") -> int:
        """Predicate evaluations of the plain synchronized join."""
        return self._lib.orc_join_tests(self._h, other._h)

    def export(self):
        """Level-major export, root level first (see orc_tree_export)."""
        L, M, F = self.levels, self.n_nodes, self.fanout
        level_nodes = np.zeros(L, dtype=np.int64)
        counts = np.zeros(M, dtype=np.int32)
        mbrs = np.zeros((M, F, 4), dtype=np.float32)
        leaf_ids = np.zeros(self.n, dtype=np.int32)
        if L:
            rc = self._lib.orc_tree_export(self._h, _l(level_nodes), _i(counts), _f(mbrs), _i(leaf_ids))
            if rc:
                raise MemoryError("oracle export failed")
        return {"level_nodes": level_nodes, "counts": counts, "mbrs": mbrs, "leaf_ids": leaf_ids}


def brute_select(rects, queries, ids=None, lib=None):
    lib = lib or load()
    r = _rects(rects)
    i = _ids(ids, r.shape[0])
    q = _rects(queries)
    off = np.zeros(q.shape[0] + 1, dtype=np.int64)
    ptr = C.POINTER(C.c_int32)()
    total = lib.orc_brute_select(_f(r), _i(i), r.shape[0], _f(q), q.shape[0], _l(off), C.byref(ptr))
    if total < 0:
        raise MemoryError("oracle brute select failed")
    return off, _take_i32(lib, ptr, total)


def brute_join(r_rects, s_rects, r_ids=None, s_ids=None, lib=None):
    lib = lib or load()
    r = _rects(r_rects)
    s = _rects(s_rects)
    ri = _ids(r_ids, r.shape[0])
    si = _ids(s_ids, s.shape[0])
    ptr = C.POINTER(C.c_int32)()
    total = lib.orc_brute_join(_f(r), _i(ri), r.shape[0], _f(s), _i(si), s.shape[0], C.byref(ptr))
    if total < 0:
        raise MemoryError("oracle brute join failed")
    return _take_i32(lib, ptr, 2 * total).reshape(-1, 2)


def o5_bounds(out_hx, in_lx, lib=None):
    """The O5 search of Section 4.2 (see orc_o5_bounds).  Returns (flip
    int32[n_out], gather indices int32[rounds, n_out], flip indices after
    each round int32[rounds, n_out] with -1 for undefined)."""
    lib = lib or load()
    o = np.ascontiguousarray(out_hx, dtype=np.float32)
    i = np.ascontiguousarray(in_lx, dtype=np.float32)
    n_out, n_in = o.shape[0], i.shape[0]
    rounds_max = 1
    while (1 << (rounds_max - 1)) < max(n_in, 1):
        rounds_max += 1
    flip = np.zeros(max(n_out, 1), np.int32)
    tg = np.zeros((rounds_max, max(n_out, 1)), np.int32)
    tf = np.zeros((rounds_max, max(n_out, 1)), np.int32)
    rounds = lib.orc_o5_bounds(_f(o), n_out, _f(i), n_in, _i(flip), _i(tg), _i(tf))
    if rounds < 0:
        raise MemoryError("oracle O5 failed")
    return flip[:n_out], tg[:rounds, :n_out], tf[:rounds, :n_out]
