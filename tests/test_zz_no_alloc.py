"""The non-allocating range select, checked against the CPU oracle and the
regular entry point.

rtree_range_select_noalloc exists for callers that cannot allocate device
memory while running (an application that keeps all GPU memory in its own
pool, or a request loop that must not block in or fail from the CUDA
allocator).  It writes into caller-owned buffers and keeps its temporary
storage in a fixed device array inside the library.  This file is collected
last so that a failure here comes after every other test has run.
"""
import ctypes as C

import numpy as np
import pytest

import oracle
from gpu_util import gpu_ready
from paper_2309_16913_gb300 import datagen as dg

pytestmark = pytest.mark.gpu


def _call(lib, handle, q, off, out, stream):
    total = C.c_int64(-1)
    rc = lib.rtree_range_select_noalloc(handle, q.data_ptr(), q.shape[0], off.data_ptr(),
                                        out.data_ptr(), out.numel(), C.byref(total), stream)
    return rc, total.value


def test_noalloc_matches_oracle_and_range_select_on_two_calls():
    import torch
    rt = gpu_ready()
    lib = rt.load_library()
    stream = torch.cuda.current_stream().cuda_stream
    w = dg.workload("scaled", n=300_000, q=20_000)
    a, b = w.queries[:12_000], w.queries[12_000:]
    t_orc = oracle.Tree(w.rects, w.ids, 16)
    with rt.RTree(torch.from_numpy(w.rects).cuda(), torch.from_numpy(w.ids).cuda(), fanout=16) as t:
        for qs in (a, b):  # two calls in a row share the library's fixed scratch
            qd = torch.from_numpy(np.ascontiguousarray(qs)).cuda()
            res = t.range_select(qd, unsorted=True)
            want_off, want_ids = res.to_numpy()
            res.close()
            o_off, o_ids = t_orc.select(qs)
            off = torch.full((qd.shape[0] + 1,), -7, dtype=torch.int64, device="cuda")
            out = torch.full((int(want_off[-1]) + 100,), -7, dtype=torch.int32, device="cuda")
            torch.cuda.synchronize()
            # any device allocation inside the call would now fail with RTREE_ENOMEM
            lib.rtree_debug_fail_alloc_after(0)
            try:
                rc, total = _call(lib, t.handle, qd, off, out, stream)
            finally:
                lib.rtree_debug_fail_alloc_after(-1)
            assert rc == rt.RTREE_OK, rt.rtree_last_error()
            assert total == want_off[-1] == o_off[-1]
            got_off = off.cpu().numpy()
            assert np.array_equal(got_off, want_off) and np.array_equal(got_off, o_off)
            got = out[:total].cpu().numpy()
            assert np.array_equal(got, want_ids)
            # traversal order within a query; sorted, each query equals the oracle's list
            for i in range(qs.shape[0]):
                seg = np.sort(got[got_off[i]:got_off[i + 1]])
                assert np.array_equal(seg, o_ids[o_off[i]:o_off[i + 1]]), f"query {i}"
            assert bool((out[total:] == -7).all())


def test_noalloc_limits_and_short_buffer():
    import torch
    rt = gpu_ready()
    lib = rt.load_library()
    stream = torch.cuda.current_stream().cuda_stream
    w = dg.workload("plain", n=50_000, q=70_000)
    with rt.RTree(torch.from_numpy(w.rects).cuda(), None, fanout=16) as t:
        qd = torch.from_numpy(w.queries).cuda()
        off = torch.zeros(qd.shape[0] + 1, dtype=torch.int64, device="cuda")
        out = torch.zeros(16, dtype=torch.int32, device="cuda")
        rc, _ = _call(lib, t.handle, qd, off, out, stream)   # 70k > 65536 queries
        assert rc == rt.RTREE_EOVERFLOW and "65536" in rt.rtree_last_error()
        q2 = qd[:4000]
        rc, total = _call(lib, t.handle, q2, off, out, stream)  # ids buffer too short
        assert rc == rt.RTREE_EOVERFLOW and total > 16
        res = t.range_select(q2, unsorted=True)
        want_off, _ = res.to_numpy()
        res.close()
        assert np.array_equal(off[:4001].cpu().numpy(), want_off)
        host_q = np.ascontiguousarray(w.queries[:10])
        total = C.c_int64()
        rc = lib.rtree_range_select_noalloc(t.handle, host_q.ctypes.data, 10, off.data_ptr(),
                                            out.data_ptr(), out.numel(), C.byref(total), stream)
        assert rc == rt.RTREE_EINVAL  # host queries would need a staging copy
