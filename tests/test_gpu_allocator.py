"""The device-memory hook (rtree_allocator_t) and stream-ordered calls.

A tree built with an allocator takes every device buffer the library
allocates for it -- the tree, the scratch of each call on it and the
results -- from that allocator and gives each one back.  The test allocator
counts calls and live blocks and takes the memory from PyTorch's caching
allocator.  Results must equal the CPU oracle; after everything is freed no
block may remain live.
"""
import numpy as np
import pytest

import oracle
from gpu_util import gpu_ready
from paper_2309_16913_gb300 import datagen as dg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rt():
    return gpu_ready()


def test_every_buffer_comes_from_the_hook(rt):
    import torch
    w = dg.workload("scaled", n=200_000, q=4_000)
    j = dg.workload("join", n=100_000)
    t_orc = oracle.Tree(w.rects, w.ids, 32)
    want = t_orc.select(w.queries)
    want_join = oracle.Tree(j.rects, j.ids, 16).join(oracle.Tree(j.rects_s, j.ids_s, 16))
    A = rt.TorchAllocator()
    q = torch.from_numpy(w.queries).cuda()
    t = rt.RTree(torch.from_numpy(w.rects).cuda(), torch.from_numpy(w.ids).cuda(), fanout=32,
                 layout="aos", allocator=A)
    n_tree = A.allocs
    assert n_tree >= 4 and len(A.live) >= 4  # node entries, metadata, boxes, ids (+ nothing else left)
    tree_blocks = set(A.live)
    for kw in ({}, {"order": "hilbert"}, {"mapping": "work_queue"}, {"unsorted": True}):
        before = A.allocs
        res = t.range_select(q, **kw)
        assert A.allocs - before >= 5, kw  # scratch and outputs of the call
        lib = rt.load_library()
        assert lib.rtree_result_offsets(res.handle) in A.live and lib.rtree_result_ids(res.handle) in A.live
        off, ids = res.to_numpy()
        res.close()
        if kw.get("unsorted"):
            ids = np.concatenate([np.sort(ids[off[i]:off[i + 1]]) for i in range(len(off) - 1)])
        assert np.array_equal(off, want[0]) and np.array_equal(ids, want[1]), kw
        assert set(A.live) == tree_blocks, kw  # scratch and results all given back
    st = t.select_stats(q)
    assert st["ids"] == int(want[0][-1])
    # host-result select, in flight while the next call starts
    h_off = torch.zeros(q.shape[0] + 1, dtype=torch.int64).pin_memory()
    h_ids = torch.zeros(int(want[0][-1]), dtype=torch.int32).pin_memory()
    p = rt.rtree_range_select_host_async(t.handle, q, h_off, h_ids)
    assert p.wait() == int(want[0][-1])
    assert np.array_equal(h_off.numpy(), want[0]) and np.array_equal(h_ids.numpy(), want[1])
    # graph-captured plan: its buffers from the hook
    before = A.allocs
    plan = rt.Plan(t, q.shape[0], int(want[0][-1]) + 100)
    assert A.allocs > before
    plan.run(q)
    po, pi = plan.to_numpy()
    plan.close()
    assert np.array_equal(po, want[0]) and np.array_equal(pi, want[1])
    # join: the result comes from the first tree's allocator
    B = rt.TorchAllocator()
    a = rt.RTree(torch.from_numpy(j.rects).cuda(), None, fanout=16, allocator=A)
    b = rt.RTree(torch.from_numpy(j.rects_s).cuda(), None, fanout=16, allocator=B)
    before = A.allocs
    res = a.join(b)
    assert A.allocs > before
    _, pairs = res.to_numpy()
    res.close()
    assert np.array_equal(pairs, want_join)
    a.close()
    b.close()
    t.close()
    torch.cuda.synchronize()
    assert not A.live and not B.live
    assert A.allocs == A.frees and B.allocs == B.frees


def test_allocator_failure_is_enomem_and_leaks_nothing(rt):
    import torch
    w = dg.workload("plain", n=50_000, q=500)
    want = oracle.Tree(w.rects, w.ids, 16).select(w.queries)
    budget = {"left": 10**9}
    inner = rt.TorchAllocator()

    def alloc(nbytes, stream):
        if budget["left"] <= 0:
            return 0
        budget["left"] -= 1
        return inner._alloc(nbytes, stream)

    A = rt.Allocator(alloc, inner._free)
    q = torch.from_numpy(w.queries).cuda()
    budget["left"] = 0
    with pytest.raises(rt.RTreeError) as e:
        rt.RTree(torch.from_numpy(w.rects).cuda(), None, fanout=16, allocator=A)
    assert e.value.status == rt.RTREE_ENOMEM
    assert not A.live
    budget["left"] = 10**9
    t = rt.RTree(torch.from_numpy(w.rects).cuda(), None, fanout=16, allocator=A)
    tree_blocks = set(A.live)
    for k in (0, 3, 7):  # the k-th allocation of the select fails
        budget["left"] = k
        with pytest.raises(rt.RTreeError) as e:
            t.range_select(q).close()
        assert e.value.status == rt.RTREE_ENOMEM
        torch.cuda.synchronize()
        assert set(A.live) == tree_blocks, k
    budget["left"] = 10**9
    res = t.range_select(q)
    off, ids = res.to_numpy()
    res.close()
    assert np.array_equal(off, want[0]) and np.array_equal(ids, want[1])
    t.close()
    assert not A.live


def test_select_is_stream_ordered(rt):
    """The select returns with its total while its sort still runs on the
    call's stream; work queued behind it on that stream sees the result."""
    import torch
    w = dg.workload("scaled", n=500_000, q=50_000)
    want = oracle.Tree(w.rects, w.ids, 64).select(w.queries)
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        rects = torch.from_numpy(w.rects).cuda()
        q = torch.from_numpy(w.queries).cuda()
        t = rt.RTree(rects, None, fanout=64, layout="aos", stream=side)
        res = t.range_select(q, stream=side, order="hilbert")
        assert res.total == int(want[0][-1])  # valid on return
        ids = res.ids_tensor().clone()        # queued on `side` behind the select
        off = res.offsets_tensor().clone()
    side.synchronize()
    assert np.array_equal(off.cpu().numpy(), want[0]) and np.array_equal(ids.cpu().numpy(), want[1])
    res.close()
    t.close()
