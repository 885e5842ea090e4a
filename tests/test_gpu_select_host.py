"""rtree_range_select_host: the same CSR result as the oracle, delivered to
host memory chunk by chunk while later chunks are still being selected."""
import numpy as np
import pytest

import oracle
from gpu_util import gpu_ready, assert_csr_equal
from paper_2309_16913_gb300 import datagen as dg
from test_oracle import random_case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rt():
    return gpu_ready()


def host_select(rt, t, q, cap=None, pinned=False, **kw):
    import torch
    n = q.shape[0]
    if pinned:
        off = torch.zeros(n + 1, dtype=torch.int64).pin_memory()
        ids = torch.full((cap,), -7, dtype=torch.int32).pin_memory()
    else:
        off = np.zeros(n + 1, np.int64)
        ids = np.full(cap, -7, np.int32)
    total = rt.rtree_range_select_host(t.handle, q, off, ids, **kw)
    if pinned:
        off, ids = off.numpy(), ids.numpy()
    return off, ids[:total], total


@pytest.mark.parametrize("order", ["input", "hilbert"])
@pytest.mark.parametrize("mapping", ["warp_per_query", "work_queue"])
def test_host_select_matches_oracle(rt, mapping, order):
    w = dg.workload("scaled", n=300_000, q=20_000)
    want = oracle.Tree(w.rects, w.ids, 64).select(w.queries)
    with rt.RTree(w.rects, w.ids, fanout=64, layout="aos") as t:
        off, ids, total = host_select(rt, t, w.queries, cap=int(want[0][-1]) + 5, pinned=True,
                                      mapping=mapping, order=order)
    assert total == want[0][-1]
    assert_csr_equal((off, ids), want, f"{mapping} {order}")


def test_host_select_long_segments_and_pageable_buffers(rt):
    w = dg.workload("uneven", n=400_000, q=6000)
    want = oracle.Tree(w.rects, w.ids, 16).select(w.queries)
    assert np.diff(want[0]).max() > 16384  # long segments go through the MSD path
    with rt.RTree(w.rects, w.ids, fanout=16) as t:
        off, ids, _ = host_select(rt, t, w.queries, cap=int(want[0][-1]))
    assert_csr_equal((off, ids), want, "uneven")


def test_host_select_unsorted_sets(rt):
    w = dg.workload("plain", n=50_000, q=3000)
    wo, wi = oracle.brute_select(w.rects, w.queries, w.ids)
    with rt.RTree(w.rects, w.ids, fanout=16) as t:
        off, ids, _ = host_select(rt, t, w.queries, cap=int(wo[-1]), unsorted=True)
    assert np.array_equal(off, wo)
    for k in range(len(wo) - 1):
        assert np.array_equal(np.sort(ids[off[k]:off[k + 1]]), wi[wo[k]:wo[k + 1]]), k


def test_host_select_small_batches_and_empty(rt):
    rects = random_case("uniform", 5000, 2)
    q = random_case("uniform", 7, 3) * np.float32(1.0)
    q[:, 2:] += np.float32(0.2)
    with rt.RTree(rects, None, fanout=8) as t:
        for n in (1, 3, 7):
            want = oracle.brute_select(rects, q[:n])
            off, ids, _ = host_select(rt, t, q[:n], cap=int(want[0][-1]) + 1)
            assert_csr_equal((off, ids), want, f"q={n}")
        off, ids, total = host_select(rt, t, np.zeros((0, 4), np.float32), cap=0)
        assert total == 0 and off.tolist() == [0]
    with rt.RTree(np.zeros((0, 4), np.float32), None, fanout=8) as e:
        off, ids, total = host_select(rt, e, q, cap=0)
        assert total == 0 and off.tolist() == [0] * 8


def test_host_select_overflow_reports_total(rt):
    w = dg.workload("plain", n=20_000, q=500)
    want = oracle.brute_select(w.rects, w.queries, w.ids)
    need = int(want[0][-1])
    with rt.RTree(w.rects, w.ids, fanout=16) as t:
        off = np.zeros(501, np.int64)
        ids = np.full(need - 1, -7, np.int32)
        with pytest.raises(rt.RTreeError) as e:
            rt.rtree_range_select_host(t.handle, w.queries, off, ids)
        assert e.value.status == rt.RTREE_EOVERFLOW and str(need) in str(e.value)
        assert np.array_equal(off, want[0])      # offsets are written
        assert np.all(ids == -7)                 # ids untouched


def test_async_selects_in_flight_together(rt):
    """Two host-result selects in flight at once (the second enqueued before
    the first is waited for, the tree freed stream-ordered in between), waited
    for in reverse order: both match the oracle."""
    import torch
    w = dg.workload("scaled", n=300_000, q=20_000)
    qa, qb = w.queries[:12_000], w.queries[12_000:]
    orc = oracle.Tree(w.rects, w.ids, 64)
    want_a, want_b = orc.select(qa), orc.select(qb)
    stream = torch.cuda.current_stream()
    bufs = []
    for want, n in ((want_a, qa.shape[0]), (want_b, qb.shape[0])):
        bufs.append((torch.zeros(n + 1, dtype=torch.int64).pin_memory(),
                     torch.full((int(want[0][-1]) + 3,), -7, dtype=torch.int32).pin_memory()))
    h = rt.rtree_build(w.rects, w.ids, 64, "aos", stream)
    pa = rt.rtree_range_select_host_async(h, qa, bufs[0][0], bufs[0][1], order="hilbert", stream=stream)
    pb = rt.rtree_range_select_host_async(h, qb, bufs[1][0], bufs[1][1], stream=stream)
    rt.rtree_free(h, stream=stream)
    assert pa.total == want_a[0][-1] and pb.total == want_b[0][-1]
    assert pb.wait() == want_b[0][-1]
    assert pa.wait() == want_a[0][-1]
    for (off, ids), want, name in ((bufs[0], want_a, "a"), (bufs[1], want_b, "b")):
        total = int(want[0][-1])
        assert_csr_equal((off.numpy(), ids.numpy()[:total]), want, name)
        assert np.all(ids.numpy()[total:] == -7)


def test_async_overflow_and_empty(rt):
    w = dg.workload("plain", n=20_000, q=500)
    want = oracle.brute_select(w.rects, w.queries, w.ids)
    need = int(want[0][-1])
    with rt.RTree(w.rects, w.ids, fanout=16) as t:
        off = np.zeros(501, np.int64)
        ids = np.full(need - 1, -7, np.int32)
        with pytest.raises(rt.RTreeError) as e:
            rt.rtree_range_select_host_async(t.handle, w.queries, off, ids)
        assert e.value.status == rt.RTREE_EOVERFLOW
        assert np.array_equal(off, want[0]) and np.all(ids == -7)
        far = np.array([[5, 5, 6, 6], [7, 7, 8, 8]], np.float32)   # nothing there
        off2 = np.full(3, -1, np.int64)
        p = rt.rtree_range_select_host_async(t.handle, far, off2, np.zeros(0, np.int32))
        assert p.total == 0 and p.wait() == 0 and off2.tolist() == [0, 0, 0]
        p = rt.rtree_range_select_host_async(t.handle, np.zeros((0, 4), np.float32), off2[:1],
                                             np.zeros(0, np.int32))
        assert p.wait() == 0 and off2[0] == 0


def test_build_reports_invalid_rectangles(rt):
    """The build's validation outcome (read with the root box at the end of
    the build) still rejects NaN and inverted rows, and reports the root."""
    rects = random_case("uniform", 3000, 4)
    with rt.RTree(rects, None, fanout=16) as t:
        root = t.info()["root_mbr"]
        assert np.array_equal(root, np.array([rects[:, 0].min(), rects[:, 1].min(),
                                              rects[:, 2].max(), rects[:, 3].max()], np.float32))
    for bad_row in (np.float32([np.nan, 0, 1, 1]), np.float32([0.5, 0, 0.4, 1]),
                    np.float32([0, 0.5, 1, 0.4])):
        r = rects.copy()
        r[1234] = bad_row
        with pytest.raises(rt.RTreeError) as e:
            rt.RTree(r, None, fanout=16)
        assert e.value.status == rt.RTREE_EINVAL and "1234" in str(e.value)
