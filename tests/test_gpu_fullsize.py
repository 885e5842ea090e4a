"""Full-size parity at the benchmark's workloads, in the benchmark's launch
configuration (the same C ABI calls bench.py times).

At 10M rectangles every one of the million queries is compared exactly with
the oracle, whose select runs on all host cores (orc_select_mt), in chunks
of 65536 queries: at the configurations the benchmark's autotuner picks
(F=128 LOHI and F=64 AoS, Hilbert order) and at F=16 SoA in input order; the uneven mix (100k queries, 1%
heavy) is compared in full too.  The remaining fanout/layout pairs are
checked for properties that hold at any size (a valid CSR, strictly
ascending id lists within the id range) and on a seeded sample.  The
2M x 2M join is compared in full, plain and with the sorted-node prunings.
"""
import os

import numpy as np
import pytest

import oracle
from gpu_util import gpu_ready
from paper_2309_16913_gb300 import datagen as dg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rt():
    return gpu_ready()


def check_sample(rt, t_gpu, t_orc, queries, sample, F):
    import torch
    q = torch.from_numpy(queries).cuda()
    res = t_gpu.range_select(q)
    try:
        off = res.offsets_tensor().cpu().numpy()
        ids_dev = res.ids_tensor()
        assert off[0] == 0 and np.all(np.diff(off) >= 0) and off[-1] == res.total
        # strictly ascending inside every segment (ids are unique here)
        d = ids_dev[1:] - ids_dev[:-1]
        bounds = torch.from_numpy(off[1:-1]).cuda()
        ok = d > 0
        if bounds.numel():
            ok[(bounds - 1)[(bounds > 0) & (bounds < res.total)]] = True
        assert bool(ok.all()), "segment not strictly ascending"
        assert int(ids_dev.min()) >= 0 and int(ids_dev.max()) < t_gpu.info()["n"]
        o_off, o_ids = t_orc.select(queries[sample])
        for k, qi in enumerate(sample):
            got = ids_dev[off[qi]:off[qi + 1]].cpu().numpy()
            assert np.array_equal(got, o_ids[o_off[k]:o_off[k + 1]]), f"query {qi} F={F}"
        return int(off[-1])
    finally:
        res.close()


THREADS = os.cpu_count() or 1
CHUNK = 65536


def compare_all(t_gpu, t_orc, queries, context, **select_kw):
    """Every query of the batch equal to the oracle (chunked)."""
    import torch
    q = torch.from_numpy(queries).cuda()
    res = t_gpu.range_select(q, **select_kw)
    try:
        off = res.offsets_tensor().cpu().numpy()
        ids_dev = res.ids_tensor()
        Q = queries.shape[0]
        for c0 in range(0, Q, CHUNK):
            c1 = min(Q, c0 + CHUNK)
            o_off, o_ids = t_orc.select(queries[c0:c1], threads=THREADS)
            g_off = off[c0:c1 + 1] - off[c0]
            if not np.array_equal(g_off, o_off):
                bad = c0 + int(np.nonzero(np.diff(g_off) != np.diff(o_off))[0][0])
                raise AssertionError(f"{context}: count of query {bad} differs")
            got = ids_dev[off[c0]:off[c1]].cpu().numpy()
            if not np.array_equal(got, o_ids):
                k = int(np.nonzero(got != o_ids)[0][0])
                qi = c0 + int(np.searchsorted(o_off, k, side="right") - 1)
                raise AssertionError(f"{context}: ids of query {qi} differ")
        return int(off[-1])
    finally:
        res.close()


@pytest.mark.parametrize("F,layout,order", [(128, "lohi", "hilbert"), (64, "aos", "hilbert"), (16, "soa", "input")])
def test_scaled_10m_every_query_exact(rt, F, layout, order):
    import torch
    w = dg.workload("scaled")
    t_orc = oracle.Tree(w.rects, w.ids, F)
    with rt.RTree(torch.from_numpy(w.rects).cuda(), torch.from_numpy(w.ids).cuda(),
                  fanout=F, layout=layout) as t:
        total = compare_all(t, t_orc, w.queries, f"F={F} {layout} {order}", order=order)
    assert total > 10**9


@pytest.mark.parametrize("F", [16, 32, 64, 128])
def test_scaled_10m_1m_queries(rt, F):
    import torch
    w = dg.workload("scaled")
    t_orc = oracle.Tree(w.rects, w.ids, F)
    rng = np.random.default_rng(100 + F)
    sample = np.sort(rng.choice(w.queries.shape[0], 1500, replace=False))
    for layout in ("soa", "aos", "lohi"):
        with rt.RTree(torch.from_numpy(w.rects).cuda(), torch.from_numpy(w.ids).cuda(),
                      fanout=F, layout=layout) as t:
            total = check_sample(rt, t, t_orc, w.queries, sample, F)
        assert total > 10**8


def test_uneven_10m_every_query_exact(rt):
    import torch
    w = dg.workload("uneven")
    t_orc = oracle.Tree(w.rects, w.ids, 16)
    sizes = (w.queries[:, 2] - w.queries[:, 0]) * (w.queries[:, 3] - w.queries[:, 1])
    assert np.count_nonzero(sizes > 0.05 * 0.05) > 500
    with rt.RTree(torch.from_numpy(w.rects).cuda(), torch.from_numpy(w.ids).cuda(), fanout=16) as t:
        for mapping in ("warp_per_query", "work_queue"):
            compare_all(t, t_orc, w.queries, f"uneven {mapping}", mapping=mapping)


def test_join_2m_x_2m_full(rt):
    w = dg.workload("join")
    want = oracle.Tree(w.rects, w.ids, 32).join(oracle.Tree(w.rects_s, w.ids_s, 32), threads=THREADS)
    import torch
    with rt.RTree(torch.from_numpy(w.rects).cuda(), None, fanout=32) as a, \
            rt.RTree(torch.from_numpy(w.rects_s).cuda(), None, fanout=32) as b:
        res = a.join(b)
        _, got = res.to_numpy()
        res.close()
    assert np.array_equal(got, want) and len(want) > 10**5
    # the sorted-node prunings (O3, O4/O5) on sorted-children trees: same pairs
    with rt.RTree(torch.from_numpy(w.rects).cuda(), None, fanout=32, sort_children=True) as a, \
            rt.RTree(torch.from_numpy(w.rects_s).cuda(), None, fanout=32, sort_children=True) as b:
        res = a.join(b, prune="on")
        _, got = res.to_numpy()
        res.close()
    assert np.array_equal(got, want)


def test_scaled_10m_host_results_pipelined(rt):
    """The end-to-end form: host inputs, results to pinned host memory in
    about a dozen chunks, two selects in flight at once (as the benchmark's
    end-to-end loop runs them).  Checked on a seeded oracle sample and for
    CSR validity over every query."""
    import torch
    w = dg.workload("scaled")
    Q = w.queries.shape[0]
    t_orc = oracle.Tree(w.rects, w.ids, 64)
    rng = np.random.default_rng(164)
    sample = np.sort(rng.choice(Q, 1200, replace=False))
    o_off, o_ids = t_orc.select(w.queries[sample])
    stream = torch.cuda.current_stream()
    h_rects = torch.from_numpy(w.rects).pin_memory()
    h_ids = torch.from_numpy(w.ids).pin_memory()
    h_q = torch.from_numpy(w.queries).pin_memory()
    half = Q // 2
    off_a = torch.zeros(Q + 1, dtype=torch.int64).pin_memory()
    off_b = torch.zeros(half + 1, dtype=torch.int64).pin_memory()
    h = rt.rtree_build(h_rects, h_ids, 64, "aos", stream)
    with pytest.raises(rt.RTreeError) as e:  # no room: the count pass alone sizes the buffers
        rt.rtree_range_select_host_async(h, h_q, off_a, torch.empty(0, dtype=torch.int32), stream=stream)
    assert e.value.status == rt.RTREE_EOVERFLOW
    need = int(off_a[-1])
    assert need > 10**9
    ids_a = torch.empty(need, dtype=torch.int32).pin_memory()
    ids_b = torch.empty(need, dtype=torch.int32).pin_memory()
    pa = rt.rtree_range_select_host_async(h, h_q, off_a, ids_a, order="hilbert", stream=stream)
    pb = rt.rtree_range_select_host_async(h, h_q[:half], off_b, ids_b, order="hilbert", stream=stream)
    rt.rtree_free(h, stream=stream)
    total_a, total_b = pa.wait(), pb.wait()
    off, ids = off_a.numpy(), ids_a.numpy()
    assert total_a == need and off[-1] == total_a and np.all(np.diff(off) >= 0)
    assert np.array_equal(off_b.numpy(), off[:half + 1]) and total_b == off[half]
    assert np.array_equal(ids_b.numpy()[:total_b], ids[:total_b])
    for k, qi in enumerate(sample):
        assert np.array_equal(ids[off[qi]:off[qi + 1]], o_ids[o_off[k]:o_off[k + 1]]), f"query {qi}"
    d = np.diff(ids.astype(np.int64))
    inner = np.ones(d.size, bool)
    b = off[1:-1]
    inner[b[(b > 0) & (b < total_a)] - 1] = False
    assert np.all(d[inner] > 0), "segment not strictly ascending"
