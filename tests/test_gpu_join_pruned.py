"""Sorted-children trees and the pruned join (O3, O4/O5 of Section 4.2):
CUDA path through the C ABI vs the CPU oracle, bit-exact.

The device build with sort_children must produce the oracle's sorted tree
node by node, and the pruned join must return exactly the pairs of the plain
join (which the oracle pins by brute force)."""
import numpy as np
import pytest

import golden_io
import oracle
from gpu_util import gpu_ready, select_gpu, assert_csr_equal
from paper_2309_16913_gb300 import datagen as dg
from test_oracle import random_case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rt():
    return gpu_ready()


def pruned_gpu(rt, r, rid, s, sid, fr, fs, lr="soa", ls="soa", prune="on"):
    with rt.RTree(r, rid, fanout=fr, layout=lr, sort_children=True) as a, \
            rt.RTree(s, sid, fanout=fs, layout=ls, sort_children=True) as b:
        res = a.join(b, prune=prune)
        try:
            return res.to_numpy()[1]
        finally:
            res.close()


@pytest.mark.parametrize("layout", ["soa", "aos", "lohi"])
@pytest.mark.parametrize("F", [4, 8, 16, 32, 64, 128])
def test_sorted_tree_matches_oracle(rt, F, layout):
    for kind, n in (("grid", 5000), ("dups", 20011), ("clustered", 4099), ("negative", 70001), ("uniform", 1)):
        rects = random_case(kind, n, n)
        ids = np.arange(n, dtype=np.int32)[::-1].copy()
        with rt.RTree(rects, ids, fanout=F, layout=layout, sort_children=True) as t:
            got, info = t.export(), t.info()
        want = oracle.Tree(rects, ids, F, sort_children=True).export()
        for k in ("level_nodes", "counts", "leaf_ids", "mbrs"):
            assert np.array_equal(got[k], want[k]), (kind, n, F, layout, k)
        assert info["sort_children"] == 1


def test_sorted_tree_signed_zero_ties(rt):
    # -0 and +0 are equal keys: such entries keep their packing order
    rects = random_case("grid", 4000, 3)
    rects[::3, 0] = np.float32(-0.0)
    rects[1::3, 0] = np.float32(0.0)
    rects[:, 2] = np.maximum(rects[:, 2], np.float32(0.0))
    ids = np.arange(4000, dtype=np.int32)
    with rt.RTree(rects, ids, fanout=16, sort_children=True) as t:
        got = t.export()
    want = oracle.Tree(rects, ids, 16, sort_children=True).export()
    for k in ("level_nodes", "counts", "leaf_ids"):
        assert np.array_equal(got[k], want[k]), k
    # values, not bits: a node MBR's minimum over -0 and +0 may carry either sign
    assert np.array_equal(got["mbrs"], want["mbrs"])


def test_select_on_sorted_tree(rt):
    w = dg.workload("plain", n=50000, q=2000)
    want = oracle.brute_select(w.rects, w.queries, w.ids)
    import torch
    r = torch.from_numpy(w.rects).cuda()
    q = torch.from_numpy(w.queries).cuda()
    for F in (16, 64):
        with rt.RTree(r, None, fanout=F, sort_children=True) as t:
            res = t.range_select(q)
            got = res.to_numpy()
            res.close()
        assert_csr_equal(got, want, f"F{F}")


def test_pruned_join_golden(rt):
    r, rid, s, sid, pairs = golden_io.join_case()
    for fr, fs in ((4, 4), (4, 8), (16, 4)):
        assert np.array_equal(pruned_gpu(rt, r, rid, s, sid, fr, fs), pairs)


@pytest.mark.parametrize("kind", ["uniform", "clustered", "grid", "dups", "negative", "points"])
def test_pruned_join_random(rt, kind):
    r = random_case(kind, 20011, 31)
    s = random_case(kind, 7003, 32)
    rid = np.arange(20011, dtype=np.int32) * 2 - 5
    sid = np.random.default_rng(4).permutation(7003).astype(np.int32)
    want = oracle.brute_join(r, s, rid, sid)
    got_o, _ = oracle.Tree(r, rid, 16, sort_children=True).join_pruned(
        oracle.Tree(s, sid, 16, sort_children=True))
    assert np.array_equal(got_o, want)
    for fr, fs, lr, ls in ((16, 16, "soa", "soa"), (32, 4, "aos", "soa"), (4, 64, "soa", "aos"),
                           (128, 8, "aos", "aos"), (8, 128, "soa", "soa"), (64, 64, "aos", "soa"),
                           (32, 32, "lohi", "lohi"), (16, 64, "lohi", "aos")):
        got = pruned_gpu(rt, r, rid, s, sid, fr, fs, lr, ls)
        assert np.array_equal(got, want), (kind, fr, fs, lr, ls)


def test_pruned_join_workload_shape(rt):
    w = dg.workload("join", n=200_000)
    want = oracle.Tree(w.rects, w.ids, 32).join(oracle.Tree(w.rects_s, w.ids_s, 32))
    got = pruned_gpu(rt, w.rects, w.ids, w.rects_s, w.ids_s, 32, 32)
    assert np.array_equal(got, want) and len(want) > 1000
    # auto prunes on sorted trees, off takes the plain kernel: same pairs
    assert np.array_equal(pruned_gpu(rt, w.rects, w.ids, w.rects_s, w.ids_s, 32, 32, prune="auto"), want)
    assert np.array_equal(pruned_gpu(rt, w.rects, w.ids, w.rects_s, w.ids_s, 32, 32, prune="off"), want)


def test_pruned_join_unequal_heights_and_empty(rt):
    r = random_case("uniform", 50000, 41)
    s = random_case("uniform", 300, 42)
    rid = np.arange(50000, dtype=np.int32)
    sid = np.arange(300, dtype=np.int32)
    assert np.array_equal(pruned_gpu(rt, r, rid, s, sid, 4, 64), oracle.brute_join(r, s, rid, sid))
    assert np.array_equal(pruned_gpu(rt, s, sid, r, rid, 64, 4), oracle.brute_join(s, r, sid, rid))
    e = np.zeros((0, 4), np.float32)
    assert pruned_gpu(rt, e, None, r, None, 16, 16).shape == (0, 2)
    assert pruned_gpu(rt, r, None, r + np.float32(10), None, 16, 16).shape == (0, 2)


def test_prune_on_needs_sorted_trees(rt):
    r = random_case("uniform", 1000, 1)
    with rt.RTree(r, None, fanout=16) as a, rt.RTree(r, None, fanout=16, sort_children=True) as b:
        with pytest.raises(rt.RTreeError) as e:
            a.join(b, prune="on")
        assert e.value.status == rt.RTREE_EINVAL and "sort_children" in str(e.value)
        # auto falls back to the plain kernel when a tree is unsorted
        res = a.join(b, prune="auto")
        got = res.to_numpy()[1]
        res.close()
    assert np.array_equal(got, oracle.brute_join(r, r))
