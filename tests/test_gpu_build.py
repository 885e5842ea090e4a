"""Device STR bulk load vs the oracle's STR: the same tree, node by node.

Query results do not depend on the tree, but building the same tree on both
sides pins every step of the device build (centre keys, stable radix sorts,
slabs, packing, MBR reduction, top-down layout) exactly.  Also: input
validation and injected allocation failures (made on the host).
"""
import numpy as np
import pytest

import oracle
from gpu_util import gpu_ready
from paper_2309_16913_gb300 import datagen as dg
from test_oracle import random_case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rt():
    return gpu_ready()


def export_gpu(rt, rects, ids, F, layout):
    with rt.RTree(rects, ids, fanout=F, layout=layout) as t:
        return t.export(), t.info()


@pytest.mark.parametrize("layout", ["soa", "aos", "lohi"])
@pytest.mark.parametrize("F", [4, 8, 16, 32, 64, 128])
def test_tree_matches_oracle(rt, F, layout):
    for kind, n in (("uniform", 1), ("grid", F + 1), ("clustered", 4099), ("dups", 20011),
                    ("negative", 70001)):
        rects = random_case(kind, n, n)
        ids = np.arange(n, dtype=np.int32)[::-1].copy()
        got, info = export_gpu(rt, rects, ids, F, layout)
        want = oracle.Tree(rects, ids, F).export()
        for k in ("level_nodes", "counts", "leaf_ids"):
            assert np.array_equal(got[k], want[k]), (kind, n, F, layout, k)
        assert np.array_equal(got["mbrs"], want["mbrs"]), (kind, n, F, layout)
        assert info["levels"] == len(want["level_nodes"])
        lo, hi = rects[:, :2].min(0), rects[:, 2:].max(0)
        assert np.array_equal(info["root_mbr"], np.concatenate([lo, hi]))


def test_tree_matches_oracle_with_infinite_extents(rt):
    rects = random_case("uniform", 3000, 5)
    inf = np.float32(np.inf)
    rects[::17, 0] = -inf          # centre key -inf
    rects[::23, 2] = inf
    rects[::29, 0], rects[::29, 2] = -inf, inf   # centre key NaN -> 0
    rects[::31, 1], rects[::31, 3] = -0.0, -0.0  # centre key -0 -> +0
    ids = np.arange(3000, dtype=np.int32)
    got, _ = export_gpu(rt, rects, ids, 8, "soa")
    want = oracle.Tree(rects, ids, 8).export()
    for k in ("level_nodes", "counts", "leaf_ids", "mbrs"):
        assert np.array_equal(got[k], want[k]), k


def test_scaled_tree_matches_oracle(rt):
    w = dg.workload("scaled", n=1_000_000, q=1)
    got, _ = export_gpu(rt, w.rects, w.ids, 16, "soa")
    want = oracle.Tree(w.rects, w.ids, 16).export()
    for k in ("level_nodes", "counts", "leaf_ids", "mbrs"):
        assert np.array_equal(got[k], want[k]), k


def test_rejects_nan_and_inverted(rt):
    rects = random_case("uniform", 100, 1)
    bad = rects.copy()
    bad[37, 1] = np.nan
    with pytest.raises(rt.RTreeError) as e:
        rt.RTree(bad, None, fanout=16)
    assert e.value.status == rt.RTREE_EINVAL and "37" in str(e.value)
    bad = rects.copy()
    bad[5, 0], bad[5, 2] = 0.7, 0.6
    with pytest.raises(rt.RTreeError) as e:
        rt.RTree(bad, None, fanout=16)
    assert e.value.status == rt.RTREE_EINVAL
    with pytest.raises(rt.RTreeError):
        rt.RTree(rects, None, fanout=12)


def test_injected_allocation_failures_recover(rt):
    w = dg.workload("plain", n=5000, q=50)
    want = oracle.Tree(w.rects, w.ids, 16).select(w.queries)
    for k in range(0, 40, 3):
        rt.rtree_debug_fail_alloc_after(k)
        try:
            with rt.RTree(w.rects, w.ids, fanout=16) as t:
                res = t.range_select(w.queries)
                res.close()
        except rt.RTreeError as e:
            assert e.status == rt.RTREE_ENOMEM and "injected" in str(e)
        finally:
            rt.rtree_debug_fail_alloc_after(-1)
        with rt.RTree(w.rects, w.ids, fanout=16) as t:  # the library still works
            res = t.range_select(w.queries)
            off, ids = res.to_numpy()
            res.close()
        assert np.array_equal(off, want[0]) and np.array_equal(ids, want[1])


def test_autotune_returns_a_measured_choice(rt):
    w = dg.workload("scaled", n=300_000, q=4000)
    tune = rt.rtree_autotune(w.rects, w.queries, w.ids, fanouts=(16, 64))
    assert len(tune["all"]) == 2 * 3 * 2
    key = f"F{tune['fanout']}_{tune['layout']}_{tune['mapping']}"
    assert tune["all"][key] == min(tune["all"].values()) and tune["ms"] > 0
    # the chosen configuration still answers exactly
    want = oracle.Tree(w.rects, w.ids, tune["fanout"]).select(w.queries[:500])
    with rt.RTree(w.rects, w.ids, fanout=tune["fanout"], layout=tune["layout"]) as t:
        res = t.range_select(w.queries[:500], mapping=tune["mapping"])
        off, ids = res.to_numpy()
        res.close()
    assert np.array_equal(off, want[0]) and np.array_equal(ids, want[1])
