"""The join's two schedules -- one launch per level, and the persistent grid
over a device work queue -- against the CPU oracle, with and without the
sorted-node prunings, at equal and unequal tree heights and all layouts."""
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


def pairs_of(rt, a, b, **kw):
    res = a.join(b, **kw)
    try:
        return res.to_numpy()[1]
    finally:
        res.close()


@pytest.mark.parametrize("traversal", ["levels", "queue"])
@pytest.mark.parametrize("kind", ["uniform", "clustered", "grid", "dups", "negative"])
def test_join_schedules_match_oracle(rt, traversal, kind):
    r = random_case(kind, 30011, 31)
    s = random_case(kind, 9001, 32)
    rid = np.arange(30011, dtype=np.int32) * 3 - 11
    sid = np.random.default_rng(5).permutation(9001).astype(np.int32)
    want = oracle.Tree(r, rid, 16).join(oracle.Tree(s, sid, 16), threads=8)
    for fr, fs, lr, ls in ((16, 16, "soa", "soa"), (4, 64, "aos", "lohi"), (128, 8, "lohi", "aos"),
                           (32, 32, "aos", "aos")):
        for sort in (False, True):
            with rt.RTree(r, rid, fanout=fr, layout=lr, sort_children=sort) as a, \
                    rt.RTree(s, sid, fanout=fs, layout=ls, sort_children=sort) as b:
                got = pairs_of(rt, a, b, traversal=traversal, prune="on" if sort else "off")
            assert np.array_equal(got, want), (fr, fs, lr, ls, sort)


@pytest.mark.parametrize("traversal", ["levels", "queue"])
def test_join_workload_200k_and_edge_cases(rt, traversal):
    w = dg.workload("join", n=200_000)
    want = oracle.Tree(w.rects, w.ids, 32).join(oracle.Tree(w.rects_s, w.ids_s, 32), threads=8)
    with rt.RTree(w.rects, w.ids, fanout=32, sort_children=True) as a, \
            rt.RTree(w.rects_s, w.ids_s, fanout=32, sort_children=True) as b:
        for prune in ("off", "on"):
            assert np.array_equal(pairs_of(rt, a, b, traversal=traversal, prune=prune), want)
            assert np.array_equal(pairs_of(rt, b, a, traversal=traversal, prune=prune),
                                  want[np.lexsort((want[:, 0], want[:, 1]))][:, ::-1])
    # empty trees, disjoint trees, a single rectangle each
    far = w.rects_s[:1000] + np.float32(10.0)
    with rt.RTree(w.rects[:1000], None, fanout=8) as a, rt.RTree(far, None, fanout=8) as b, \
            rt.RTree(np.zeros((0, 4), np.float32), None, fanout=8) as e:
        assert pairs_of(rt, a, b, traversal=traversal).shape == (0, 2)
        assert pairs_of(rt, a, e, traversal=traversal).shape == (0, 2)
        assert pairs_of(rt, e, a, traversal=traversal).shape == (0, 2)
    one = np.array([[0.5, 0.5, 0.5, 0.5]], np.float32)
    with rt.RTree(one, None, fanout=4) as a, rt.RTree(one, None, fanout=128) as b:
        assert np.array_equal(pairs_of(rt, a, b, traversal=traversal), np.array([[0, 0]], np.int32))


def test_join_queue_wait_runs_out_then_next_join_is_exact(rt):
    """The queue's bounded waits, made to run out (one never-published item):
    RTREE_ETIMEOUT, and the next join on the same trees is exact."""
    w = dg.workload("join", n=100_000)
    want = oracle.Tree(w.rects, w.ids, 16).join(oracle.Tree(w.rects_s, w.ids_s, 16))
    with rt.RTree(w.rects, w.ids, fanout=16) as a, rt.RTree(w.rects_s, w.ids_s, fanout=16) as b:
        rt.rtree_debug_wq_wait(2_000_000, hold=True)
        with pytest.raises(rt.RTreeError) as e:
            pairs_of(rt, a, b, traversal="queue")
        assert e.value.status == rt.RTREE_ETIMEOUT
        assert np.array_equal(pairs_of(rt, a, b, traversal="queue"), want)
