"""R-tree join parity: CUDA path (through the C ABI) vs the CPU oracle.

Bit-exact: the same lexicographically sorted (r_id, s_id) pair list.
"""
import numpy as np
import pytest

import golden_io
import oracle
from gpu_util import gpu_ready
from paper_2309_16913_gb300 import datagen as dg
from test_oracle import random_case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rt():
    return gpu_ready()


def join_gpu(rt, r, rid, s, sid, fr, fs, lr="soa", ls="soa"):
    with rt.RTree(r, rid, fanout=fr, layout=lr) as a, rt.RTree(s, sid, fanout=fs, layout=ls) as b:
        res = a.join(b)
        try:
            return res.to_numpy()[1]
        finally:
            res.close()


def test_join_golden(rt):
    r, rid, s, sid, pairs = golden_io.join_case()
    for fr, fs in ((4, 4), (4, 8), (16, 4)):
        assert np.array_equal(join_gpu(rt, r, rid, s, sid, fr, fs), pairs)


@pytest.mark.parametrize("kind", ["uniform", "clustered", "grid", "dups", "negative"])
def test_join_random(rt, kind):
    r = random_case(kind, 20011, 11)
    s = random_case(kind, 7003, 12)
    rid = np.arange(20011, dtype=np.int32) * 2 - 5
    sid = np.random.default_rng(3).permutation(7003).astype(np.int32)
    want = oracle.brute_join(r, s, rid, sid) if kind != "dups" else \
        oracle.Tree(r, rid, 16).join(oracle.Tree(s, sid, 16))
    for fr, fs, lr, ls in ((16, 16, "soa", "soa"), (32, 4, "aos", "soa"), (4, 64, "soa", "aos"),
                           (128, 8, "aos", "aos"), (32, 16, "lohi", "soa"), (8, 32, "aos", "lohi")):
        got = join_gpu(rt, r, rid, s, sid, fr, fs, lr, ls)
        assert np.array_equal(got, want), (kind, fr, fs, lr, ls)


def test_join_unequal_heights(rt):
    r = random_case("uniform", 50000, 21)
    s = random_case("uniform", 300, 22)
    rid = np.arange(50000, dtype=np.int32)
    sid = np.arange(300, dtype=np.int32)
    want = oracle.brute_join(r, s, rid, sid)
    assert np.array_equal(join_gpu(rt, r, rid, s, sid, 4, 64), want)
    want_t = oracle.brute_join(s, r, sid, rid)
    assert np.array_equal(join_gpu(rt, s, sid, r, rid, 64, 4), want_t)


def test_join_shape_small(rt):
    w = dg.workload("join", n=200_000)
    want = oracle.Tree(w.rects, w.ids, 32).join(oracle.Tree(w.rects_s, w.ids_s, 32))
    got = join_gpu(rt, w.rects, w.ids, w.rects_s, w.ids_s, 32, 32)
    assert np.array_equal(got, want) and len(want) > 1000


def test_join_empty(rt):
    e = np.zeros((0, 4), np.float32)
    r = random_case("uniform", 100, 1)
    assert join_gpu(rt, e, None, r, None, 16, 16).shape == (0, 2)
    assert join_gpu(rt, r, None, e, None, 16, 16).shape == (0, 2)
    far = r + np.float32(10)
    assert join_gpu(rt, r, None, far, None, 16, 16).shape == (0, 2)


def test_self_join_diagonal(rt):
    r = random_case("grid", 3000, 5)
    rid = np.arange(3000, dtype=np.int32)
    got = join_gpu(rt, r, rid, r, rid, 8, 16)
    assert np.array_equal(got, oracle.brute_join(r, r, rid, rid))
    assert np.array_equal(got[got[:, 0] == got[:, 1]][:, 0], rid)


def test_join_stats_counts(rt):
    """rtree_join_stats: the pairs found equal the oracle's; the pruned join
    visits exactly the same node pairs (its prunings skip only tests whose
    pairs do not qualify); unequal heights show up as one-sided descents."""
    w = dg.workload("join", n=200_000)
    want = oracle.Tree(w.rects, w.ids, 8).join(oracle.Tree(w.rects_s, w.ids_s, 32))
    with rt.RTree(w.rects, w.ids, fanout=8, sort_children=True) as a, \
            rt.RTree(w.rects_s, w.ids_s, fanout=32, sort_children=True) as b:
        plain = a.join_stats(b, prune="off")
        pruned = a.join_stats(b, prune="on")
    assert plain["pairs_found"] == len(want) > 5000
    assert plain == pruned
    assert plain["pairs_r_descends"] > 0 and plain["pairs_s_descends"] == 0  # R (F=8) is taller
    assert plain["pairs_leaf"] >= plain["pairs_found"] / (8 * 32)
