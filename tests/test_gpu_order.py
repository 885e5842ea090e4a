"""Hilbert-ordered traversal of a query batch: results must be exactly the
oracle's, in the caller's query order, whatever order the warps take."""
import numpy as np
import pytest

import oracle
from gpu_util import gpu_ready, select_gpu, assert_csr_equal
from paper_2309_16913_gb300 import datagen as dg
from test_oracle import random_case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rt():
    return gpu_ready()


@pytest.mark.parametrize("mapping", ["warp_per_query", "work_queue"])
@pytest.mark.parametrize("F,layout", [(16, "soa"), (64, "aos"), (4, "aos"), (128, "soa"), (32, "lohi")])
def test_hilbert_order_matches_oracle(rt, F, layout, mapping):
    w = dg.workload("scaled", n=300_000, q=20_000)
    want = oracle.Tree(w.rects, w.ids, F).select(w.queries)
    got = select_gpu(rt, w.rects, w.ids, w.queries, F, layout, order="hilbert", mapping=mapping)
    assert_csr_equal(got, want, f"F{F} {layout} {mapping}")


def test_hilbert_order_unsorted_mode_same_sets(rt):
    w = dg.workload("plain", n=50_000, q=3000)
    wo, wi = oracle.brute_select(w.rects, w.queries, w.ids)
    go, gi = select_gpu(rt, w.rects, w.ids, w.queries, 16, "soa", order="hilbert", unsorted=True)
    assert np.array_equal(go, wo)
    for k in range(len(wo) - 1):
        assert np.array_equal(np.sort(gi[go[k]:go[k + 1]]), wi[wo[k]:wo[k + 1]]), k


def test_hilbert_order_special_queries(rt):
    rects = random_case("uniform", 5000, 7)
    inf, nan = np.float32(np.inf), np.float32(np.nan)
    q = np.array([[-inf, -inf, inf, inf], [nan, 0, 1, 1], [0.5, 0.5, 0.4, 0.6],
                  [2, 2, 3, 3], [0.2, 0.2, 0.2, 0.2], [-inf, 0.3, inf, 0.31]], np.float32)
    q = np.concatenate([q, random_case("uniform", 300, 8)])
    want = oracle.brute_select(rects, q)
    assert_csr_equal(select_gpu(rt, rects, None, q, 16, "soa", order="hilbert"), want)


def test_hilbert_order_degenerate_boxes(rt):
    # all data in one point (zero-width bounding box), and infinite extents
    pts = np.tile(np.array([[0.25, 0.75, 0.25, 0.75]], np.float32), (700, 1))
    q = random_case("uniform", 200, 3)
    q[::7] = [0.25, 0.75, 0.25, 0.75]
    assert_csr_equal(select_gpu(rt, pts, None, q, 8, "soa", order="hilbert"), oracle.brute_select(pts, q))
    r = random_case("uniform", 3000, 4)
    r[::50, 0] = -np.inf
    r[::70, 3] = np.inf
    assert_csr_equal(select_gpu(rt, r, None, q, 16, "aos", order="hilbert"), oracle.brute_select(r, q))
    assert_csr_equal(select_gpu(rt, r, None, q[:1], 16, "aos", order="hilbert"),
                     oracle.brute_select(r, q[:1]))


def test_plan_refuses_order(rt):
    import ctypes as C
    w = dg.workload("plain", n=2000, q=10)
    lib = rt.load_library()
    with rt.RTree(w.rects, w.ids, fanout=16) as t:
        opts = rt.rtree_select_opts_t()
        opts.order = rt.ORDERS["hilbert"]
        out = C.c_void_p()
        assert lib.rtree_plan_create(t.handle, 256, 1 << 16, C.byref(opts), C.byref(out)) == rt.RTREE_EINVAL
        assert b"input order" in lib.rtree_last_error()


def test_autotune_tries_orders(rt):
    w = dg.workload("scaled", n=200_000, q=3000)
    tune = rt.rtree_autotune(w.rects, w.queries, w.ids, fanouts=(16, 64), orders=True)
    assert len(tune["all"]) == 2 * 3 * 2 * 2
    assert sum(k.endswith("_hilbert") for k in tune["all"]) == 12
    assert tune["order"] in ("input", "hilbert") and abs(tune["ms"] - min(tune["all"].values())) < 1e-3
    want = oracle.Tree(w.rects, w.ids, tune["fanout"]).select(w.queries)
    got = select_gpu(rt, w.rects, w.ids, w.queries, tune["fanout"], tune["layout"],
                     mapping=tune["mapping"], order=tune["order"])
    assert_csr_equal(got, want, str(tune))
