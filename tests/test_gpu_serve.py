"""Serving loop: continuous batching over a resident index.

Every reply must be exactly the result of the same request run alone, however
requests were batched, split or run side by side on several streams.
"""
import threading

import numpy as np
import pytest

import oracle
from gpu_util import gpu_ready
from paper_2309_16913_gb300 import datagen as dg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rt():
    return gpu_ready()


def make_requests(seed, n_req, mean_side):
    rng = dg.rng_for(seed)
    reqs = []
    for k in range(n_req):
        if rng.random() < 0.15:   # probe join: 1k-3k uniform rectangles
            m = 1000 + int(rng.random() * 2000)
            reqs.append((1, dg.uniform_rects(m, rng, 0.0, 1e-3)))
        else:                     # 1-4 range queries, selectivity log-U[1e-7, 1e-3]
            m = 1 + int(rng.random() * 4)
            reqs.append((0, dg.selectivity_queries(m, rng, 1e-7, 1e-3, mean_side)))
    return reqs


@pytest.mark.parametrize("workers,max_ids", [(3, 4 << 20), (2, "half")])
def test_replies_equal_results_alone(rt, workers, max_ids):
    import torch
    w = dg.workload("serve", n=600_000, q=1)
    reqs = make_requests(11, 240, dg._log_uniform_mean(1e-5, 1e-3))
    t_orc = oracle.Tree(w.rects, w.ids, 16)
    with rt.RTree(torch.from_numpy(w.rects).cuda(), torch.from_numpy(w.ids).cuda(), fanout=16) as t:
        alone = []
        for _, r in reqs:
            res = t.range_select(r)
            alone.append(res.to_numpy())
            res.close()
        small = max_ids == "half"
        if small:  # the largest reply cannot fit: it must take the fallback path
            max_ids = max(1, max(a[1].size for a in alone) // 2)
        srv = rt.Server(t, workers=workers, max_batch_queries=8192, max_batch_ids=max_ids)
        tickets = [None] * len(reqs)

        def client(idx):
            for i in idx:
                tickets[i] = srv.submit(reqs[i][1], reqs[i][0])

        threads = [threading.Thread(target=client, args=(range(c, len(reqs), 4),)) for c in range(4)]
        for th in threads:
            th.start()
        for th in threads:
            th.join()
        for i, tk in enumerate(tickets):
            off, ids, lat = srv.wait(tk, timeout_us=60_000_000)
            assert np.array_equal(off, alone[i][0]) and np.array_equal(ids, alone[i][1]), i
            assert lat > 0
        for i in range(0, len(reqs), 37):  # and alone equals the oracle
            want = t_orc.select(reqs[i][1])
            assert np.array_equal(alone[i][0], want[0]) and np.array_equal(alone[i][1], want[1])
        st = srv.stats()
        assert st["completed"] == len(reqs) and st["pending"] == 0
        assert 0 < st["p50_us"] <= st["p99_us"] <= st["max_us"]
        assert st["batches"] >= 1
        if small:
            assert st["fallbacks"] > 0  # the small budget forced the allocating path
        srv.stop()


def test_wait_timeout_and_stop_answers_pending(rt):
    w = dg.workload("plain", n=50_000, q=200)
    with rt.RTree(w.rects, w.ids, fanout=16) as t:
        srv = rt.Server(t, workers=1)
        with pytest.raises(rt.RTreeError) as e:
            srv.wait(987654321, timeout_us=1000)
        assert e.value.status == rt.RTREE_ETIMEOUT
        tickets = [srv.submit(w.queries[i:i + 3]) for i in range(0, 200, 3)]
        first = srv.wait(tickets[0])
        srv_handle = srv.handle
        assert srv_handle
        rest = [srv.wait(tk) for tk in tickets[1:]]
        srv.stop()
        want = oracle.Tree(w.rects, w.ids, 16).select(w.queries[0:3])
        assert np.array_equal(first[0], want[0]) and np.array_equal(first[1], want[1])
        assert len(rest) == len(tickets) - 1
