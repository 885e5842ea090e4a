"""Graph-captured batched select (plans) vs the CPU oracle.

A plan records the whole select pipeline as one CUDA graph per batch-size
bucket; results must equal the oracle's exactly for every batch, across
repeated replays and bucket changes, with either thread mapping.
"""
import numpy as np
import pytest

import oracle
from gpu_util import assert_csr_equal, gpu_ready
from paper_2309_16913_gb300 import datagen as dg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rt():
    return gpu_ready()


@pytest.mark.parametrize("mapping", ["warp_per_query", "work_queue"])
def test_plan_matches_oracle_over_batches(rt, mapping):
    import torch
    w = dg.workload("uneven", n=300_000, q=5000)
    t_orc = oracle.Tree(w.rects, w.ids, 16)
    with rt.RTree(torch.from_numpy(w.rects).cuda(), torch.from_numpy(w.ids).cuda(), fanout=16) as t:
        plan = rt.Plan(t, max_queries=4096, max_ids=20_000_000, mapping=mapping)
        try:
            start = 0
            for q in (1, 100, 256, 257, 1000, 4096, 100, 3000, 1):  # replays and bucket changes
                qs = w.queries[start:start + q]
                start = (start + q) % 900
                total = plan.run(torch.from_numpy(np.ascontiguousarray(qs)).cuda())
                want = t_orc.select(qs)
                assert total == want[0][-1]
                assert_csr_equal(plan.to_numpy(), want, f"plan q={q} {mapping}")
        finally:
            plan.close()


def test_plan_host_queries_and_empty_batch(rt):
    w = dg.workload("plain", n=50_000, q=700)
    with rt.RTree(w.rects, w.ids, fanout=32) as t:
        plan = rt.Plan(t, max_queries=1000, max_ids=1_000_000)
        total = plan.run(w.queries)  # host memory
        assert_csr_equal(plan.to_numpy(), oracle.Tree(w.rects, w.ids, 32).select(w.queries), "host")
        assert plan.run(np.zeros((0, 4), np.float32)) == 0
        assert plan.offsets_tensor().cpu().numpy().tolist() == [0]
        plan.close()
        assert total > 0


def test_plan_overflow_is_reported(rt):
    import torch
    w = dg.workload("plain", n=100_000, q=1000)
    want = oracle.Tree(w.rects, w.ids, 16).select(w.queries)
    with rt.RTree(w.rects, w.ids, fanout=16) as t:
        plan = rt.Plan(t, max_queries=1000, max_ids=1000)
        q = torch.from_numpy(w.queries).cuda()
        with pytest.raises(rt.RTreeError) as e:
            plan.run(q)
        assert e.value.status == rt.RTREE_EOVERFLOW and str(want[0][-1]) in str(e.value)
        small = w.queries[:50]
        total = plan.run(torch.from_numpy(small).cuda())   # fits: works after an overflow
        assert_csr_equal(plan.to_numpy(), oracle.Tree(w.rects, w.ids, 16).select(small), "after overflow")
        with pytest.raises(rt.RTreeError) as e:
            plan.run(torch.from_numpy(np.concatenate([w.queries, w.queries])).cuda())
        assert e.value.status == rt.RTREE_EOVERFLOW and "at most 1000" in str(e.value)
        plan.close()
        assert total >= 0
