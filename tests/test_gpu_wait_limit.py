"""The work-queue mapping's bounded device waits, made to run out on purpose.

Warps of the persistent work-queue select wait for work that other warps
publish.  Every such wait has a limit; past it the warp records a timeout
and returns, and the call reports RTREE_ETIMEOUT.  The test hook
rtree_debug_wq_wait lowers the limit for one pass and counts one work item
that is never published, so the pass can only end through those limits.
No GPU fault is involved.  The next call on the same tree must be exact.
"""
import numpy as np
import pytest

import oracle
from gpu_util import gpu_ready
from paper_2309_16913_gb300 import datagen as dg

pytestmark = pytest.mark.gpu


def test_work_queue_wait_runs_out_then_next_call_is_exact():
    import torch
    rt = gpu_ready()
    w = dg.workload("plain", n=60_000, q=3_000)
    want = oracle.Tree(w.rects, w.ids, 16).select(w.queries)
    q = torch.from_numpy(w.queries).cuda()
    with rt.RTree(torch.from_numpy(w.rects).cuda(), torch.from_numpy(w.ids).cuda(), fanout=16) as t:
        for _ in range(2):
            rt.rtree_debug_wq_wait(2_000_000, hold=True)  # about a millisecond per wait
            with pytest.raises(rt.RTreeError) as e:
                t.range_select(q, mapping="work_queue").close()
            assert e.value.status == rt.RTREE_ETIMEOUT, str(e.value)
            for mapping in ("work_queue", "warp_per_query"):
                res = t.range_select(q, mapping=mapping)
                try:
                    off, ids = res.to_numpy()
                finally:
                    res.close()
                assert np.array_equal(off, want[0]) and np.array_equal(ids, want[1]), mapping


def test_lowered_limit_alone_still_completes():
    """A short limit with every item published: waits end as soon as work
    or the end of the pass is seen, so the call succeeds."""
    import torch
    rt = gpu_ready()
    w = dg.workload("plain", n=60_000, q=3_000)
    want = oracle.Tree(w.rects, w.ids, 16).select(w.queries)
    q = torch.from_numpy(w.queries).cuda()
    with rt.RTree(torch.from_numpy(w.rects).cuda(), torch.from_numpy(w.ids).cuda(), fanout=16) as t:
        rt.rtree_debug_wq_wait(200_000_000, hold=False)
        res = t.range_select(q, mapping="work_queue")
        try:
            off, ids = res.to_numpy()
        finally:
            res.close()
        assert np.array_equal(off, want[0]) and np.array_equal(ids, want[1])
