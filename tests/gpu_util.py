"""Helpers shared by the GPU parity tests (test helper, not product code)."""
import numpy as np


def gpu_ready():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2309_16913_gb300 import build
    build.build()
    from paper_2309_16913_gb300 import rtree as rt
    rt.load_library()
    return rt


def select_gpu(rt, rects, ids, queries, fanout=16, layout="soa", device_inputs=True, **kw):
    import torch
    if device_inputs:
        r = torch.from_numpy(np.ascontiguousarray(rects, np.float32).reshape(-1, 4)).cuda()
        i = None if ids is None else torch.from_numpy(np.ascontiguousarray(ids, np.int32)).cuda()
        q = torch.from_numpy(np.ascontiguousarray(queries, np.float32).reshape(-1, 4)).cuda()
    else:
        r, i, q = rects, ids, queries
    with rt.RTree(r, i, fanout=fanout, layout=layout) as t:
        res = t.range_select(q, **kw)
        try:
            return res.to_numpy()
        finally:
            res.close()


def assert_csr_equal(got, want, context=""):
    go, gi = got
    wo, wi = want
    assert go.shape == wo.shape, context
    if not np.array_equal(go, wo):
        bad = np.nonzero(np.diff(go) != np.diff(wo))[0][:5]
        raise AssertionError(f"{context}: per-query counts differ at queries {bad.tolist()}")
    if not np.array_equal(gi, wi):
        k = int(np.nonzero(gi != wi)[0][0])
        qi = int(np.searchsorted(wo, k, side="right") - 1)
        raise AssertionError(f"{context}: ids differ first at position {k} (query {qi})")
