"""Range-select parity: CUDA path (through the C ABI) vs the CPU oracle.

The bar is bit-exact: the same sorted id list for every query (the paper's
select result is a set; comparisons are exact float32, nothing is rounded).
"""
import numpy as np
import pytest

import golden_io
import oracle
from gpu_util import assert_csr_equal, gpu_ready, select_gpu
from paper_2309_16913_gb300 import datagen as dg
from test_oracle import random_case

pytestmark = pytest.mark.gpu
INF = np.float32(np.inf)
FANOUTS = [4, 8, 16, 32, 64, 128]


@pytest.fixture(scope="module")
def rt():
    return gpu_ready()


def test_predicate_golden_cases(rt):
    for a, b, exp in golden_io.predicate_cases():
        ids = np.array([7], np.int32)
        off, got = select_gpu(rt, a[None], ids, b[None], fanout=4)
        assert len(got) == exp, (a, b, exp)
        off, got = select_gpu(rt, b[None], ids, a[None], fanout=4, layout="aos")
        assert len(got) == exp, (b, a, exp)


@pytest.mark.parametrize("layout", ["soa", "aos", "lohi"])
@pytest.mark.parametrize("F", [4, 8, 16])
def test_select_golden(rt, F, layout):
    rects, ids, queries, expected = golden_io.select_case()
    off, got = select_gpu(rt, rects, ids, queries, fanout=F, layout=layout)
    for i, e in enumerate(expected):
        assert np.array_equal(got[off[i]:off[i + 1]], e), (i, F, layout)


@pytest.mark.parametrize("layout", ["soa", "aos", "lohi"])
@pytest.mark.parametrize("F", FANOUTS)
def test_plain_workload_full_size(rt, F, layout):
    """100k uniform rectangles, 1k queries: every query checked."""
    w = dg.workload("plain")
    want = oracle.Tree(w.rects, w.ids, F).select(w.queries)
    got = select_gpu(rt, w.rects, w.ids, w.queries, fanout=F, layout=layout)
    assert_csr_equal(got, want, f"plain F={F} {layout}")
    assert want[0][-1] > 1000


@pytest.mark.parametrize("kind", ["clustered", "grid", "points", "dups", "negative"])
@pytest.mark.parametrize("F", [4, 16, 64])
def test_random_kinds(rt, kind, F):
    n = 30011
    rects = random_case(kind, n, 3)
    ids = np.random.default_rng(1).permutation(n).astype(np.int32) - np.int32(12345)
    queries = random_case(kind, 700, 4)
    want = oracle.Tree(rects, ids, F).select(queries)
    for layout in ("soa", "aos", "lohi"):
        got = select_gpu(rt, rects, ids, queries, fanout=F, layout=layout)
        assert_csr_equal(got, want, f"{kind} F={F} {layout}")


def test_scaled_shape_small(rt):
    """The scaled workload's distributions at 200k rects / 3k queries."""
    w = dg.workload("scaled", n=200_000, q=3000)
    want = oracle.Tree(w.rects, w.ids, 16).select(w.queries)
    for F in (16, 32, 64):
        got = select_gpu(rt, w.rects, w.ids, w.queries, fanout=F)
        assert_csr_equal(got, want, f"scaled-small F={F}")


def test_uneven_shape_small(rt):
    """Heavy-tailed query mix (1% large queries) at 300k rects."""
    w = dg.workload("uneven", n=300_000, q=4000)
    want = oracle.Tree(w.rects, w.ids, 16).select(w.queries)
    got = select_gpu(rt, w.rects, w.ids, w.queries, fanout=16)
    assert_csr_equal(got, want, "uneven-small")
    counts = np.diff(want[0])
    assert counts.max() > 4096  # exercises the long-segment sort


def test_unsorted_mode_is_a_permutation(rt):
    w = dg.workload("plain", n=50_000, q=500)
    so, si = select_gpu(rt, w.rects, w.ids, w.queries, fanout=16)
    uo, ui = select_gpu(rt, w.rects, w.ids, w.queries, fanout=16, unsorted=True)
    assert np.array_equal(so, uo)
    for i in range(len(so) - 1):
        assert np.array_equal(np.sort(ui[uo[i]:uo[i + 1]]), si[so[i]:so[i + 1]])


def test_host_inputs_match_device_inputs(rt):
    w = dg.workload("plain", n=40_000, q=400)
    a = select_gpu(rt, w.rects, w.ids, w.queries, fanout=16, device_inputs=True)
    b = select_gpu(rt, w.rects, w.ids, w.queries, fanout=16, device_inputs=False)
    assert_csr_equal(a, b, "host vs device inputs")


def test_unaligned_device_inputs(rt):
    import torch
    w = dg.workload("plain", n=10_000, q=100)
    buf = torch.zeros(w.rects.size + 1, dtype=torch.float32, device="cuda")
    buf[1:] = torch.from_numpy(w.rects.reshape(-1)).cuda()
    r = buf[1:].view(-1, 4)  # 4 bytes off a 16-byte boundary
    qbuf = torch.zeros(w.queries.size + 2, dtype=torch.float32, device="cuda")
    qbuf[2:] = torch.from_numpy(w.queries.reshape(-1)).cuda()
    q = qbuf[2:].view(-1, 4)
    assert r.data_ptr() % 16 != 0 and q.data_ptr() % 16 != 0
    got = select_gpu(rt, r, None, q, fanout=16, device_inputs=False)
    want = oracle.Tree(w.rects, None, 16).select(w.queries)
    assert_csr_equal(got, want, "unaligned")


# ------------------------------------------------------------ edge cases
@pytest.mark.parametrize("F", [4, 16, 64])
def test_small_trees(rt, F):
    for n in (1, F - 1, F, F + 1, F * F - 1, F * F, F * F + 1):
        rects = random_case("grid", n, n)
        ids = np.arange(n, dtype=np.int32)
        queries = np.concatenate([random_case("grid", 50, n + 1),
                                  np.array([[-INF, -INF, INF, INF]], np.float32)])
        want = oracle.Tree(rects, ids, F).select(queries)
        got = select_gpu(rt, rects, ids, queries, fanout=F)
        assert_csr_equal(got, want, f"n={n} F={F}")
        assert np.array_equal(got[1][got[0][-2]:], ids)  # whole plane: every id


def test_empty_tree_and_empty_batch(rt):
    e = np.zeros((0, 4), np.float32)
    q = np.array([[-INF, -INF, INF, INF], [0, 0, 1, 1]], np.float32)
    off, ids = select_gpu(rt, e, None, q, fanout=16)
    assert off.tolist() == [0, 0, 0] and ids.size == 0
    w = dg.workload("plain", n=1000, q=1)
    off, ids = select_gpu(rt, w.rects, w.ids, np.zeros((0, 4), np.float32), fanout=16)
    assert off.tolist() == [0] and ids.size == 0


def test_special_queries(rt):
    w = dg.workload("plain", n=20_000, q=10)
    nan = np.float32(np.nan)
    q = np.array([
        [-INF, -INF, INF, INF],           # everything
        [5, 5, 6, 6],                     # disjoint from the data
        [nan, 0, 1, 1],                   # NaN: the predicate is false
        [0.6, 0.2, 0.4, 0.8],             # inverted in x: evaluated literally
        [0.5, 0.5, 0.5, 0.5],             # a point
        [0.25, -INF, 0.25, INF],          # a vertical line through everything
    ], np.float32)
    want = oracle.Tree(w.rects, w.ids, 16).select(q)
    got = select_gpu(rt, w.rects, w.ids, q, fanout=16)
    assert_csr_equal(got, want, "special queries")
    assert want[0][1] - want[0][0] == 20_000 and want[0][2] == want[0][1]
    assert want[0][3] == want[0][2]


def test_duplicate_and_extreme_ids(rt):
    rects = random_case("dups", 5000, 9)
    ids = np.full(5000, 7, np.int32)
    ids[::3] = np.iinfo(np.int32).min
    ids[1::3] = np.iinfo(np.int32).max
    q = random_case("grid", 200, 10)
    want = oracle.Tree(rects, ids, 8).select(q)
    got = select_gpu(rt, rects, ids, q, fanout=8)
    assert_csr_equal(got, want, "duplicate ids")


def test_long_segments_msd_and_skewed_fallback(rt):
    """Segments longer than 16384 ids take the MSD partition; ids crowded
    into one bucket take the global fallback.  Both must match the oracle."""
    n = 120_000
    rects = random_case("uniform", n, 77)
    rng = np.random.default_rng(5)
    spread = rng.permutation(n).astype(np.int32) * np.int32(7) - np.int32(400_000)
    crowded = np.arange(n, dtype=np.int32)
    crowded[::9999] += np.int32(1 << 30)      # a few far ids: most land in one bucket
    queries = np.array([[-INF, -INF, INF, INF], [0.0, 0.0, 0.6, 0.7], [0.2, 0.1, 0.9, 0.5],
                        [0.5, 0.5, 0.55, 0.55]], np.float32)
    for ids in (spread, crowded):
        want = oracle.Tree(rects, ids, 16).select(queries)
        assert np.diff(want[0]).max() > 16384
        for F in (16, 64):
            got = select_gpu(rt, rects, ids, queries, fanout=F)
            assert_csr_equal(got, want, f"long segments F={F}")


@pytest.mark.parametrize("case", ["ragged", "crowded", "crowded_20k", "over_128k", "two_values",
                                  "one_value", "both_signs_mid", "large_buckets"])
def test_sort_edge_cases(rt, case):
    """Per-query sort edges: a segment just above 16384 ids (ragged), a
    dense id run with far outliers (crowded buckets, at 60k and at 20k ids),
    a segment over 131072 ids, duplicate ids (two values; one value, all
    keys equal), and mid-size segments whose ids straddle zero (value-range
    buckets must not crowd), and a 40953-id segment whose value buckets all
    hold 17 ids (every warp takes the 32-key network)."""
    everything = np.array([[-INF, -INF, INF, INF]], np.float32)
    rng = np.random.default_rng(13)
    queries = everything
    if case == "ragged":
        n = 16391
        ids = rng.permutation(n).astype(np.int32) * np.int32(3)
        rects = random_case("uniform", n, 21)
        queries = np.concatenate([everything, np.array([[0.0, 0.0, 0.999, 0.9995]], np.float32)])
    elif case == "crowded":
        n = 60_000
        ids = np.arange(n, dtype=np.int32)
        ids[::6000] += np.int32(1 << 20)
        rects = random_case("uniform", n, 22)
    elif case == "crowded_20k":  # crowded in the one-CTA sort above 16384 ids: MSD path
        n = 20_000
        ids = np.arange(n, dtype=np.int32)
        ids[::5000] += np.int32(1 << 20)
        rects = random_case("uniform", n, 27)
    elif case == "over_128k":
        n = 140_000
        ids = rng.permutation(n).astype(np.int32)
        rects = random_case("uniform", n, 23)
        queries = np.concatenate([everything, np.array([[0.0, 0.0, 0.95, 0.98]], np.float32)])
    elif case == "two_values":
        n = 30_000
        ids = np.where(np.arange(n) % 2 == 0, 7, 8).astype(np.int32)
        rects = random_case("uniform", n, 24)
    elif case == "large_buckets":
        ids = (64 * np.arange(2409)[:, None] + np.arange(17)[None, :]).astype(np.int32).ravel()
        ids = rng.permutation(ids)
        n = ids.size
        rects = random_case("uniform", n, 28)
    elif case == "one_value":
        n = 20_000
        ids = np.full(n, -5, np.int32)
        rects = random_case("uniform", n, 25)
    else:
        n = 12_000
        ids = (rng.permutation(n) - n // 2).astype(np.int32)
        rects = random_case("uniform", n, 26)
        lo = rng.random((40, 2)).astype(np.float32) * np.float32(0.5)
        queries = np.concatenate([lo, lo + np.float32(0.45)], axis=1).astype(np.float32)
    want = oracle.Tree(rects, ids, 16).select(queries)
    if case == "both_signs_mid":
        c = np.diff(want[0])
        assert ((c > 256) & (c <= 16384)).sum() > 20
    else:
        assert np.diff(want[0]).max() > 16384
    for F in (16, 64):
        got = select_gpu(rt, rects, ids, queries, fanout=F)
        assert_csr_equal(got, want, f"{case} F={F}")


def test_crowded_buckets_fall_back_to_lsd(rt):
    """Dense id runs plus a few far outliers crowd the shared-memory buckets
    of mid-size segments; the LSD fallback must give the same result."""
    n = 40_000
    rects = random_case("uniform", n, 91)
    ids = np.arange(n, dtype=np.int32)
    ids[::4000] += np.int32(1 << 22)
    rng = np.random.default_rng(8)
    lo = rng.random((60, 2)).astype(np.float32) * np.float32(0.7)
    side = (rng.random((60, 1)) * 0.3).astype(np.float32)
    queries = np.concatenate([lo, lo + side], axis=1).astype(np.float32)
    want = oracle.Tree(rects, ids, 16).select(queries)
    counts = np.diff(want[0])
    assert ((counts > 256) & (counts <= 16384)).sum() > 20
    got = select_gpu(rt, rects, ids, queries, fanout=16)
    assert_csr_equal(got, want, "crowded buckets")


@pytest.mark.parametrize("unsorted", [False, True])
def test_work_queue_mapping(rt, unsorted):
    """The persistent work-queue mapping (warps split large queries between
    them) gives the same result sets as the oracle; heavy queries included."""
    w = dg.workload("uneven", n=400_000, q=6000)
    want = oracle.Tree(w.rects, w.ids, 16).select(w.queries)
    for F, layout in ((16, "soa"), (64, "aos"), (4, "soa"), (32, "lohi")):
        off, ids = select_gpu(rt, w.rects, w.ids, w.queries, fanout=F, layout=layout,
                              mapping="work_queue", unsorted=unsorted)
        assert np.array_equal(off, want[0]), (F, layout)
        if unsorted:
            for i in range(len(off) - 1):
                seg = np.sort(ids[off[i]:off[i + 1]])
                assert np.array_equal(seg, want[1][off[i]:off[i + 1]]), (F, i)
        else:
            assert np.array_equal(ids, want[1]), (F, layout)


def test_work_queue_mapping_small_and_empty(rt):
    for n, q in ((1, 5), (17, 40), (3000, 1)):
        rects = random_case("grid", n, n)
        queries = np.concatenate([random_case("grid", q, n + 3),
                                  np.array([[-INF, -INF, INF, INF]], np.float32)])
        want = oracle.Tree(rects, None, 8).select(queries)
        got = select_gpu(rt, rects, None, queries, fanout=8, mapping="work_queue")
        assert_csr_equal(got, want, f"wq n={n}")
