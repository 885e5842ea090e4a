"""Index persistence: a tree saved with rtree_save and loaded with
rtree_load is the same tree (node by node against the oracle) and answers
selects and joins exactly; damaged or hand-made files are refused."""
import os
import struct

import numpy as np
import pytest

import oracle
from gpu_util import gpu_ready, assert_csr_equal
from paper_2309_16913_gb300 import datagen as dg
from persist_util import HEADER_BYTES, O_NODES, O_VERSION, reseal
from test_oracle import random_case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rt():
    return gpu_ready()


def select_np(t, q):
    res = t.range_select(q)
    try:
        return res.to_numpy()
    finally:
        res.close()


@pytest.mark.parametrize("sort_children", [False, True])
@pytest.mark.parametrize("F,layout", [(4, "soa"), (16, "aos"), (64, "lohi"), (128, "soa")])
def test_roundtrip(rt, tmp_path, F, layout, sort_children):
    rects = random_case("clustered", 20011, 5)
    ids = np.arange(20011, dtype=np.int32) * 3 - 7
    q = random_case("clustered", 500, 6)
    p = tmp_path / "t.rtree"
    with rt.RTree(rects, ids, fanout=F, layout=layout, sort_children=sort_children) as t:
        t.save(str(p))
        info0 = t.info()
    with rt.RTree.load(str(p)) as t2:
        info = t2.info()
        got = t2.export()
        sel = select_np(t2, q)
    for k in ("n", "nodes", "levels", "fanout", "layout", "device_bytes", "sort_children"):
        assert info[k] == info0[k], k
    assert np.array_equal(info["root_mbr"], info0["root_mbr"])
    want = oracle.Tree(rects, ids, F, sort_children=sort_children).export()
    for k in ("level_nodes", "counts", "leaf_ids", "mbrs"):
        assert np.array_equal(got[k], want[k]), k
    assert_csr_equal(sel, oracle.brute_select(rects, q, ids))
    M = info["nodes"]
    assert os.path.getsize(p) == HEADER_BYTES + M * F * 16 + M * 32 + 20011 * 4
    assert [f.name for f in tmp_path.iterdir()] == ["t.rtree"]  # no temporary left behind


def test_loaded_trees_join_and_serve(rt, tmp_path):
    w = dg.workload("join", n=100_000)
    with rt.RTree(w.rects, w.ids, fanout=32, sort_children=True) as a, \
            rt.RTree(w.rects_s, w.ids_s, fanout=32, sort_children=True) as b:
        a.save(str(tmp_path / "a.rtree"))
        b.save(str(tmp_path / "b.rtree"))
    want = oracle.Tree(w.rects, w.ids, 32).join(oracle.Tree(w.rects_s, w.ids_s, 32))
    with rt.RTree.load(str(tmp_path / "a.rtree")) as a, rt.RTree.load(str(tmp_path / "b.rtree")) as b:
        for prune in ("on", "off"):
            res = a.join(b, prune=prune)
            pairs = res.to_numpy()[1]
            res.close()
            assert np.array_equal(pairs, want), prune
        q = random_case("uniform", 200, 9)
        srv = rt.Server(a, workers=2)
        try:
            reqs = [srv.submit(q[i:i + 1]) for i in range(len(q))]
            replies = [srv.wait(r) for r in reqs]
        finally:
            srv.stop()
        want_q = oracle.brute_select(w.rects, q, w.ids)
        for i, (_, ids, _) in enumerate(replies):
            assert np.array_equal(ids, want_q[1][want_q[0][i]:want_q[0][i + 1]]), i


def test_overwrite_and_empty_tree(rt, tmp_path):
    p = tmp_path / "x.rtree"
    r = random_case("uniform", 3000, 1)
    with rt.RTree(r, None, fanout=16) as t:
        t.save(str(p))
    with rt.RTree(np.zeros((0, 4), np.float32), None, fanout=16) as e:
        e.save(str(p))  # replaces the file
    with rt.RTree.load(str(p)) as t2:
        assert t2.info()["n"] == 0
        off, ids = select_np(t2, r[:10])
        assert off.tolist() == [0] * 11 and ids.size == 0


def damaged(rt, path, data):
    path.write_bytes(bytes(data))
    with pytest.raises(rt.RTreeError) as e:
        rt.RTree.load(str(path))
    return e.value


def test_damaged_files_are_refused(rt, tmp_path):
    src = tmp_path / "ok.rtree"
    r = random_case("uniform", 5000, 2)
    with rt.RTree(r, None, fanout=8) as t:
        t.save(str(src))
    good = bytearray(src.read_bytes())
    bad = tmp_path / "bad.rtree"
    # one flipped payload byte: payload checksum
    b = bytearray(good)
    b[HEADER_BYTES + 1000] ^= 0x40
    e = damaged(rt, bad, b)
    assert e.status == rt.RTREE_EINVAL and "payload checksum" in str(e)
    # one flipped header byte: header checksum
    b = bytearray(good)
    b[O_NODES] ^= 1
    e = damaged(rt, bad, b)
    assert e.status == rt.RTREE_EINVAL and "header checksum" in str(e)
    # truncated, and one byte too many
    e = damaged(rt, bad, good[:-4])
    assert e.status == rt.RTREE_EINVAL and "bytes" in str(e)
    e = damaged(rt, bad, good + b"\0")
    assert e.status == rt.RTREE_EINVAL and "bytes" in str(e)
    # another version, sealed
    b = bytearray(good)
    struct.pack_into("<I", b, O_VERSION, 9)
    e = damaged(rt, bad, reseal(b))
    assert e.status == rt.RTREE_EINVAL and "version 9" in str(e)
    # still loads after all that
    with rt.RTree.load(str(src)) as t2:
        assert t2.info()["n"] == 5000


def test_handmade_structure_is_refused(rt, tmp_path):
    """A file whose checksums are right but whose node metadata points
    outside the tree is refused by the device structure check."""
    src = tmp_path / "ok.rtree"
    r = random_case("uniform", 3000, 3)
    with rt.RTree(r, None, fanout=16) as t:
        t.save(str(src))
        info = t.info()
    good = bytearray(src.read_bytes())
    M, F = info["nodes"], info["fanout"]
    meta_off = HEADER_BYTES + M * F * 16
    bad = tmp_path / "bad.rtree"
    cases = [(0, 0, 10**6), (0, 4, 0), (M - 1, 0, 2999), (M - 1, 12, 3001), (1, 0, 0)]
    for node, field, value in cases:
        b = bytearray(good)
        struct.pack_into("<i", b, meta_off + 16 * node + field, value)
        e = damaged(rt, bad, reseal(b))
        assert e.status == rt.RTREE_EINVAL and "tree structure" in str(e), (node, field, value)


def test_loaded_tree_with_two_short_leaves(rt, tmp_path):
    """A loaded tree whose leaf level holds two short leaves: one entry is
    moved across the boundary between the built tree's short leaf and a full
    sibling (same parent), with the leaves' metadata, the entry boxes and the
    parent's child box edited to match.  The traversal cannot derive leaf
    spans from positions here and must read the leaves' metadata; selects
    (small queries and queries that contain whole leaves) equal brute force."""
    F, n = 64, 20000  # 313 leaves, the last packed one holding 32 entries
    rects = random_case("uniform", n, 41)
    ids = np.arange(n, dtype=np.int32) * 5 + 3
    rng = np.random.default_rng(43)
    lo = rng.random((40, 2)).astype(np.float32) * np.float32(0.6)
    big = np.concatenate([lo, lo + np.float32(0.35)], axis=1).astype(np.float32)
    q = np.concatenate([random_case("uniform", 600, 42), big,
                        np.array([[-1, -1, 2, 2]], np.float32)]).astype(np.float32)
    src = tmp_path / "built.rtree"
    with rt.RTree(rects, ids, fanout=F, layout="aos") as t:
        t.save(str(src))
        info, level_nodes = t.info(), t.export()["level_nodes"]
    M = info["nodes"]
    base = np.concatenate([[0], np.cumsum(level_nodes)])
    leaf_base, parent_base = int(base[-2]), int(base[-3])
    buf = bytearray(src.read_bytes())
    mbr_off = HEADER_BYTES
    meta_off = mbr_off + M * F * 16
    nbox_off = meta_off + M * 16
    mbr = np.frombuffer(buf, np.float32, M * F * 4, mbr_off).reshape(M, F, 4).copy()
    meta = np.frombuffer(buf, np.int32, M * 4, meta_off).reshape(M, 4).copy()
    nbox = np.frombuffer(buf, np.float32, M * 4, nbox_off).reshape(M, 4).copy()
    short = [g for g in range(leaf_base, M) if meta[g, 1] != F]
    assert len(short) == 1
    gs = short[0]
    c = int(meta[gs, 1])
    par = [p for p in range(parent_base, leaf_base) if meta[p, 0] <= gs < meta[p, 0] + meta[p, 1]][0]
    empty = mbr[gs, F - 1].copy()

    def grow(box, other):
        return np.array([min(box[0], other[0]), min(box[1], other[1]),
                         max(box[2], other[2]), max(box[3], other[3])], np.float32)
    if gs - 1 >= meta[par, 0]:  # the donor precedes: its last entry opens the short leaf
        d = gs - 1
        moved = mbr[d, F - 1].copy()
        mbr[d, F - 1] = empty
        meta[d, 1] -= 1
        meta[d, 3] -= 1
        mbr[gs, 1:c + 1] = mbr[gs, 0:c].copy()
        mbr[gs, 0] = moved
        meta[gs, 0] -= 1
        meta[gs, 2] -= 1
    else:  # the donor follows: its first entry closes the short leaf
        d = gs + 1
        assert d < meta[par, 0] + meta[par, 1]
        moved = mbr[d, 0].copy()
        mbr[d, 0:F - 1] = mbr[d, 1:F].copy()
        mbr[d, F - 1] = empty
        meta[d, 0] += 1
        meta[d, 2] += 1
        meta[d, 1] -= 1
        mbr[gs, c] = moved
        meta[gs, 3] += 1
    meta[gs, 1] += 1
    slot = gs - meta[par, 0]
    mbr[par, slot] = grow(mbr[par, slot], moved)
    nbox[gs] = grow(nbox[gs], moved)
    buf[mbr_off:meta_off] = mbr.tobytes()
    buf[meta_off:nbox_off] = meta.tobytes()
    buf[nbox_off:nbox_off + M * 16] = nbox.tobytes()
    moved_file = tmp_path / "two_short.rtree"
    moved_file.write_bytes(bytes(reseal(buf)))
    with rt.RTree.load(str(moved_file)) as t2:
        counts = t2.export()["counts"][leaf_base:]
        assert np.count_nonzero(counts != F) == 2
        sel = select_np(t2, q)
    assert_csr_equal(sel, oracle.brute_select(rects, q, ids))
