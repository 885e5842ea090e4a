"""Pins for the CPU oracle (no GPU).

The oracle is checked against things other than itself: hand-written golden
cases (tests/golden/), closed forms, tree invariants, brute-force nested loops
on small inputs, an interval-overlap formulation written with NumPy, and an
independent sort-and-scan join.  ``test_planted_mistakes_are_caught`` compiles
copies of the oracle with one plausible mistake each and checks that these
pins reject every copy.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

import golden_io
import oracle
from paper_2309_16913_gb300 import datagen as dg

INF = np.float32(np.inf)


# ----------------------------------------------------------------- helpers
def split_csr(off, ids):
    return [ids[off[i]:off[i + 1]] for i in range(len(off) - 1)]


def numpy_interval_select(rects, queries, ids):
    """Intervals [a,b] and [c,d] meet iff max(a,c) <= min(b,d); per axis."""
    r = rects.astype(np.float32)
    out = []
    for q in queries.astype(np.float32):
        okx = np.maximum(r[:, 0], q[0]) <= np.minimum(r[:, 2], q[2])
        oky = np.maximum(r[:, 1], q[1]) <= np.minimum(r[:, 3], q[3])
        out.append(np.sort(ids[okx & oky]))
    return out


def sweep_join(r, rid, s, sid):
    """Sort S by xmin; for each r take the prefix with s.xmin <= r.xmax and
    keep those with s.xmax >= r.xmin and overlapping y.  Different algorithm
    from both the nested loops and the tree traversal."""
    order = np.argsort(s[:, 0], kind="stable")
    s_sorted = s[order]
    pairs = []
    for i in range(r.shape[0]):
        k = np.searchsorted(s_sorted[:, 0], r[i, 2], side="right")
        cand = s_sorted[:k]
        ok = (cand[:, 2] >= r[i, 0]) & (cand[:, 1] <= r[i, 3]) & (cand[:, 3] >= r[i, 1])
        for j in order[:k][ok]:
            pairs.append((rid[i], sid[j]))
    if not pairs:
        return np.zeros((0, 2), np.int32)
    p = np.array(pairs, np.int32)
    return p[np.lexsort((p[:, 1], p[:, 0]))]


def grid_rects(rng, n, cells=8):
    """Coordinates on a coarse grid: many exact ties, touching edges, points."""
    a = rng.integers(0, cells, size=(n, 2)).astype(np.float32)
    w = rng.integers(0, 3, size=(n, 2)).astype(np.float32)
    return np.concatenate([a, a + w], axis=1).astype(np.float32) / np.float32(cells)


def random_case(kind, n, seed):
    rng = np.random.default_rng(seed)
    if kind == "uniform":
        return dg.uniform_rects(n, dg.rng_for(seed), 0.0, 0.05)
    if kind == "clustered":
        return dg.clustered_rects(n, dg.rng_for(seed), 4, 0.05, 1e-4, 0.05)
    if kind == "grid":
        return grid_rects(rng, n)
    if kind == "points":
        p = dg.uniform_rects(n, dg.rng_for(seed), 0.0, 0.0)
        return p
    if kind == "dups":
        base = grid_rects(rng, max(1, n // 5))
        return base[rng.integers(0, base.shape[0], size=n)]
    if kind == "negative":
        r = dg.uniform_rects(n, dg.rng_for(seed), 0.0, 0.3)
        return (r - np.float32(0.5)) * np.float32(4.0)
    raise KeyError(kind)


# ------------------------------------------------------ pin suite (reusable)
def check_predicate(lib):
    for a, b, exp in golden_io.predicate_cases():
        ids = np.array([7], np.int32)
        _, got = oracle.brute_select(a[None], b[None], ids, lib=lib)
        assert len(got) == exp, (a, b, exp)
        _, got2 = oracle.brute_select(b[None], a[None], ids, lib=lib)
        assert len(got2) == exp, (b, a, exp, "predicate must be symmetric")
        t = oracle.Tree(a[None], ids, 2, lib=lib)
        _, got3 = t.select(b[None])
        assert len(got3) == exp, (a, b, exp, "tree")
        pj = oracle.brute_join(a[None], b[None], ids, ids, lib=lib)
        assert len(pj) == exp, (a, b, exp, "join")


def check_select_golden(lib):
    rects, ids, queries, expected = golden_io.select_case()
    off, got = oracle.brute_select(rects, queries, ids, lib=lib)
    for g, e in zip(split_csr(off, got), expected):
        assert np.array_equal(g, e), ("brute", g, e)
    for F in (2, 3, 4, 16):
        t = oracle.Tree(rects, ids, F, lib=lib)
        off, got = t.select(queries)
        for g, e in zip(split_csr(off, got), expected):
            assert np.array_equal(g, e), (F, g, e)


def check_join_golden(lib):
    r, rid, s, sid, pairs = golden_io.join_case()
    assert np.array_equal(oracle.brute_join(r, s, rid, sid, lib=lib), pairs)
    for fr, fs in ((2, 2), (2, 3), (3, 2), (4, 4)):
        a = oracle.Tree(r, rid, fr, lib=lib)
        b = oracle.Tree(s, sid, fs, lib=lib)
        assert np.array_equal(a.join(b), pairs), (fr, fs)


def check_str_golden(lib):
    for name in ("str_8points_f2.txt", "str_8boxes_f2.txt"):
        F, rects, ids, exp = golden_io.str_case(name)
        t = oracle.Tree(rects, ids, F, lib=lib)
        got = t.export()
        for k in ("level_nodes", "counts", "leaf_ids"):
            assert np.array_equal(got[k], exp[k]), (name, k, got[k], exp[k])
        assert np.array_equal(got["mbrs"], exp["mbrs"]), name


def check_random_vs_brute(lib, seeds=(0, 1), n=300, q=40):
    for seed in seeds:
        for kind in ("uniform", "grid", "negative"):
            rects = random_case(kind, n, seed)
            ids = np.arange(n, dtype=np.int32)[::-1].copy()
            qs = random_case(kind, q, seed + 100)
            ob, ib = oracle.brute_select(rects, qs, ids, lib=lib)
            for F in (2, 3, 16):
                ot, it = oracle.Tree(rects, ids, F, lib=lib).select(qs)
                assert np.array_equal(ob, ot) and np.array_equal(ib, it), (kind, F, seed)
            # join with unequal heights and fanouts
            s = random_case(kind, n // 3, seed + 7)
            sid = np.arange(s.shape[0], dtype=np.int32) + 1000
            pb = oracle.brute_join(rects, s, ids, sid, lib=lib)
            for fr, fs in ((2, 16), (16, 2), (3, 4)):
                pt = oracle.Tree(rects, ids, fr, lib=lib).join(oracle.Tree(s, sid, fs, lib=lib))
                assert np.array_equal(pb, pt), (kind, fr, fs, seed)


def check_threaded_vs_brute(lib):
    """The all-cores forms (orc_select_mt, orc_join_mt) equal brute force,
    with more threads than queries, uneven chunks and unequal tree heights."""
    for kind, seed in (("uniform", 40), ("grid", 41), ("clustered", 42)):
        rects = random_case(kind, 900, seed)
        ids = np.random.default_rng(seed).permutation(900).astype(np.int32) - np.int32(300)
        qs = random_case(kind, 37, seed + 1)
        ob, ib = oracle.brute_select(rects, qs, ids, lib=lib)
        t = oracle.Tree(rects, ids, 4, lib=lib)
        for threads in (2, 7, 64):
            ot, it = t.select(qs, threads=threads)
            assert np.array_equal(ob, ot) and np.array_equal(ib, it), (kind, threads)
        s = random_case(kind, 700, seed + 2)
        sid = np.arange(700, dtype=np.int32) * 2 - 5
        pb = oracle.brute_join(rects, s, ids, sid, lib=lib)
        for fr, fs, threads in ((4, 16, 3), (2, 32, 8), (16, 2, 5), (64, 64, 4)):
            pt = oracle.Tree(rects, ids, fr, lib=lib).join(oracle.Tree(s, sid, fs, lib=lib), threads=threads)
            assert np.array_equal(pt, pb), (kind, fr, fs, threads)


def sorted_export_reference(e):
    """From the export of a tree, the export of the same tree with every
    node's entries stably reordered by ascending lx (written independently of
    the oracle: NumPy over the exported arrays)."""
    ln, counts, mbrs, leaf_ids = e["level_nodes"], e["counts"], e["mbrs"], e["leaf_ids"]
    L = len(ln)
    bases = np.concatenate([[0], np.cumsum(ln)]).astype(np.int64)
    # children of each internal node / ids of each leaf, in export order
    kids, leaf_of, nxt = {}, {}, {}
    for lv in range(L):
        ptr = 0
        for k in range(ln[lv]):
            g = bases[lv] + k
            c = counts[g]
            if lv < L - 1:
                kids[g] = np.arange(bases[lv + 1] + ptr, bases[lv + 1] + ptr + c)
            else:
                leaf_of[g] = leaf_ids[ptr:ptr + c]
            ptr += c
    out_counts, out_mbrs, out_ids = [], [], []
    level = [0] if L else []
    for lv in range(L):
        nxt = []
        for g in level:
            c = counts[g]
            perm = np.argsort(mbrs[g, :c, 0], kind="stable")
            m = mbrs[g].copy()
            m[:c] = mbrs[g, :c][perm]
            out_counts.append(c)
            out_mbrs.append(m)
            if lv < L - 1:
                nxt.extend(kids[g][perm].tolist())
            else:
                out_ids.append(leaf_of[g][perm])
        level = nxt
    F = mbrs.shape[1]
    return {"level_nodes": ln.copy(), "counts": np.array(out_counts, np.int32),
            "mbrs": np.array(out_mbrs, np.float32).reshape(-1, F, 4),
            "leaf_ids": np.concatenate(out_ids) if out_ids else leaf_ids.copy()}


def check_sorted_build(lib):
    for kind, n in (("grid", 257), ("dups", 300), ("uniform", 500), ("negative", 130)):
        rects = random_case(kind, n, 5)
        ids = np.arange(n, dtype=np.int32)[::-1].copy()
        for F in (2, 3, 4, 16):
            plain = oracle.Tree(rects, ids, F, lib=lib).export()
            got = oracle.Tree(rects, ids, F, lib=lib, sort_children=True).export()
            want = sorted_export_reference(plain)
            for k in ("level_nodes", "counts", "leaf_ids", "mbrs"):
                assert np.array_equal(got[k], want[k]), (kind, F, k)


def check_pruned_join(lib):
    saved = 0
    for seed, kind in ((3, "grid"), (4, "uniform"), (5, "negative"), (6, "dups"), (7, "points")):
        r = random_case(kind, 240, seed)
        s = random_case(kind, 90, seed + 50)
        rid = np.arange(240, dtype=np.int32)
        sid = np.arange(90, dtype=np.int32) + 500
        want = oracle.brute_join(r, s, rid, sid, lib=lib)
        for fr, fs in ((2, 2), (4, 4), (3, 16), (16, 2)):
            a = oracle.Tree(r, rid, fr, lib=lib, sort_children=True)
            b = oracle.Tree(s, sid, fs, lib=lib, sort_children=True)
            got, tests = a.join_pruned(b)
            assert np.array_equal(got, want), (kind, fr, fs)
            plain = oracle.Tree(r, rid, fr, lib=lib).join_tests(oracle.Tree(s, sid, fs, lib=lib))
            assert tests <= plain, (kind, fr, fs, tests, plain)
            saved += plain - tests
    assert saved > 0
    with pytest.raises(ValueError):  # unsorted trees are refused
        oracle.Tree(r, rid, 4, lib=lib).join_pruned(oracle.Tree(s, sid, 4, lib=lib))


def check_o5(lib):
    g = golden_io.o5_case()
    flip, tg, tf = oracle.o5_bounds(g["OUT_HX"], g["IN_LX"], lib=lib)
    assert np.array_equal(tg[0], g["G1"]) and np.array_equal(tg[1], g["G2"])
    assert np.array_equal(tf[0], g["F1"])
    assert np.array_equal((g["OUT_HX"] >= g["IN_LX"][2]).astype(np.int32), g["MASK1"])
    assert np.array_equal(flip, g["FLIP"]) and len(tg) == 3
    # brute force: the bound is the number of inner lx <= out.hx
    rng = np.random.default_rng(9)
    for n_in in range(1, 18):
        for _ in range(6):
            in_lx = np.sort(rng.integers(0, 6, n_in).astype(np.float32))
            out_hx = np.concatenate([rng.integers(-1, 7, 12).astype(np.float32), in_lx,
                                     np.array([-INF, INF], np.float32)])
            flip, tg, _ = oracle.o5_bounds(out_hx, in_lx, lib=lib)
            want = np.searchsorted(in_lx, out_hx, side="right").astype(np.int32)
            assert np.array_equal(flip, want), (in_lx, out_hx, flip, want)
            assert len(tg) == int(np.ceil(np.log2(n_in))) + 1


PIN_SUITE = (check_predicate, check_select_golden, check_join_golden, check_str_golden,
             check_random_vs_brute, check_sorted_build, check_pruned_join, check_o5,
             check_threaded_vs_brute)


# -------------------------------------------------------------- the pins
def test_predicate_golden():
    check_predicate(oracle.load())


def test_select_golden():
    check_select_golden(oracle.load())


def test_join_golden():
    check_join_golden(oracle.load())


def test_str_golden():
    check_str_golden(oracle.load())


def test_sorted_children_build():
    check_sorted_build(oracle.load())


def test_sorted_children_entries_ascend():
    rects = random_case("clustered", 4000, 12)
    e = oracle.Tree(rects, None, 16, sort_children=True).export()
    for g, c in enumerate(e["counts"]):
        assert np.all(np.diff(e["mbrs"][g, :c, 0]) >= 0)


def test_threaded_forms_match_brute():
    check_threaded_vs_brute(oracle.load())


def test_pruned_join_matches_brute():
    check_pruned_join(oracle.load())


def test_o5_worked_example_and_brute_force():
    check_o5(oracle.load())


def test_pruned_join_saves_tests_on_workload_shapes():
    j = dg.workload("join", n=20000)
    a = oracle.Tree(j.rects, j.ids, 32, sort_children=True)
    b = oracle.Tree(j.rects_s, j.ids_s, 32, sort_children=True)
    got, tests = a.join_pruned(b)
    assert np.array_equal(got, oracle.Tree(j.rects, j.ids, 32).join(oracle.Tree(j.rects_s, j.ids_s, 32)))
    plain = oracle.Tree(j.rects, j.ids, 32).join_tests(oracle.Tree(j.rects_s, j.ids_s, 32))
    assert tests < plain


@pytest.mark.parametrize("kind", ["uniform", "clustered", "grid", "points", "dups", "negative"])
@pytest.mark.parametrize("F", [2, 3, 4, 16, 64])
def test_select_matches_brute_force(kind, F):
    for seed in range(3):
        n = [1, 7, 64, 65, 500, 2000][(seed * 2 + F) % 6]
        rects = random_case(kind, n, seed)
        ids = np.random.default_rng(seed).permutation(n).astype(np.int32) - np.int32(n // 2)
        qs = random_case(kind, 60, seed + 11)
        ob, ib = oracle.brute_select(rects, qs, ids)
        ot, it = oracle.Tree(rects, ids, F).select(qs)
        assert np.array_equal(ob, ot)
        assert np.array_equal(ib, it)


@pytest.mark.parametrize("kind", ["uniform", "grid", "negative", "points"])
def test_brute_matches_interval_form(kind):
    rects = random_case(kind, 1500, 5)
    ids = np.arange(1500, dtype=np.int32)
    qs = random_case(kind, 80, 6)
    off, got = oracle.brute_select(rects, qs, ids)
    for g, e in zip(split_csr(off, got), numpy_interval_select(rects, qs, ids)):
        assert np.array_equal(g, e)


@pytest.mark.parametrize("kind", ["uniform", "clustered", "grid", "dups"])
def test_join_matches_brute_and_sweep(kind):
    r = random_case(kind, 700, 21)
    s = random_case(kind, 500, 22)
    rid = np.arange(700, dtype=np.int32)
    sid = np.arange(500, dtype=np.int32) * 3 - 7
    pb = oracle.brute_join(r, s, rid, sid)
    assert np.array_equal(pb, sweep_join(r, rid, s, sid))
    for fr, fs in ((2, 2), (4, 16), (16, 4), (32, 32), (64, 3)):
        pt = oracle.Tree(r, rid, fr).join(oracle.Tree(s, sid, fs))
        assert np.array_equal(pt, pb), (fr, fs)


def test_join_swap_symmetry():
    r = random_case("grid", 400, 31)
    s = random_case("grid", 300, 32)
    rid = np.arange(400, dtype=np.int32)
    sid = np.arange(300, dtype=np.int32)
    a = oracle.Tree(r, rid, 4).join(oracle.Tree(s, sid, 8))
    b = oracle.Tree(s, sid, 8).join(oracle.Tree(r, rid, 4))
    bt = b[:, ::-1]
    bt = bt[np.lexsort((bt[:, 1], bt[:, 0]))]
    assert np.array_equal(a, bt)


def test_self_join_contains_diagonal():
    r = random_case("uniform", 300, 41)
    rid = np.arange(300, dtype=np.int32)
    p = oracle.Tree(r, rid, 4).join(oracle.Tree(r, rid, 5))
    diag = p[p[:, 0] == p[:, 1]]
    assert np.array_equal(diag[:, 0], rid)  # every valid rectangle meets itself


# ------------------------------------------------------------ closed forms
def test_closed_forms():
    rects = random_case("uniform", 1000, 51)
    ids = np.arange(1000, dtype=np.int32) * 2
    t = oracle.Tree(rects, ids, 16)
    everything = np.array([[-INF, -INF, INF, INF]], np.float32)
    off, got = t.select(everything)
    assert np.array_equal(got, np.sort(ids))
    lo, hi = rects[:, :2].min(0), rects[:, 2:].max(0)
    outside = np.array([[hi[0] + 1, hi[1] + 1, hi[0] + 2, hi[1] + 2],
                        [lo[0] - 2, lo[1] - 2, np.nextafter(lo[0], -INF), lo[1]]], np.float32)
    off, got = t.select(outside)
    assert off.tolist() == [0, 0, 0] and got.size == 0
    off, got = t.select(np.zeros((0, 4), np.float32))
    assert off.tolist() == [0] and got.size == 0


def test_empty_tree():
    t = oracle.Tree(np.zeros((0, 4), np.float32), np.zeros(0, np.int32), 16)
    assert t.levels == 0 and t.n_nodes == 0
    off, got = t.select(np.array([[-INF, -INF, INF, INF]], np.float32))
    assert off.tolist() == [0, 0]
    other = oracle.Tree(random_case("uniform", 50, 1), None, 4)
    assert t.join(other).shape == (0, 2) and other.join(t).shape == (0, 2)


@pytest.mark.parametrize("F", [2, 4, 16])
def test_small_sizes(F):
    for n in (1, F - 1, F, F + 1, F * F, F * F + 1):
        if n < 1:
            continue
        rects = random_case("grid", n, n)
        ids = np.arange(n, dtype=np.int32)
        t = oracle.Tree(rects, ids, F)
        levels, m = 1, n
        while (m + F - 1) // F > 1:
            m = (m + F - 1) // F
            levels += 1
        assert t.levels == levels, (n, F)
        everything = np.array([[-INF, -INF, INF, INF]], np.float32)
        assert np.array_equal(t.select(everything)[1], ids)


# -------------------------------------------------------------- invariants
@pytest.mark.parametrize("F", [2, 3, 16, 64])
def test_tree_invariants(F):
    rects = random_case("clustered", 3000, 61)
    ids = np.arange(3000, dtype=np.int32)
    t = oracle.Tree(rects, ids, F)
    e = t.export()
    ln, counts, mbrs, leaf_ids = e["level_nodes"], e["counts"], e["mbrs"], e["leaf_ids"]
    # every id in exactly one leaf
    assert np.array_equal(np.sort(leaf_ids), ids)
    # per level: all nodes full except at most one
    g = 0
    bases = []
    for L in ln:
        c = counts[g:g + L]
        bases.append(g)
        assert (c == F).sum() >= L - 1 and c.min() >= 1
        g += L
    # a parent's entry MBR is the exact min/max over the child's entries
    for lv in range(len(ln) - 1):
        child = bases[lv + 1]
        for k in range(ln[lv]):
            node = bases[lv] + k
            for j in range(counts[node]):
                cm = mbrs[child, :counts[child]]
                want = [cm[:, 0].min(), cm[:, 1].min(), cm[:, 2].max(), cm[:, 3].max()]
                assert np.array_equal(mbrs[node, j], np.array(want, np.float32))
                child += 1
        assert child == bases[lv + 1] + ln[lv + 1]
    # leaf entries are the data rectangles, in leaf_ids order
    leaf0 = bases[-1]
    flat = np.concatenate([mbrs[leaf0 + k, :counts[leaf0 + k]] for k in range(ln[-1])])
    assert np.array_equal(flat, rects[leaf_ids])
    # unused slots hold the empty box
    for node in range(counts.size):
        pad = mbrs[node, counts[node]:]
        assert np.all(pad == np.array([INF, INF, -INF, -INF], np.float32))


def test_hit_totals_match_brute():
    w = dg.workload("plain", n=20000, q=300)
    ob, _ = oracle.brute_select(w.rects, w.queries, w.ids)
    ot, _ = oracle.Tree(w.rects, w.ids, 16).select(w.queries)
    assert ob[-1] == ot[-1] and ob[-1] > 100


# ------------------------------------------------------ planted mistakes
MUTANTS = [
    ("touching edges dropped", "return a.lx <= b.hx && b.lx <= a.hx", "return a.lx < b.hx && b.lx <= a.hx"),
    ("y terms dropped", "&& a.ly <= b.hy && b.ly <= a.hy;\n}", ";\n}"),
    ("wrong operand", "&& b.ly <= a.hy;\n}", "&& b.ly <= a.ly;\n}"),
    ("tree select operand swapped", "q.lx <= c.hx && c.ly", "q.hx <= c.hx && c.ly"),
    ("tree select y dropped", "c.ly <= q.hy && q.ly <= c.hy", "1"),
    ("join pair transposed", "emit_pair(out, a->id[i], b->id[j])", "emit_pair(out, b->id[j], a->id[i])"),
    ("unequal heights: wrong child", "join_rec(a->child[i], a->mbr[i], b, bmb, out)",
     "join_rec(a->child[0], a->mbr[0], b, bmb, out)"),
    ("STR slab index", "slab[t[r].idx] = r / cap;", "slab[t[r].idx] = r % cap;"),
    ("STR centre key", "float k = lo + hi;", "float k = lo;"),
    ("STR tie order", "return (a->idx > b->idx) - (a->idx < b->idx);", "return (a->idx < b->idx) - (a->idx > b->idx);"),
    ("leaf packing off by one", "int64_t lo = k * fanout, hi", "int64_t lo = k * fanout + (k > 0), hi"),
    ("child sort unstable on ties", "while (k >= 0 && nd->mbr[k].lx > b.lx)",
     "while (k >= 0 && nd->mbr[k].lx >= b.lx)"),
    ("child sort moves MBRs only", "nd->child[k + 1] = nd->child[k];", "nd->child[k + 1] = nd->child[k + 1];"),
    ("O3 on the wrong key", "if (a->mbr[i].lx <= b->mbr[j].hx)", "if (a->mbr[i].hx <= b->mbr[j].lx)"),
    ("O4 drops touching pairs", "if (b->mbr[j].lx > a->mbr[i].hx) /* O4 */",
     "if (b->mbr[j].lx >= a->mbr[i].hx) /* O4 */"),
    ("O5 moves the wrong way", "g[i] = pass ? g[i] + step : g[i] - step;",
     "g[i] = pass ? g[i] - step : g[i] + step;"),
    ("O5 one round short", "int rounds = logp + 1;", "int rounds = logp;"),
    ("threaded select drops each chunk's last query", "jobs[k].q1 = Q * (k + 1) / threads;",
     "jobs[k].q1 = Q * (k + 1) / threads - (k + 1 < threads);"),
    ("threaded join expands the wrong child", "jcall d = {a->child[i], b, a->mbr[i], c.bmb};",
     "jcall d = {a->child[0], b, a->mbr[0], c.bmb};"),
    ("threaded join expands one level short", "jcall d = {a, b->child[j], c.amb, b->mbr[j]};",
     "jcall d = {a, b, c.amb, c.bmb};"),
]


@pytest.mark.skipif(shutil.which("gcc") is None, reason="gcc not available")
def test_planted_mistakes_are_caught(tmp_path):
    with open(os.path.join(os.path.dirname(oracle.__file__), "rtree_oracle.c")) as f:
        src = f.read()
    for name, old, new in MUTANTS:
        assert old in src, f"mutation anchor missing: {name}"
        path = tmp_path / f"m{abs(hash(name))}.c"
        path.write_text(src.replace(old, new, 1))
        so = str(path) + ".so"
        subprocess.run(["gcc", *oracle.CFLAGS, "-o", so, str(path), "-lm", "-lpthread"], check=True)
        lib = oracle.load(so)
        caught = False
        for check in PIN_SUITE:
            try:
                check(lib)
            except (AssertionError, MemoryError, IndexError, ValueError):
                caught = True
                break
        assert caught, f"planted mistake survived the pins: {name}"
