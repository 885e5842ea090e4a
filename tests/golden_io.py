"""Parsers for the hand-written fixtures under tests/golden/ (test helper)."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _num(tok: str) -> float:
    t = tok.strip()
    if "0x" in t.lower():
        return float.fromhex(t)
    return float(t)


def _lines(name):
    with open(os.path.join(GOLDEN, name)) as f:
        for raw in f:
            line = raw.split("#", 1)[0].strip()
            if line:
                yield line


def predicate_cases():
    """[(a[4], b[4], expected)] with values checked to be exact in float32."""
    out = []
    for line in _lines("predicate_cases.txt"):
        toks = line.split()
        assert len(toks) == 9, line
        vals = [_num(t) for t in toks[:8]]
        f32 = np.array(vals, dtype=np.float32)
        assert all((float(x) == v) or (np.isnan(v) and np.isnan(x)) for x, v in zip(f32, vals)), line
        # -0.0 must survive the cast too
        assert all(np.signbit(x) == np.signbit(v) for x, v in zip(f32, vals)), line
        out.append((f32[:4].copy(), f32[4:].copy(), int(toks[8])))
    return out


def select_case(name="select_small.txt"):
    rects, ids, queries, expected = [], [], [], []
    for line in _lines(name):
        if line.startswith("R "):
            t = line.split()
            ids.append(int(t[1]))
            rects.append([_num(x) for x in t[2:6]])
        elif line.startswith("Q "):
            lhs, rhs = line[2:].split(":")
            queries.append([_num(x) for x in lhs.split()])
            expected.append(np.array([int(x) for x in rhs.split()], dtype=np.int32))
    return (np.array(rects, dtype=np.float32), np.array(ids, dtype=np.int32),
            np.array(queries, dtype=np.float32).reshape(-1, 4), expected)


def join_case(name="join_small.txt"):
    r, rid, s, sid, pairs = [], [], [], [], []
    for line in _lines(name):
        t = line.split()
        if t[0] == "R":
            rid.append(int(t[1])); r.append([_num(x) for x in t[2:6]])
        elif t[0] == "S":
            sid.append(int(t[1])); s.append([_num(x) for x in t[2:6]])
        elif t[0] == "P":
            pairs.append([int(t[1]), int(t[2])])
    return (np.array(r, np.float32), np.array(rid, np.int32), np.array(s, np.float32),
            np.array(sid, np.int32), np.array(pairs, np.int32).reshape(-1, 2))


def str_case(name):
    """Returns (fanout, rects, ids, expected export dict); coordinates in 1/16."""
    F, rects, ids, exp = None, [], [], {}
    entries = {}
    for line in _lines(name):
        t = line.split()
        if t[0] == "F":
            F = int(t[1])
        elif t[0] == "P":  # point id x y
            ids.append(int(t[1])); x, y = int(t[2]) / 16, int(t[3]) / 16
            rects.append([x, y, x, y])
        elif t[0] == "B":
            ids.append(int(t[1])); rects.append([int(v) / 16 for v in t[2:6]])
        elif t[0] == "LEVEL_NODES":
            exp["level_nodes"] = np.array([int(v) for v in t[1:]], np.int64)
        elif t[0] == "COUNTS":
            exp["counts"] = np.array([int(v) for v in t[1:]], np.int32)
        elif t[0] == "LEAF_IDS":
            exp["leaf_ids"] = np.array([int(v) for v in t[1:]], np.int32)
        elif t[0] == "E":
            entries[(int(t[1]), int(t[2]))] = [int(v) / 16 for v in t[3:7]]
    M = int(exp["level_nodes"].sum())
    mbrs = np.empty((M, F, 4), np.float32)
    mbrs[:] = np.array([np.inf, np.inf, -np.inf, -np.inf], np.float32)
    for (g, e), v in entries.items():
        mbrs[g, e] = v
    exp["mbrs"] = mbrs
    return F, np.array(rects, np.float32), np.array(ids, np.int32), exp


def o5_case(name="o5_example.txt"):
    """{key: np.ndarray} for the O5 worked example."""
    out = {}
    for line in _lines(name):
        t = line.split()
        dt = np.float32 if t[0] in ("IN_LX", "OUT_HX") else np.int32
        out[t[0]] = np.array([_num(x) for x in t[1:]], dtype=dt)
    return out
