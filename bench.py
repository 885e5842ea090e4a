#!/usr/bin/env python3
"""Benchmark: batched R-tree range select on GB300 (plus join and oracle baselines).

One step = one pass of the whole hot path over one batch: STR bulk load of
10M rectangles (80% in 64 Gaussian clusters, 20% uniform; sides log-uniform
in [1e-5, 1e-3]) followed by a sorted range select of 1M square queries
whose selectivity is log-uniform in [1e-6, 1e-3].  ``value`` = queries/s
over the whole job (all ranks), inputs resident in HBM.  The node fanout and
layout are picked once before the warm-up by timing one step of each
candidate.  Under torchrun every rank builds and queries its own instance
(weak scaling; no collective on the data path).

``--impl reference`` times the CPU oracle (plain scalar C, on every host
core, one POSIX thread per core over query chunks) on the same workload
instead: the tree is built once at fanout 64 (the paper's default), each
step selects a fixed subset of 65536 queries, and ``value`` extrapolates to
the full batch (1M / (build + per-query time * 1M)).

Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import platform
import re
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "range queries/s at 10M rects"
UNIT = "queries/s"
WORKLOAD = "scaled"
CPU_SAMPLE_QUERIES = 65536   # fixed subset of the batch the oracle is timed on
REF_FANOUT = 64               # the paper's default fanout (Section 5)


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--fanout", type=int, default=0, help="0: pick by timing 16/32/64")
    ap.add_argument("--layout", choices=["soa", "aos", "lohi", "auto"], default="auto")
    ap.add_argument("--mapping", choices=["warp_per_query", "work_queue", "auto"], default="auto")
    ap.add_argument("--rects", "--n", dest="n", type=int, default=None,
                    help="override rectangles (testing only)")
    ap.add_argument("--queries", "--q", dest="q", type=int, default=None,
                    help="override queries (testing only)")
    ap.add_argument("--sel", type=float, nargs=2, default=None, metavar=("LO", "HI"),
                    help="override the query selectivity range (profiling a smaller index "
                         "with the full-size hit-count mix)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-join", action="store_true")
    ap.add_argument("--no-order", action="store_true")
    ap.add_argument("--no-persist", action="store_true")
    ap.add_argument("--order", choices=["auto", "input", "hilbert"], default="auto",
                    help="traversal order of the query batch (auto: the autotuner picks)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-tune", action="store_true",
                    help="skip the autotuner; needs --fanout, --layout, --mapping and --order set")
    ap.add_argument("--no-uneven", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--serve-n", type=int, default=50_000_000, help="index size of the serving run")
    ap.add_argument("--serve-requests", type=int, default=20000)
    return ap.parse_args()


# ------------------------------------------------------------------ ranks
def dist_init(backend):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group(backend=backend)
    return rank, local, world


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int, device=None) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ----------------------------------------------------------------- clocks
class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        # the raw samples stay next to the run (RTREE_CLOCKS_DIR, else the temp dir)
        out_dir = os.environ.get("RTREE_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(out_dir, f"clocks_rank{gpu_index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names[1:], parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        under_load = [v for v in sm if v > 0.5 * max(sm)] or sm
        return {"sm_mhz": float(np.median(under_load)), "sm_max_mhz": max(mx),
                "samples": len(sm), "reasons": sorted(reasons)}


# ---------------------------------------------------------------- helpers
def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def strip_comments(text: str) -> str:
    """C/C++ source without its comments and blank lines (string and
    character literals kept): edits to comments leave a kernel's stamp alone."""
    out, i, n = [], 0, len(text)
    while i < n:
        c = text[i]
        if c in "\"'":
            j = i + 1
            while j < n and text[j] != c:
                j += 2 if text[j] == "\\" else 1
            out.append(text[i:j + 1])
            i = j + 1
        elif text.startswith("//", i):
            while i < n and text[i] != "\n":
                i += 1
        elif text.startswith("/*", i):
            j = text.find("*/", i + 2)
            i = n if j < 0 else j + 2
        else:
            out.append(c)
            i += 1
    return "\n".join(line.rstrip() for line in "".join(out).splitlines() if line.strip())


def source_sha(files, read=None):
    """Stamp of a kernel's source files (comments removed)."""
    h = hashlib.sha256()
    for f in files:
        if read is None:
            with open(os.path.join(ROOT, "paper_2309_16913_gb300", "csrc", f), encoding="utf-8") as fh:
                text = fh.read()
        else:
            text = read(f)
        h.update(strip_comments(text).encode())
    return h.hexdigest()[:16]


KERNEL_SOURCES = {"select_count": ["select.cu", "internal.cuh"], "select_bound": ["select.cu", "internal.cuh"],
                  "select_desc": ["select.cu", "internal.cuh"],
                  "join_scatter": ["join.cu", "internal.cuh"],
                  "join_pruned_count": ["join.cu", "internal.cuh"],
                  "join_pruned_scatter": ["join.cu", "internal.cuh"],
                  "select_scatter": ["select.cu", "internal.cuh"],
                  "sort_warp": ["segsort.cu"], "sort_cta": ["segsort.cu"], "sort_gather": ["segsort.cu"],
                  "sort_msd": ["segsort.cu"], "sort_bucket": ["segsort.cu"], "sort_all": ["segsort.cu"],
                  "scatter": ["radix_sort.cu"], "join_count": ["join.cu", "internal.cuh"]}


def config_matches(kv, fanout, layout=None):
    """A summary line taken at one fanout (and node layout) serves only a run
    in that configuration."""
    if fanout is not None and "fanout" in kv and int(kv["fanout"]) != fanout:
        return False
    return layout is None or "layout" not in kv or kv["layout"] == layout


def ncu_traffic(kernel: str, fanout=None, layout=None):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current source of that kernel (and in this configuration); else
    None."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    if not os.path.exists(path):
        return None, None
    want = source_sha(KERNEL_SOURCES.get(kernel, []))
    note = None
    for line in open(path):
        kv = dict(re.findall(r"(\w+)=(\S+)", line))
        if kv.get("kernel") == kernel and kv.get("workload") == WORKLOAD:
            if not config_matches(kv, fanout, layout):
                note = note or "no capture in this configuration"
            elif kv.get("source_sha") == want:
                return float(kv["bytes_per_step"]), kv.get("note")
            else:
                note = "kernel changed since the ncu capture"
    return None, note


def algorithmic_bytes(stats, F, Q, seg_sizes):
    """Bytes each kernel must move in one step (all its launches), from the
    traversal counters and the per-query result sizes.

    Node visit: F entry MBRs (16 B each, unused slots included) + 16 B of node
    metadata.  Whole subtree: 16 B metadata read + 8 B (lo, hi) written.  Leaf
    hit: 4 B id read + 4 B written.  Sorting an id: 4 B gathered + 4 B written
    (segments over 40960 ids take the MSD path, which adds three reads and one
    write for the split).
    The bound pass visits the internal nodes only; the descriptor pass after
    it also writes two exact counts per query.
    """
    node = F * 16 + 16
    nodes = stats["nodes_visited"]
    whole = stats["whole_children"]
    hits = stats["ids"]
    leaf_hits = hits - stats["ids_from_whole"]
    traverse = nodes * node + whole * 16
    internal = (nodes - stats["leaves_visited"]) * node + whole * 16
    seg = np.asarray(seg_sizes, dtype=np.int64)
    in_range = lambda lo, hi: int(seg[(seg >= lo) & (seg <= hi)].sum())
    warp_ids, cta_ids, large_ids = in_range(2, 256), in_range(257, 40960), in_range(40961, 1 << 62)
    return {
        "select_count": float(traverse + Q * (16 + 3 * 4)),
        "select_bound": float(internal + Q * (16 + 3 * 4)),
        "select_desc": float(traverse + Q * (16 + 32 + 8) + leaf_hits * 8 + whole * 8),
        "select_scatter": float(traverse + Q * (16 + 16) + hits * 8),
        "sort_warp": float(warp_ids * 8),
        "sort_cta": float(cta_ids * 8),
        "sort_gather": float(large_ids * 8),
        "sort_msd": float(large_ids * 16),
        "sort_bucket": float(large_ids * 8),
        # the whole segmented sort as one span (its class kernels run side by side)
        "sort_all": float((warp_ids + cta_ids + large_ids) * 8 + large_ids * 24),
    }


def join_roofline(st, Fr, Fs, kern, hbm, peak_kind, clk):
    """Roofline of the join's traversal kernels (count and scatter passes of
    every level, one launch each), from the traversal counters.

    Bytes: a node pair tested at equal heights reads both nodes' entries
    ((Fr + Fs) * 16 B) and two node records (32 B); a one-sided descent
    reads the taller node's entries and the other node's box.  The scatter
    pass also writes 8 B per child pair or result pair it emits.  Tests: a
    node pair at equal heights takes Fr * Fs predicate tests, a one-sided
    descent F tests.  The issue-slot side needs instruction counts from ncu
    (profiles/ncu_metrics.txt) and is reported when they were taken on the
    current source."""
    eq = st["pairs_equal_internal"] + st["pairs_leaf"]
    node_bytes = eq * ((Fr + Fs) * 16 + 32) + st["pairs_r_descends"] * (Fr * 16 + 32) + \
        st["pairs_s_descends"] * (Fs * 16 + 32)
    visited = eq + st["pairs_r_descends"] + st["pairs_s_descends"]
    emitted = (visited - 1) + st["pairs_found"]
    tests = eq * Fr * Fs + st["pairs_r_descends"] * Fr + st["pairs_s_descends"] * Fs
    names = sorted(kern)
    ms = sum(v[1] for v in kern.values())
    if ms <= 0:
        return None
    algo = 2 * node_bytes + 8 * emitted
    achieved = algo / (ms / 1e3) / 1e9
    out = {"kernels": names, "bound": "hbm", "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
           "frac": round(achieved / hbm, 4), "peak_kind": peak_kind, "ms_per_step": round(ms, 4),
           "algorithmic_bytes_per_step": int(algo), "node_pairs": int(visited),
           "predicate_tests_per_s": round(2 * tests / (ms / 1e3), 1)}
    issue = issue_fraction([n for n in names], visited, ms, clk, fanout=Fr)
    if issue:
        out["issue"] = issue
    return out


def node_test_roofline(kern, algo, stats, steps, hbm, peak_kind, clk, F, layout):
    """Per node-test kernel: the logical rate (algorithmic bytes, upper tree
    levels included though L2 serves them), the DRAM rate from ncu's DRAM
    bytes per node visit on the profile case scaled to this run's visits,
    and the issue-slot use; `bound` names the larger fraction."""
    internal = stats["nodes_visited"] - stats["leaves_visited"]
    units = {"select_bound": internal, "select_desc": stats["nodes_visited"],
             "select_count": stats["nodes_visited"]}
    out = {}
    for k in ("select_bound", "select_count", "select_desc"):
        if k not in kern or kern[k][0] == 0 or k not in algo:
            continue
        ms = kern[k][1] / steps
        logical = algo[k] / (ms / 1e3) / 1e9
        e = {"ms_per_step": round(ms, 4), "node_visits": int(units[k]),
             "logical_gbs": round(logical, 1), "logical_frac": round(logical / hbm, 4)}
        m = ncu_metrics(k, F, layout)
        if m is not None and "dram_bytes_per_unit" in m:
            dram = float(m["dram_bytes_per_unit"]) * units[k] / (ms / 1e3) / 1e9
            e["dram_gbs"] = round(dram, 1)
            e["dram_frac"] = round(dram / hbm, 4)
        iss = issue_fraction([k], units[k], ms, clk, fanout=F, layout=layout)
        if iss:
            e["issue"] = iss
        fr = {"hbm": e.get("dram_frac"), "issue": (iss or {}).get("frac")}
        fr = {a: b for a, b in fr.items() if b is not None}
        if fr:
            e["bound"] = max(fr, key=fr.get)
            e["frac"] = fr[e["bound"]]
        out[k] = e
    if not out:
        return None
    out["peak"] = hbm
    out["peak_kind"] = peak_kind
    out["note"] = ("dram from ncu DRAM bytes per node visit on the profile case (profiles/ncu_metrics.txt) "
                   "scaled to this run's visits; issue = warp instructions per visit x visits over the "
                   "kernel's issue slots; logical counts every node byte, most served by L2")
    return out


def ncu_metrics(kernel: str, fanout=None, layout=None):
    """Instruction and DRAM counters of `kernel` from the committed ncu
    summary, if taken on the current source of that kernel (and in this
    configuration); else None."""
    path = os.path.join(ROOT, "profiles", "ncu_metrics.txt")
    if not os.path.exists(path):
        return None
    want = source_sha(KERNEL_SOURCES.get(kernel, []))
    for line in open(path):
        kv = dict(re.findall(r"(\w+)=(\S+)", line))
        if kv.get("kernel") == kernel and config_matches(kv, fanout, layout) and kv.get("source_sha") == want:
            return kv
    return None


def issue_fraction(kernels, units, ms, clk, sms=152, schedulers=4, fanout=None, layout=None):
    """Issue-slot use of kernels that process `units` work units in `ms`:
    instructions per unit (ncu, profile case) * units / (issue slots per
    second * time).  Issue slots per second = SMs * 4 schedulers * the
    median SM clock sampled during the timed region."""
    inst_per_unit = 0.0
    for k in kernels:
        m = ncu_metrics(k, fanout, layout)
        if m is None or "inst_per_unit" not in m:
            return None
        inst_per_unit += float(m["inst_per_unit"])
    mhz = (clk or {}).get("sm_mhz") or 2070.0
    slots = sms * schedulers * mhz * 1e6 * (ms / 1e3)
    return {"inst_per_unit": round(inst_per_unit, 2), "units": int(units),
            "frac": round(inst_per_unit * units / slots, 4), "sm_mhz": mhz,
            "what": "warp instructions per work unit from ncu on the profile case, scaled to this run's "
                    "units, over the issue slots of the kernels' time"}


# ------------------------------------------------------------------- ours
def run_ours(args):
    import torch

    from paper_2309_16913_gb300 import build as build_mod
    from paper_2309_16913_gb300 import datagen as dg

    rank, local, world = dist_init("nccl")
    torch.cuda.set_device(local)
    build_mod.build()
    from paper_2309_16913_gb300 import rtree as rt
    rt.load_library()
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()

    seed = 1 + 1000 * rank
    w = dg.workload(WORKLOAD, seed=seed, n=args.n, q=args.q)
    if args.sel:
        w.queries = dg.selectivity_queries(w.queries.shape[0], dg.rng_for(seed + 7), args.sel[0],
                                           args.sel[1], dg._log_uniform_mean(1e-5, 1e-3))
    N, Q = w.rects.shape[0], w.queries.shape[0]
    rects = torch.from_numpy(w.rects).to(dev)
    ids = torch.from_numpy(w.ids).to(dev)
    queries = torch.from_numpy(w.queries).to(dev)
    torch.cuda.synchronize()

    def step(F, layout, mapping, order="input"):
        # stream-ordered: the build and the select return once their work is
        # enqueued (after the host reads they need), and the result and tree
        # are released in the stream's order, so the host enqueues the next
        # step while this one's sort still runs
        t = rt.RTree(rects, ids, fanout=F, layout=layout, stream=stream)
        res = t.range_select(queries, mapping=mapping, stream=stream, order=order)
        total = res.total
        res.close(stream)
        t.close(stream)
        return total

    # ---- pick fanout / layout / mapping / traversal order with the library's
    # autotuner (one build + sorted select per configuration, CUDA-event timed)
    # the configured sweep is F = 16/32/64; F=128 is timed beside it (reported
    # as an extension, not used for the headline)
    swept = [16, 32, 64]
    fanouts = [args.fanout] if args.fanout else swept + [128]
    if args.no_tune:
        if not args.fanout or "auto" in (args.layout, args.mapping, args.order):
            raise SystemExit("--no-tune needs --fanout, --layout, --mapping and --order")
        F, layout, mapping, order = args.fanout, args.layout, args.mapping, args.order
        sweep = None
        beyond = {}
    else:
        tune = rt.rtree_autotune(rects, queries, ids, fanouts=fanouts, include_build=True, stream=stream,
                                 orders=args.order != "input")
        sweep = {k: v for k, v in tune["all"].items()
                 if (args.layout == "auto" or f"_{args.layout}_" in k)
                 and (args.mapping == "auto" or args.mapping in k)
                 and (args.order == "auto" or k.endswith("_hilbert") == (args.order == "hilbert"))}
        beyond = {k: v for k, v in sweep.items() if not args.fanout and int(k.split("_")[0][1:]) not in swept}
        sweep = {k: v for k, v in sweep.items() if k not in beyond}
        best = min(sweep, key=sweep.get)
        F = int(best.split("_")[0][1:])
        layout = best.split("_")[1]
        order = "hilbert" if best.endswith("_hilbert") else "input"
        mapping = best[len(f"F{F}_{layout}_"):].replace("_hilbert", "")
    total_hits = step(F, layout, mapping, order)

    for _ in range(args.warmup):
        step(F, layout, mapping, order)
    torch.cuda.synchronize()

    # ---- timed region (no per-kernel events inside it)
    rt.rtree_timing_reset()
    launches0 = rt.rtree_launch_count()
    clocks = ClockSampler(local)
    clocks.start()
    barrier(world)
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step(F, layout, mapping, order)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    ms_total = ev0.elapsed_time(ev1)
    launches = rt.rtree_launch_count() - launches0
    ms_max = max_over_ranks(ms_total, world, dev)
    value = Q * args.steps * world / (ms_max / 1e3)

    # ---- per-kernel breakdown: the same steps again with CUDA events around
    # every launch (and around the sort's span), outside the timed region
    rt.rtree_timing_reset()
    rt.rtree_timing_enable(True)
    ev2 = torch.cuda.Event(enable_timing=True)
    ev3 = torch.cuda.Event(enable_timing=True)
    ev2.record(stream)
    for _ in range(args.steps):
        step(F, layout, mapping, order)
    ev3.record(stream)
    torch.cuda.synchronize()
    rt.rtree_timing_enable(False)
    kern = rt.rtree_timing_get()
    ms_instrumented = ev2.elapsed_time(ev3)

    # ---- roofline of the dominant kernel; query-order comparison on the same tree
    with rt.RTree(rects, ids, fanout=F, layout=layout) as t:
        stats = t.select_stats(queries)
        res = t.range_select(queries)
        seg = np.diff(res.offsets_tensor().cpu().numpy())
        res.close()
        order_cmp = None if args.no_order else compare_orders(rt, torch, t, queries, stream, mapping)
    layout_cmp = None if args.no_order else compare_layouts(rt, torch, rects, ids, queries, stream, F,
                                                            mapping, order)
    persist = None if args.no_persist else run_persist(rt, torch, rects, ids, queries, F, layout, rank)
    algo = algorithmic_bytes(stats, F, Q, seg)
    hbm, peak_kind = peaks()
    # share = the kernel's event time over the instrumented steps' wall time
    # (the sort's class kernels overlap one another, so their shares can add
    # up past 1; sort_all is their span)
    breakdown = {}
    for name, (n_l, ms) in kern.items():
        if n_l == 0:
            continue
        entry = {"launches": n_l, "ms_per_step": round(ms / args.steps, 3),
                 "share": round(ms / max(1e-9, ms_instrumented), 4)}
        if name in algo and ms > 0:
            entry["gbs"] = round(algo[name] / (ms / args.steps / 1e3) / 1e9, 1)
        breakdown[name] = entry
    # the sort's class kernels overlap on side streams, so their event times
    # are not additive: the sort counts as one unit timed by its span
    overlapped = {"sort_warp", "sort_cta", "sort_gather", "sort_msd", "sort_bucket"} if "sort_all" in kern else set()
    dominant = max((k for k in kern if k in algo and k not in overlapped), key=lambda k: kern[k][1])
    n_l, ms = kern[dominant]
    ms_step = ms / args.steps  # the kernel's time in one step, all its launches
    achieved = algo[dominant] / (ms_step / 1e3) / 1e9
    traffic, traffic_note = ncu_traffic(dominant, F, layout)
    roofline = {"kernel": dominant, "bound": "hbm", "achieved": round(achieved, 1), "peak": hbm,
                "unit": "GB/s", "frac": round(achieved / hbm, 4), "peak_kind": peak_kind,
                "launches_per_step": n_l // args.steps,
                "algorithmic_bytes_per_step": algo[dominant],
                "traffic": traffic}
    if traffic_note:
        roofline["traffic_note"] = traffic_note
    if dominant.startswith("sort_"):
        roofline["note"] = ("sort_all = the whole segmented sort (warp, CTA and long-segment classes on side "
                            "streams), wall time of its span; 8 B per id (gathered + written), 24 B more per id of "
                            "segments over 40960; bound by shared-memory work and per-segment latency, not by HBM "
                            "(ncu: 45-53% issue active, a few % of DRAM peak)")
    # the node-test kernels, each against HBM (ncu DRAM bytes) and issue slots
    roofline_node_test = node_test_roofline(kern, algo, stats, args.steps, hbm, peak_kind, clk, F, layout)

    # ---- end to end through the C ABI with host (pinned) buffers
    e2e = None
    if not args.no_e2e:
        h_rects = torch.from_numpy(w.rects).pin_memory()
        h_ids = torch.from_numpy(w.ids).pin_memory()
        h_q = torch.from_numpy(w.queries).pin_memory()
        # two result buffers: step k+1 runs while step k's ids still travel
        h_off = [torch.empty(Q + 1, dtype=torch.int64).pin_memory() for _ in range(2)]
        h_out = [torch.empty(max(1, int(total_hits)), dtype=torch.int32).pin_memory() for _ in range(2)]

        def e2e_run(steps, log=None):
            # per step: host rects/ids/queries in, host offsets/ids out.  Each
            # select returns once its work and copies are enqueued
            # (rtree_range_select_host_async); the previous step's results are
            # waited for after the next step has started, so its copies to
            # host memory overlap the next build and select.  `log` gets the
            # host time of each step's build call, select call and wait for
            # the previous step's results (ms).
            pending = None
            for k in range(steps):
                a = time.perf_counter()
                h = rt.rtree_build(h_rects, h_ids, F, layout, stream)
                b = time.perf_counter()
                p = rt.rtree_range_select_host_async(h, h_q, h_off[k % 2], h_out[k % 2], mapping=mapping,
                                                     order=order, stream=stream)
                c = time.perf_counter()
                rt.rtree_free(h, stream=stream)
                if pending is not None:
                    assert pending.wait() == total_hits
                pending = p
                if log is not None:
                    log.append([round((b - a) * 1e3, 1), round((c - b) * 1e3, 1),
                                round((time.perf_counter() - c) * 1e3, 1)])
            a = time.perf_counter()
            assert pending.wait() == total_hits
            if log is not None:
                log.append([0.0, 0.0, round((time.perf_counter() - a) * 1e3, 1)])

        e2e_run(2)
        k2 = max(2, min(args.steps, 6))
        # the host link is shared and its rate drifts: five timed runs, the median reported
        runs, step_logs = [], []
        for _ in range(5):
            barrier(world)
            log = []
            t0 = time.perf_counter()
            e2e_run(k2, log)
            torch.cuda.synchronize()
            el = max_over_ranks(time.perf_counter() - t0, world, dev)
            runs.append(Q * k2 * world / el)
            step_logs.append(log)
        e2e = {"value": round(float(np.median(runs)), 1), "unit": UNIT,
               "h2d_bytes_per_step": int(w.rects.nbytes + w.ids.nbytes + w.queries.nbytes),
               "d2h_bytes_per_step": int(8 * (Q + 1) + 4 * int(total_hits)), "steps": k2,
               "runs": [round(r, 1) for r in runs],
               "host_ms_per_step": step_logs,  # per run: [build call, select call, wait for the previous step]
               "note": "build + select per step from pinned host inputs to pinned host results; "
                       "two steps in flight (double-buffered results), all copies inside the timed "
                       "region; median of five runs of `steps` steps"}

    # ---- batched uneven select: graph-captured plans vs one query per launch
    uneven = None
    if not args.no_uneven:
        uneven = run_uneven(args, rt, dg, torch, dev, stream, rank, world, F, layout)

    # ---- serving loop: Poisson request stream over a resident index
    serve = None
    if not args.no_serve:
        serve = run_serve(args, rt, dg, torch, dev, rank, world, F, layout)

    # ---- join workload (R, S 2M each, fanout 32)
    join = None
    if not args.no_join:
        j = dg.workload("join", seed=2 + 1000 * rank)
        jr = torch.from_numpy(j.rects).to(dev)
        js = torch.from_numpy(j.rects_s).to(dev)

        def jstep(sort_children=False, prune="off", traversal="auto"):
            a = rt.RTree(jr, None, fanout=32, stream=stream, sort_children=sort_children)
            b = rt.RTree(js, None, fanout=32, stream=stream, sort_children=sort_children)
            r = a.join(b, stream=stream, prune=prune, traversal=traversal)
            tot = r.total
            r.close(stream); a.close(stream); b.close(stream)
            return tot

        def jtime(**kw):
            pairs = jstep(**kw)
            jstep(**kw)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            kj = max(1, args.steps)
            e0.record(stream)
            for _ in range(kj):
                jstep(**kw)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = max_over_ranks(e0.elapsed_time(e1) / kj, world, dev)
            # kernel breakdown from a separate, instrumented step
            rt.rtree_timing_reset()
            rt.rtree_timing_enable(True)
            jstep(**kw)
            torch.cuda.synchronize()
            rt.rtree_timing_enable(False)
            k = rt.rtree_timing_get()
            trav = sum(v[1] for n, v in k.items() if n.startswith("join_") or n.startswith("jq_"))
            return pairs, ms, trav, {n: v for n, v in k.items() if n.startswith("join_") and v[0]}

        pairs, jms, jtrav, jk = jtime()
        ppairs, pms, ptrav, pk = jtime(sort_children=True, prune="on")
        assert ppairs == pairs
        # the two schedules of the traversal, plain and pruned
        sched = {}
        for trv in ("levels", "queue"):
            for pr in ("off", "on"):
                p_, ms_, tr_, _ = jtime(sort_children=pr == "on", prune=pr, traversal=trv)
                assert p_ == pairs
                sched[f"{trv}_prune_{pr}"] = {"ms_per_step": round(ms_, 3), "traversal_ms": round(tr_, 3)}
        a = rt.RTree(jr, None, fanout=32, stream=stream, sort_children=True)
        b = rt.RTree(js, None, fanout=32, stream=stream, sort_children=True)
        jstats = a.join_stats(b, stream=stream, prune="off")
        a.close(); b.close()
        join = {"metric": "join pairs/s (2M x 2M, build of both trees included)",
                "value": round(pairs * world / (jms / 1e3), 1), "unit": "pairs/s",
                "pairs": int(pairs), "ms_per_step": round(jms, 3),
                "traversal_ms": round(jtrav, 3),
                "schedules": sched,
                "join_stats": jstats,
                "roofline": join_roofline(jstats, 32, 32, jk, hbm, peak_kind, clk),
                "pruned": {"what": "sorted-children trees, O3 + O4/O5 pruned join (Section 4.2)",
                           "value": round(ppairs * world / (pms / 1e3), 1), "unit": "pairs/s",
                           "ms_per_step": round(pms, 3), "traversal_ms": round(ptrav, 3),
                           "roofline": join_roofline(jstats, 32, 32, pk, hbm, peak_kind, clk)}}
        if rank == 0 and world == 1 and not args.no_cpu_baseline:
            join["cpu_baseline"] = oracle_join_rate(j, 32)

    # ---- CPU oracle baseline (rank 0, one GPU runs only)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = oracle_rate(w, F)

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(ms_max / args.steps, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"scaled range select: {N} rects (80% 64-cluster gaussian, "
                                   f"20% uniform, sides log-U[1e-5,1e-3]), {Q} queries "
                                   "(selectivity log-U[1e-6,1e-3]), STR build + sorted select per step",
                       "fanout": F, "layout": layout, "mapping": mapping, "order": order,
                       "ids_returned_per_step": int(total_hits),
                       "l2": "inputs larger than L2 (rects 160 MB, tree ~200 MB; no flush)",
                       "sweep_ms_per_step": sweep, "seed": seed,
                       "beyond_sweep": ({"best": min(beyond, key=beyond.get), "ms_per_step": min(beyond.values()),
                                         "note": "F=128, outside the configured 16/32/64 sweep: timed by the same "
                                                 "autotune call, not used for the headline"} if beyond else None)},
            "gpu_launches": int(launches),
            "ms_per_step_instrumented": round(ms_instrumented / args.steps, 3),
            "clocks": clk,
            "roofline": roofline,
            "roofline_node_test": roofline_node_test,
            "kernels": breakdown,
            "e2e": e2e,
            "cpu_baseline": cpu,
            "join": join,
            "query_order": order_cmp,
            "layouts": layout_cmp,
            "persist": persist,
            "uneven": uneven,
            "serve": serve,
            "select_stats": stats,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def compare_orders(rt, torch, tree, queries, stream, mapping, reps=3):
    """Select time (no build) with the batch taken in input order and in
    Hilbert order of the query centres; the results are identical."""
    out = {}
    for order in ("input", "hilbert"):
        for _ in range(2):
            tree.range_select(queries, mapping=mapping, stream=stream, order=order).close()
        torch.cuda.synchronize()
        rt.rtree_timing_reset()
        rt.rtree_timing_enable(True)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            tree.range_select(queries, mapping=mapping, stream=stream, order=order).close()
        e1.record(stream)
        torch.cuda.synchronize()
        rt.rtree_timing_enable(False)
        k = rt.rtree_timing_get()
        trav = sum(v[1] for n, v in k.items() if n.startswith("select_")) / reps
        out[order] = {"ms_per_select": round(e0.elapsed_time(e1) / reps, 3),
                      "traversal_ms": round(trav, 3)}
    out["what"] = "1M-query select on the built tree, no build; traversal = select_bound + select_desc"
    return out


def run_persist(rt, torch, rects, ids, queries, F, layout, rank):
    """Save the built 10M tree to a file and load it back (the serving
    restart path); the file sits in the page cache, so this times the
    library's write/read, checksum and copy path, not the disk."""
    import tempfile
    path = os.path.join(tempfile.gettempdir(), f"bench_rank{rank}_{os.getpid()}.rtree")
    t = rt.RTree(rects, ids, fanout=F, layout=layout)
    try:
        t0 = time.perf_counter()
        t.save(path)
        save_s = time.perf_counter() - t0
        size = os.path.getsize(path)
        t0 = time.perf_counter()
        t2 = rt.RTree.load(path)
        torch.cuda.synchronize()
        load_s = time.perf_counter() - t0
        a = t.range_select(queries[:20000])
        b = t2.range_select(queries[:20000])
        same = bool(torch.equal(a.offsets_tensor(), b.offsets_tensor()) and
                    torch.equal(a.ids_tensor(), b.ids_tensor()))
        a.close(); b.close(); t2.close()
    finally:
        t.close()
        if os.path.exists(path):
            os.remove(path)
    return {"file_bytes": size, "save_ms": round(save_s * 1e3, 1), "load_ms": round(load_s * 1e3, 1),
            "load_gbs": round(size / load_s / 1e9, 2), "loaded_tree_answers_same": same,
            "what": "rtree_save / rtree_load of the bench's tree via the page cache (host wall clock)"}


def compare_layouts(rt, torch, rects, ids, queries, stream, F, mapping, order, reps=3):
    """Traversal kernel time (bound + descriptor passes) of the same select
    on trees built in each node layout: D0 (aos), D1 (soa), D2 (lohi)."""
    out = {}
    for layout in ("aos", "soa", "lohi"):
        with rt.RTree(rects, ids, fanout=F, layout=layout, stream=stream) as t:
            for _ in range(2):
                t.range_select(queries, mapping=mapping, stream=stream, order=order).close()
            torch.cuda.synchronize()
            rt.rtree_timing_reset()
            rt.rtree_timing_enable(True)
            for _ in range(reps):
                t.range_select(queries, mapping=mapping, stream=stream, order=order).close()
            torch.cuda.synchronize()
            rt.rtree_timing_enable(False)
            k = rt.rtree_timing_get()
        out[layout] = {n: round(v[1] / reps, 3) for n, v in k.items()
                       if n in ("select_bound", "select_count", "select_desc")}
    out["what"] = f"F={F}, {mapping}, {order} order: traversal kernel ms per 1M-query select"
    return out


def run_uneven(args, rt, dg, torch, dev, stream, rank, world, F, layout):
    """The heavy-tailed batch (10M-rect index, 100k queries, 1% large): the
    graph-captured batched form against one query per launch."""
    u = dg.workload("uneven", seed=3 + 1000 * rank, n=args.n, q=None if args.q is None else args.q // 10)
    Q = u.queries.shape[0]
    q_dev = torch.from_numpy(u.queries).to(dev)
    tree = rt.RTree(torch.from_numpy(u.rects).to(dev), torch.from_numpy(u.ids).to(dev), fanout=F,
                    layout=layout, stream=stream)
    res = tree.range_select(q_dev, stream=stream)
    total = res.total
    res.close()
    reps = max(3, args.steps)
    out = {"workload": f"uneven: {u.rects.shape[0]} rects, {Q} queries per batch (1% with sides "
                       "U[0.05,0.2]), sorted results", "fanout": F, "layout": layout,
           "ids_per_batch": int(total)}

    def timed(fn, n):
        fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(n):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / n

    for mapping in ("warp_per_query", "work_queue"):
        plan = rt.Plan(tree, Q, int(total * 1.02) + 4096, mapping)
        ms = timed(lambda: plan.run(q_dev, stream), reps)
        out[f"graph_{mapping}_qps"] = round(Q * world / (ms / 1e3), 1)
        out[f"graph_{mapping}_ms"] = round(ms, 3)
        plan.close()

    def plain(mapping):
        r = tree.range_select(q_dev, mapping=mapping, stream=stream)
        r.close()

    for mapping in ("warp_per_query", "work_queue"):
        ms = timed(lambda: plain(mapping), reps)
        out[f"call_{mapping}_qps"] = round(Q * world / (ms / 1e3), 1)
    # one query per launch: every query its own select call (sample of 2000)
    sample = q_dev[:2000]
    n1 = sample.shape[0]

    def one_by_one():
        for i in range(n1):
            r = tree.range_select(sample[i:i + 1], stream=stream)
            r.close()

    ms = timed(one_by_one, 1)
    out["one_query_per_launch_qps"] = round(n1 * world / (ms / 1e3), 1)
    best = max(v for k, v in out.items() if k.startswith("graph_") and k.endswith("_qps"))
    out["batched_over_one_per_launch"] = round(best / out["one_query_per_launch_qps"], 1)
    tree.close()
    return out


def run_serve(args, rt, dg, torch, dev, rank, world, F, layout):
    """A Poisson stream of requests over a resident index: 90% single range
    queries (selectivity log-uniform in [1e-7, 1e-3]), 10% probe joins of 1k-10k
    uniform rectangles.  One client thread submits at the arrival times,
    another collects the replies; the server batches continuously."""
    import threading
    w = dg.workload("serve", seed=4 + 1000 * rank, n=args.serve_n, q=1)
    tree = rt.RTree(torch.from_numpy(w.rects).to(dev), torch.from_numpy(w.ids).to(dev), fanout=F,
                    layout=layout)
    del w
    rng = dg.rng_for(40 + rank)
    n_req = args.serve_requests
    mean_side = dg._log_uniform_mean(1e-5, 1e-3)
    kinds = rng.random(n_req) < 0.10
    reqs = []
    for k in range(n_req):
        if kinds[k]:
            m = 1000 + int(rng.random() * 9000)
            reqs.append((rt.RTREE_REQ_PROBE_JOIN, dg.uniform_rects(m, rng, 0.0, 1e-3)))
        else:
            reqs.append((rt.RTREE_REQ_SELECT, dg.selectivity_queries(1, rng, 1e-7, 1e-3, mean_side)))
    n_queries = sum(r[1].shape[0] for r in reqs)
    out = {"workload": f"serving: {tree.info()['n']} rects (50/50 uniform/clustered), {n_req} requests "
                       "(90% single range queries, selectivity log-U[1e-7,1e-3]; 10% probe joins of "
                       "1k-10k uniform rects), Poisson arrivals", "queries_per_run": int(n_queries),
           "runs": []}
    srv = rt.Server(tree, workers=3, max_batch_queries=65536, max_batch_ids=64 << 20)
    # warm: capture the graphs of the common batch sizes
    warm = [srv.submit(r[1], r[0]) for r in reqs[:200]]
    for tk in warm:
        srv.wait(tk)
    for rate in (5000.0, 20000.0, 80000.0):
        srv.reset_stats()
        gaps = -np.log(1.0 - rng.random(n_req)) / rate
        arrivals = np.cumsum(gaps)
        tickets = [None] * n_req
        got = [0]

        def collect():
            for i in range(n_req):
                while tickets[i] is None:
                    time.sleep(0.0002)
                srv.wait(tickets[i])
                got[0] += 1

        col = threading.Thread(target=collect)
        col.start()
        t0 = time.perf_counter()
        for i, (kind, rects) in enumerate(reqs):
            while time.perf_counter() - t0 < arrivals[i]:
                pass
            tickets[i] = srv.submit(rects, kind)
        col.join()
        el = time.perf_counter() - t0
        st = srv.stats()
        out["runs"].append({
            "offered_req_s": rate, "achieved_req_s": round(n_req / el, 1),
            "queries_s": round(n_queries / el, 1), "p50_ms": round(st["p50_us"] / 1e3, 3),
            "p99_ms": round(st["p99_us"] / 1e3, 3), "max_ms": round(st["max_us"] / 1e3, 3),
            "batches": st["batches"], "mean_batch_queries": round(st["batch_queries"] / max(1, st["batches"]), 1),
            "splits": st["splits"], "fallbacks": st["fallbacks"]})
    srv.stop()
    tree.close()
    return out


# ------------------------------------------------------------- reference
def cpu_info():
    """Host CPU as the OS reports it (lscpu, else /proc/cpuinfo)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            k, _, v = line.partition(":")
            if k.strip().lower() in ("model name", "model"):
                if v.strip() and not v.strip().isdigit():
                    model = v.strip()
                    break
    except (OSError, subprocess.SubprocessError):
        pass
    if model is None:
        try:
            for line in open("/proc/cpuinfo"):
                k, _, v = line.partition(":")
                if k.strip().lower() in ("model name", "cpu part"):
                    model = v.strip()
                    break
        except OSError:
            pass
    return {"nproc": os.cpu_count(), "model": model, "machine": platform.machine()}


def oracle_rate(w, F, sample=CPU_SAMPLE_QUERIES):
    """The CPU oracle on this host: STR build of all rectangles (one thread),
    then a sorted select of a fixed subset of the queries, once on one
    thread and once on every core; extrapolated to the whole batch."""
    import oracle
    threads = os.cpu_count() or 1
    t0 = time.perf_counter()
    tree = oracle.Tree(w.rects, w.ids, F)
    tb = time.perf_counter() - t0
    qs = w.queries[:sample]
    t1 = time.perf_counter()
    tree.select(qs, threads=1)
    per_q1 = (time.perf_counter() - t1) / qs.shape[0]
    t1 = time.perf_counter()
    tree.select(qs, threads=threads)
    per_qn = (time.perf_counter() - t1) / qs.shape[0]
    Q = w.queries.shape[0]
    return {"value": round(Q / (tb + per_qn * Q), 2), "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"oracle STR build of all {w.rects.shape[0]} rects at F={F} ({tb:.2f} s, one thread) + "
                      f"sorted select of the first {qs.shape[0]} queries on {threads} threads "
                      f"({per_qn * 1e6:.2f} us/query), extrapolated to {Q} queries: "
                      f"{Q} / (build + per_query * {Q})",
            "build_s": round(tb, 3),
            "select_qps": {"threads_1": round(1.0 / per_q1, 1), f"threads_{threads}": round(1.0 / per_qn, 1)},
            "single_thread": {"value": round(Q / (tb + per_q1 * Q), 2), "cores": 1,
                              "per_query_us": round(per_q1 * 1e6, 2)},
            "cpu": cpu_info()}


def oracle_join_rate(j, F=32):
    """The CPU oracle's join of the join workload: both STR builds (one
    thread each) + the synchronized traversal on one thread and on every
    core; pairs/s over builds + traversal, as the GPU step counts them."""
    import oracle
    threads = os.cpu_count() or 1
    t0 = time.perf_counter()
    a = oracle.Tree(j.rects, j.ids, F)
    b = oracle.Tree(j.rects_s, j.ids_s, F)
    tb = time.perf_counter() - t0
    t1 = time.perf_counter()
    p1 = a.join(b, threads=1)
    tj1 = time.perf_counter() - t1
    t1 = time.perf_counter()
    pn = a.join(b, threads=threads)
    tjn = time.perf_counter() - t1
    assert np.array_equal(p1, pn)
    pairs = len(pn)
    return {"value": round(pairs / (tb + tjn), 1), "unit": "pairs/s", "cores": threads, "kind": "oracle",
            "sample": f"the whole join workload: STR builds of R and S ({tb:.2f} s, one thread) + join "
                      f"on {threads} threads ({tjn:.2f} s); pairs / (builds + join)",
            "pairs": int(pairs), "build_s": round(tb, 3),
            "single_thread": {"value": round(pairs / (tb + tj1), 1), "cores": 1, "join_s": round(tj1, 3)},
            "join_s": round(tjn, 3), "cpu": cpu_info()}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_2309_16913_gb300 import datagen as dg
    import oracle
    w = dg.workload(WORKLOAD, seed=1, n=args.n, q=args.q)
    F = args.fanout or REF_FANOUT
    threads = os.cpu_count() or 1
    t0 = time.perf_counter()
    tree = oracle.Tree(w.rects, w.ids, F)
    tb = time.perf_counter() - t0
    qs = w.queries[:CPU_SAMPLE_QUERIES]
    for _ in range(args.warmup):
        tree.select(qs, threads=threads)
    t1 = time.perf_counter()
    for _ in range(args.steps):
        tree.select(qs, threads=threads)
    el = time.perf_counter() - t1
    per_q = el / (args.steps * qs.shape[0])
    Q = w.queries.shape[0]
    value = Q / (tb + per_q * Q)
    cpu = {"value": round(value, 2), "unit": UNIT, "cores": threads, "kind": "oracle",
           "sample": f"tree built once at F={F} ({tb:.2f} s, one thread); each step = sorted select "
                     f"of the first {qs.shape[0]} of {Q} queries on {threads} threads; "
                     f"value = {Q} / (build + per_query * {Q})",
           "cpu": cpu_info()}
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 2), "unit": UNIT,
            "n_gpus": int(os.environ.get("WORLD_SIZE", "1")), "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(el / args.steps * 1e3, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": f"scaled range select: {w.rects.shape[0]} rects, {Q} queries",
                       "fanout": F},
            "cpu_baseline": cpu,
            "e2e": {"value": round(value, 2), "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
