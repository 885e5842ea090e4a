// select.cu -- batched range select (Section 3), one warp per query.
//
// The paper's vectorized select (Section 3, steps 1-4 with the queue of O1)
// maps onto a warp as follows:
//   step 1, query vector: every lane holds the query box in registers;
//   step 2, child-MBR vector: lane j loads child j of the node being tested
//           (SoA: four coalesced 4-byte loads; AoS: one 16-byte load); with
//           F < 32 a warp tests 32/F nodes at once, with F > 32 a lane holds
//           F/32 children;
//   step 3, predicate: four float32 comparisons, then __ballot_sync gives the
//           bitmask of qualifying children;
//   step 4, queue insertion: popc(mask & lanemask_lt) gives each qualifying
//           lane its slot, so the children are compacted onto a per-warp
//           stack in shared memory in lane order (the compress-store).
// The stack is depth-first (LIFO) rather than the paper's breadth-first
// queue so that it has a fixed bound: every push segment sits one level
// deeper than the segment it was popped from, so at most H segments of at
// most 32*ceil(F/32) entries are alive, H*max(32,F) ints per warp.
//
// Two additions that leave the result unchanged: a child whose MBR lies
// inside the query contributes its whole subtree (a contiguous run of leaf
// entries) without being visited, and the output is produced in two passes
// over the same traversal: count, exclusive scan, scatter at the offsets.
//
// Mappings: warp per query (a warp takes the next query from a counter and
// walks its whole subtree), or a persistent device work queue of (query,
// node) items from which warps split large queries (k_select_wq below).
//
// Pass kinds:
//   COUNT    per query: ids found, and (optionally) how many came one by one
//            from leaves and how many whole subtrees were taken;
//   SCATTER  writes the ids themselves in traversal order (unsorted output);
//   DESC     writes the leaf hits and, for every whole subtree, its (lo, hi)
//            range of the tree's id array; the sorted output is then built
//            by the segmented sort, which reads the ranges directly;
//   BOUND    the count pass stopped above the leaves, sizing DESC's slots.
// With warp per query at F = 64 and 128, DESC visits a leaf-parent's
// intersecting leaves in place (no push, no pop) and derives each leaf's id
// span from its position (STR fills every leaf but one, whose position the
// build records), so a leaf costs one memory round trip: its entries and its
// ids are requested together.
#include <atomic>
#include <cstring>

#include "internal.cuh"

namespace rt {
namespace {

constexpr int kWarps = 8;
constexpr int kThreads = kWarps * 32;
// PASS_BOUND is the count pass stopped above the leaves: an intersecting leaf
// child that is not inside the query is not visited but reserves F slots (an
// upper bound on its hits); whole subtrees are counted exactly.  It sizes a
// descriptor pass whose leaf-hit slots are such bounds.
enum { PASS_COUNT = 0, PASS_SCATTER = 1, PASS_DESC = 2, PASS_BOUND = 3 };
enum { FLAG_STACK = 1, FLAG_COUNT_MISMATCH = 2, FLAG_TIMEOUT = 4 };

// Copies ids[lo, hi) to out[0, hi-lo) with the whole warp.
__device__ __forceinline__ void warp_copy(int32_t *__restrict__ out,
                                          const int32_t *__restrict__ ids, int lo, int hi,
                                          int lane)
{
    int e = lo + lane;
    for (; e + 96 < hi; e += 128) {
        const int32_t a = __ldg(ids + e), b = __ldg(ids + e + 32), c = __ldg(ids + e + 64),
                      d = __ldg(ids + e + 96);
        out[e - lo] = a;
        out[e - lo + 32] = b;
        out[e - lo + 64] = c;
        out[e - lo + 96] = d;
    }
    for (; e < hi; e += 32)
        out[e - lo] = __ldg(ids + e);
}

// Results of one walk (a query, or one (query, subtree) work item).
struct Walk {
    int32_t cur;   // ids found, warp-uniform (a query's ids fit 31 bits)
    int32_t lcur;  // of which found one by one in leaves
    int32_t rcur;  // whole subtrees taken
    unsigned long long n_visit, n_leaf;
    bool overflow;
};

// Output limits of one query (non-work-queue passes write at fixed offsets).
struct Seg {
    int64_t base, lim, lbase, llim, rbase, rlim;
};

// The leaf level's short leaf (TreeDev::leaf_part), read once per kernel;
// ok: at most one short leaf, so leaf spans follow from positions.
struct LeafPart {
    int64_t pos;
    int cnt;
    bool ok;
};

__device__ __forceinline__ LeafPart leaf_part_of(const TreeDev &t)
{
    LeafPart lp{-1, 0, false};
    if (t.leaf_part) {
        lp.pos = __ldg(t.leaf_part);
        lp.cnt = (int)__ldg(t.leaf_part + 1);
        lp.ok = __ldg(t.leaf_part + 2) <= 1;
    }
    return lp;
}

// Entries [first, first + cnt) of the id array belong to leaf node g.
template <int F>
__device__ __forceinline__ void leaf_span(const TreeDev &t, const LeafPart &lp, int64_t g, int &first, int &cnt)
{
    if (lp.ok) {
        const int64_t s = g - t.leaf_base;
        cnt = s == lp.pos ? lp.cnt : F;
        first = (int)(s * F - (lp.pos >= 0 && s > lp.pos ? F - lp.cnt : 0));
    } else {
        const int4 lm = __ldg(t.meta + g);
        first = lm.x;
        cnt = lm.y;
    }
}

// Reserves n slots of a per-query cursor (lane 0 does the atomic).
__device__ __forceinline__ int64_t reserve(int32_t *cursor, int n, int lane)
{
    int r = 0;
    if (lane == 0 && n > 0)
        r = atomicAdd(cursor, n);
    return __shfl_sync(RT_FULL, r, 0);
}

// One step of a walk: pops up to K nodes from the warp's stack, tests their
// children against the query (ballot), pushes children that need a visit,
// and emits leaf hits and whole subtrees.  WQ: output slots are reserved from
// per-query cursors (several warps may serve one query); otherwise they
// follow the walk's own counters from the query's segment start.
template <int F, int LAYOUT, int PASS, bool WQ>
__device__ __forceinline__ void select_step(const TreeDev &t, const float4 q, int32_t *st, int &top,
                                            int cap, const SelIO &io, int64_t qi, const Seg &sg,
                                            Walk &wk, bool stats, int lane, int grp, int sub,
                                            unsigned lt, const LeafPart &lp)
{
    constexpr int G = F < 32 ? F : 32;
    constexpr int K = 32 / G;
    constexpr int C = F / G;
    const int k = top < K ? top : K;
    const int node = grp < k ? st[top - 1 - grp] : -1;
    top -= k;
    __syncwarp();
    if (stats) {
        wk.n_visit += k;
        wk.n_leaf += __popc(__ballot_sync(RT_FULL, node >= t.leaf_base && sub == 0));
    }
    // Entry loads do not wait for the node's metadata: unused slots hold the
    // empty box, and the count only masks them afterwards.
    float4 b[C];
#pragma unroll
    for (int c = 0; c < C; ++c)
        b[c] = node >= 0 ? load_entry_t<F, LAYOUT>(t.mbr, node, sub + c * G) : empty_box();
    const int4 m = node >= 0 ? __ldg(t.meta + node) : make_int4(0, 0, 0, 0);
    const bool leaf = node >= t.leaf_base;
    // Every node of this step is a leaf (warp-uniform; with K == 1 there is
    // one node): only the overlap test and the emit are needed.  Lanes
    // without a node see count 0.
    const bool all_leaf = K == 1 ? leaf : __all_sync(RT_FULL, node < 0 || leaf);
    const bool any_leaf = K == 1 ? leaf : __any_sync(RT_FULL, node >= 0 && leaf);
    if (all_leaf) {
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const int j = sub + c * G;
            const bool emit = j < m.y && meets(b[c], q);
            const unsigned me = __ballot_sync(RT_FULL, emit);
            if (PASS == PASS_SCATTER && me) {
                const int64_t at = WQ ? sg.base + reserve(io.cur_ids + qi, __popc(me), lane) : sg.base + wk.cur;
                const int64_t o = at + __popc(me & lt);
                if (emit && o < sg.lim && o < io.out_cap)
                    io.out[o] = __ldg(t.ids + m.x + j);
            }
            if (PASS == PASS_DESC && me) {
                const int64_t at = WQ ? sg.lbase + reserve(io.cur_leaf + qi, __popc(me), lane) : sg.lbase + wk.lcur;
                const int64_t o = at + __popc(me & lt);
                if (emit && o < sg.llim && o < io.leaf_cap)
                    io.leaf_out[o] = __ldg(t.ids + m.x + j);
            }
            wk.cur += __popc(me);
            wk.lcur += __popc(me);
        }
        __syncwarp();
        return;
    }
    if (PASS == PASS_BOUND && K == 1 && !leaf && m.x >= t.leaf_base) {
        // the bound pass at a node whose children are leaves: an intersecting
        // leaf inside the query is counted whole, any other reserves F slots;
        // nothing is pushed (one node per step: the test is warp-uniform)
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const int j = sub + c * G;
            const bool hit = j < m.y && meets(b[c], q);
            const bool cont = hit && inside(b[c], q);
            const int r = F * __popc(__ballot_sync(RT_FULL, hit && !cont));
            wk.lcur += r;
            wk.cur += r;
            const unsigned mc = __ballot_sync(RT_FULL, cont);
            if (mc) {
                int n = 0;
                if (cont) {
                    int lo;
                    leaf_span<F>(t, lp, m.x + j, lo, n);
                }
                wk.rcur += __popc(mc);
                wk.cur += __reduce_add_sync(RT_FULL, (unsigned)n);
            }
        }
        __syncwarp();
        return;
    }
    if (PASS == PASS_DESC && !WQ && (F == 64 || F == 128) && node >= 0 && !leaf && m.x >= t.leaf_base) {
        // the descriptor pass at a node whose children are leaves: a leaf
        // inside the query is emitted as its id range, and the other
        // intersecting leaves are visited here, one after another from the
        // ballot, instead of through the stack (the sort makes the order of
        // the hits immaterial).  Measured faster at F=64 and F=128 (with
        // the CTAs per SM of select_min_blocks); at F=32 the stack form is
        // faster.  Leaf spans come from the leaf's position (leaf_span), so a
        // leaf's ids are requested with its entries.
        unsigned mv[C];
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const int j = sub + c * G;
            const bool hit = j < m.y && meets(b[c], q);
            const bool cont = hit && inside(b[c], q);
            mv[c] = __ballot_sync(RT_FULL, hit && !cont);
            const unsigned mc = __ballot_sync(RT_FULL, cont);
            if (mc) {
                int lo = 0, hi = 0;
                if (cont) {
                    int cn;
                    leaf_span<F>(t, lp, m.x + j, lo, cn);
                    hi = lo + cn;
                }
                const int64_t o = sg.rbase + wk.rcur + __popc(mc & lt);
                if (cont && o < sg.rlim && o < io.rng_cap)
                    io.rng_out[o] = make_int2(lo, hi);
                wk.rcur += __popc(mc);
                wk.cur += __reduce_add_sync(RT_FULL, (unsigned)(hi - lo));
            }
        }
#pragma unroll
        for (int c = 0; c < C; ++c) {
            unsigned mm = mv[c];
            while (mm) {
                const int lf = m.x + c * G + __ffs(mm) - 1;
                mm &= mm - 1;
                int first, cnt;
                leaf_span<F>(t, lp, lf, first, cnt);
                float4 e[C];
                int32_t id[C];
#pragma unroll
                for (int cc = 0; cc < C; ++cc) {
                    const int jj = sub + cc * G;
                    e[cc] = load_entry_t<F, LAYOUT>(t.mbr, lf, jj);
                    id[cc] = jj < cnt ? __ldg(t.ids + first + jj) : 0;
                }
                if (stats) {
                    ++wk.n_visit;
                    ++wk.n_leaf;
                }
#pragma unroll
                for (int cc = 0; cc < C; ++cc) {
                    const int jj = sub + cc * G;
                    const bool emit = jj < cnt && meets(e[cc], q);
                    const unsigned me = __ballot_sync(RT_FULL, emit);
                    if (me) {
                        const int64_t o = sg.lbase + wk.lcur + __popc(me & lt);
                        if (emit && o < sg.llim && o < io.leaf_cap)
                            io.leaf_out[o] = id[cc];
                    }
                    wk.cur += __popc(me);
                    wk.lcur += __popc(me);
                }
            }
        }
        __syncwarp();
        return;
    }
#pragma unroll
    for (int c = 0; c < C; ++c) {
        const int j = sub + c * G;
        const bool hit = node >= 0 && j < m.y && meets(b[c], q);
        const bool cont = hit && !leaf && inside(b[c], q);
        // bound pass: children of this node are leaves (all children of a
        // node are on one level), so they are reserved, not visited
        const bool slot = PASS == PASS_BOUND && hit && !leaf && !cont && m.x >= t.leaf_base;
        const bool push = hit && !leaf && !cont && !slot;
        const bool emit = hit && leaf;
        if (PASS == PASS_BOUND) {
            const int r = F * __popc(__ballot_sync(RT_FULL, slot));
            wk.lcur += r;
            wk.cur += r;
        }
        const unsigned mp = __ballot_sync(RT_FULL, push);
        if (push) {
            const int pos = top + __popc(mp & lt);
            if (pos < cap)
                st[pos] = m.x + j;
        }
        top += __popc(mp);
        if (any_leaf) {  // a step of internal nodes only emits nothing
            const unsigned me = __ballot_sync(RT_FULL, emit);
            if (PASS == PASS_SCATTER && me) {
                const int64_t at = WQ ? sg.base + reserve(io.cur_ids + qi, __popc(me), lane) : sg.base + wk.cur;
                const int64_t o = at + __popc(me & lt);
                if (emit && o < sg.lim && o < io.out_cap)
                    io.out[o] = __ldg(t.ids + m.x + j);
            }
            if (PASS == PASS_DESC && me) {
                const int64_t at = WQ ? sg.lbase + reserve(io.cur_leaf + qi, __popc(me), lane) : sg.lbase + wk.lcur;
                const int64_t o = at + __popc(me & lt);
                if (emit && o < sg.llim && o < io.leaf_cap)
                    io.leaf_out[o] = __ldg(t.ids + m.x + j);
            }
            wk.cur += __popc(me);
            wk.lcur += __popc(me);
        }
        const unsigned mc = __ballot_sync(RT_FULL, cont);
        if (mc) {
            int lo = 0, hi = 0;
            if (cont) {
                const int4 cm = __ldg(t.meta + m.x + j);
                lo = cm.z;
                hi = cm.w;
            }
            if (PASS == PASS_DESC) {
                const int64_t at = WQ ? sg.rbase + reserve(io.cur_rng + qi, __popc(mc), lane) : sg.rbase + wk.rcur;
                const int64_t o = at + __popc(mc & lt);
                if (cont && o < sg.rlim && o < io.rng_cap)
                    io.rng_out[o] = make_int2(lo, hi);
            }
            wk.rcur += __popc(mc);
            if (PASS == PASS_SCATTER) {
                unsigned mm = mc;
                while (mm) {
                    const int src = __ffs(mm) - 1;
                    mm &= mm - 1;
                    const int l = __shfl_sync(RT_FULL, lo, src);
                    const int h = __shfl_sync(RT_FULL, hi, src);
                    const int64_t at = WQ ? sg.base + reserve(io.cur_ids + qi, h - l, lane) : sg.base + wk.cur;
                    const int64_t end = sg.lim < io.out_cap ? sg.lim : io.out_cap;
                    const int64_t room = end - at;
                    const int hh = (int64_t)(h - l) <= room ? h : l + (int)(room > 0 ? room : 0);
                    warp_copy(io.out + at, t.ids, l, hh, lane);
                    wk.cur += h - l;
                }
            } else {
                wk.cur += __reduce_add_sync(RT_FULL, (unsigned)(hi - lo));
            }
        }
    }
    if (top > cap) {  // cannot happen with cap = H*max(32,F); guarded anyway
        wk.overflow = true;
        top = 0;
    }
    __syncwarp();
}

__device__ __forceinline__ Seg seg_of(const SelIO &io, int pass, int64_t qi)
{
    Seg sg{0, 0, 0, 0, 0, 0};
    if (pass == PASS_SCATTER) {
        sg.base = __ldg(io.offsets + qi);
        sg.lim = __ldg(io.offsets + qi + 1);  // writes never pass the segment end
    }
    if (pass == PASS_DESC) {
        sg.lbase = __ldg(io.off_leaf + qi);
        sg.llim = __ldg(io.off_leaf + qi + 1);
        sg.rbase = __ldg(io.off_rng + qi);
        sg.rlim = __ldg(io.off_rng + qi + 1);
    }
    return sg;
}

__device__ __forceinline__ void flush_stats(unsigned long long *stats, const Walk &wk, bool new_query)
{
    if (new_query)
        atomicAdd(stats + 0, 1ull);
    atomicAdd(stats + 1, wk.n_visit);
    atomicAdd(stats + 2, wk.n_leaf);
    atomicAdd(stats + 3, (unsigned long long)wk.rcur);
    atomicAdd(stats + 4, (unsigned long long)wk.cur);
    atomicAdd(stats + 5, (unsigned long long)(wk.cur - wk.lcur));
}

// CTAs per SM the warp-per-query kernel is compiled for.  The descriptor
// pass at F=64 takes six (40 registers a thread): its walk is bound by the
// latency of dependent node loads, and the extra resident warps were
// measured to outweigh a few spilled registers; at F=128 four (64
// registers, no spills); elsewhere the compiler chooses.
constexpr int select_min_blocks(int F, int pass)
{
    return pass != PASS_DESC ? 1 : (F == 64 ? 6 : (F == 128 ? 4 : 1));
}

// Warp per query: each warp takes the next query from a counter and walks
// its whole subtree.
template <int F, int LAYOUT, int PASS>
__global__ void __launch_bounds__(kThreads, select_min_blocks(F, PASS))
    k_select(TreeDev t, const float4 *__restrict__ queries, int64_t Q, SelIO io,
             unsigned long long *__restrict__ next_query, int32_t *__restrict__ flags, int cap,
             unsigned long long *__restrict__ stats)
{
    constexpr int G = F < 32 ? F : 32;
    extern __shared__ int32_t smem[];
    const int lane = threadIdx.x & 31;
    int32_t *st = smem + (threadIdx.x >> 5) * cap;
    const int grp = lane / G, sub = lane % G;
    const unsigned lt = lanemask_lt();
    const LeafPart lp = PASS == PASS_DESC || PASS == PASS_BOUND ? leaf_part_of(t) : LeafPart{-1, 0, false};

    for (;;) {
        unsigned long long qi = 0;
        if (lane == 0)
            qi = atomicAdd(next_query, 1ull);
        qi = __shfl_sync(RT_FULL, qi, 0);
        if (qi >= (unsigned long long)Q)
            break;
        if (io.order)
            qi = __ldg(io.order + qi);
        const float4 q = __ldg(queries + qi);
        const Seg sg = seg_of(io, PASS, (int64_t)qi);
        Walk wk{0, 0, 0, 0, 0, false};
        int top = 0;
        if (t.nodes > 0) {
            if (lane == 0)
                st[0] = 0;
            top = 1;
        }
        __syncwarp();
        int steps = 0;  // a query visits each node at most once
        while (top > 0) {
            if (++steps > t.nodes) {
                wk.overflow = true;
                break;
            }
            select_step<F, LAYOUT, PASS, false>(t, q, st, top, cap, io, (int64_t)qi, sg, wk,
                                                PASS == PASS_COUNT && stats != nullptr, lane, grp, sub, lt, lp);
        }
        if (PASS == PASS_COUNT && stats && lane == 0)
            flush_stats(stats, wk, true);
        if (lane == 0) {
            if (wk.overflow)
                atomicOr(flags, FLAG_STACK);
            if (PASS == PASS_COUNT || PASS == PASS_BOUND) {
                io.counts[qi] = (int32_t)wk.cur;
                if (io.counts_leaf)
                    io.counts_leaf[qi] = (int32_t)wk.lcur;
                if (io.counts_rng)
                    io.counts_rng[qi] = (int32_t)wk.rcur;
            } else if (PASS == PASS_SCATTER) {
                if (wk.cur != sg.lim - sg.base)
                    atomicOr(flags, FLAG_COUNT_MISMATCH);
            } else if (io.counts) {  // leaf slots are bounds: report the exact counts
                if (wk.lcur > sg.llim - sg.lbase || wk.rcur != sg.rlim - sg.rbase)
                    atomicOr(flags, FLAG_COUNT_MISMATCH);
                io.counts[qi] = (int32_t)wk.cur;
                io.counts_leaf[qi] = (int32_t)wk.lcur;
            } else {
                if (wk.lcur != sg.llim - sg.lbase || wk.rcur != sg.rlim - sg.rbase)
                    atomicOr(flags, FLAG_COUNT_MISMATCH);
            }
        }
    }
}

// ------------------------------------------------- persistent work queue
// Device work queue of (query, node) items, each published as one 64-bit
// word (query in the low half, node in the high half; all ones = empty).
// Slots [0, Q) start as (q, root); the others are filled by donations.  A
// warp takes a ticket (head++) and waits for that slot to be filled, or for
// `pending` (items not yet finished) to reach zero, which ends the pass.  A
// warp whose stack holds two or more entries while other warps wait
// (head > tail) donates the older half of its stack (the nodes nearest the
// root, i.e. the largest subtrees) to new slots.  pending cannot reach zero
// while a donor runs, because the donor's own item is still pending.  Waits
// are bounded: past kWaitCycles the warp sets FLAG_TIMEOUT and leaves (the
// host reports RTREE_ETIMEOUT).
struct WorkQueue {
    unsigned long long *items;
    long long cap;
    unsigned long long *head;
    unsigned long long *tail;
    long long *pending;
    long long wait_cycles;  // limit of one wait, in GPU clock cycles
};

constexpr unsigned long long kEmpty = ~0ull;
constexpr long long kWaitCycles = 2000000000LL;  // about one second



__device__ __forceinline__ unsigned long long pack_item(int q, int node)
{
    return (unsigned long long)(unsigned)q | ((unsigned long long)(unsigned)node << 32);
}

template <int F, int LAYOUT, int PASS>
__global__ void __launch_bounds__(kThreads)
    k_select_wq(TreeDev t, const float4 *__restrict__ queries, int64_t Q, SelIO io, WorkQueue wq,
                int32_t *__restrict__ flags, int cap, unsigned long long *__restrict__ stats)
{
    constexpr int G = F < 32 ? F : 32;
    extern __shared__ int32_t smem[];
    const int lane = threadIdx.x & 31;
    int32_t *st = smem + (threadIdx.x >> 5) * cap;
    const int grp = lane / G, sub = lane % G;
    const unsigned lt = lanemask_lt();
    const LeafPart lp{-1, 0, false};  // the work queue keeps leaves on the stack

    for (;;) {
        unsigned long long ticket = 0;
        if (lane == 0)
            ticket = atomicAdd(wq.head, 1ull);
        ticket = __shfl_sync(RT_FULL, ticket, 0);
        if ((long long)ticket >= wq.cap)
            return;
        // wait for the slot to be filled (or for the pass to end)
        unsigned long long word = kEmpty;
        if (lane == 0) {
            const long long t0 = clock64();
            const volatile unsigned long long *slot = wq.items + ticket;
            const volatile long long *pend = wq.pending;
            unsigned ns = 32;
            for (;;) {
                word = *slot;
                if (word != kEmpty)
                    break;
                if (*pend == 0)
                    break;
                if (clock64() - t0 > wq.wait_cycles) {
                    atomicOr(flags, FLAG_TIMEOUT);
                    break;
                }
                __nanosleep(ns);
                if (ns < 2048)
                    ns <<= 1;
            }
            __threadfence();
        }
        word = __shfl_sync(RT_FULL, word, 0);
        if (word == kEmpty)
            return;
        const int64_t qi = (int64_t)(unsigned)(word & 0xffffffffull);
        const int root = (int)(word >> 32);
        const float4 q = __ldg(queries + qi);
        const Seg sg = seg_of(io, PASS, qi);
        Walk wk{0, 0, 0, 0, 0, false};
        if (lane == 0)
            st[0] = root;
        int top = 1;
        __syncwarp();
        int steps = 0;
        while (top > 0) {
            if (++steps > t.nodes) {
                wk.overflow = true;
                break;
            }
            select_step<F, LAYOUT, PASS, true>(t, q, st, top, cap, io, qi, sg, wk,
                                               PASS == PASS_COUNT && stats != nullptr, lane, grp, sub, lt, lp);
            // donate the older half of the stack when other warps are waiting
            if (top >= 2 && (steps & 3) == 0) {
                unsigned long long h = 0, tl = 0;
                if (lane == 0) {
                    h = *reinterpret_cast<volatile unsigned long long *>(wq.head);
                    tl = *reinterpret_cast<volatile unsigned long long *>(wq.tail);
                }
                h = __shfl_sync(RT_FULL, h, 0);
                tl = __shfl_sync(RT_FULL, tl, 0);
                if (h > tl && (long long)tl < wq.cap) {
                    const int give = top / 2;
                    long long pos = 0;
                    if (lane == 0)
                        pos = (long long)atomicAdd(wq.tail, (unsigned long long)give);
                    pos = __shfl_sync(RT_FULL, pos, 0);
                    const long long room = wq.cap - pos;
                    const int n = room <= 0 ? 0 : (room < give ? (int)room : give);
                    if (n > 0) {
                        if (lane == 0)
                            atomicAdd(reinterpret_cast<unsigned long long *>(wq.pending),
                                      (unsigned long long)n);
                        __threadfence();
                        for (int e = lane; e < n; e += 32) {
                            volatile unsigned long long *slot = wq.items + pos + e;
                            *slot = pack_item((int)qi, st[e]);
                        }
                        __syncwarp();
                        // shift the kept entries down, 32 at a time: a chunk is
                        // read before it is written, and later chunks read
                        // strictly higher indices
                        const int keep = top - n;
                        for (int c0 = 0; c0 < keep; c0 += 32) {
                            const int e = c0 + lane;
                            int v = 0;
                            if (e < keep)
                                v = st[n + e];
                            __syncwarp();
                            if (e < keep)
                                st[e] = v;
                            __syncwarp();
                        }
                        top = keep;
                    }
                }
            }
        }
        if (PASS == PASS_COUNT && stats && lane == 0)
            flush_stats(stats, wk, root == 0);
        if (lane == 0) {
            if (wk.overflow)
                atomicOr(flags, FLAG_STACK);
            if (PASS == PASS_COUNT) {
                if (wk.cur)
                    atomicAdd(io.counts + qi, (int)wk.cur);
                if (io.counts_leaf && wk.lcur)
                    atomicAdd(io.counts_leaf + qi, (int)wk.lcur);
                if (io.counts_rng && wk.rcur)
                    atomicAdd(io.counts_rng + qi, (int)wk.rcur);
            }
            __threadfence();
            atomicAdd(reinterpret_cast<unsigned long long *>(wq.pending), ~0ull);  // -1
        }
    }
}

// hold: items counted as pending but never published (0 in normal use).
__global__ void k_wq_init(unsigned long long *__restrict__ items, long long cap, int64_t Q,
                          unsigned long long *__restrict__ ctl, const uint32_t *__restrict__ order,
                          int hold)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < cap;
         i += (long long)gridDim.x * blockDim.x)
        items[i] = i < Q ? pack_item(order ? (int)order[i] : (int)i, 0) : kEmpty;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctl[0] = 0;                        // head
        ctl[1] = (unsigned long long)Q;    // tail
        ctl[2] = (unsigned long long)(Q + hold);  // pending
    }
}

// After a work-queue scatter/descriptor pass: every query's cursors must
// have reached its segment length.
__global__ void k_wq_check(const SelIO io, int pass, int64_t Q, int32_t *__restrict__ flags)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < Q;
         i += (int64_t)gridDim.x * blockDim.x) {
        bool bad;
        if (pass == PASS_SCATTER)
            bad = io.cur_ids[i] != io.offsets[i + 1] - io.offsets[i];
        else
            bad = io.cur_leaf[i] != io.off_leaf[i + 1] - io.off_leaf[i] ||
                  io.cur_rng[i] != io.off_rng[i + 1] - io.off_rng[i];
        if (bad)
            atomicOr(flags, FLAG_COUNT_MISMATCH);
    }
}

using SelectKernel = void (*)(TreeDev, const float4 *, int64_t, SelIO, unsigned long long *,
                              int32_t *, int, unsigned long long *);

template <int F, int LAYOUT>
SelectKernel pick_pass(int pass)
{
    return pass == PASS_COUNT     ? k_select<F, LAYOUT, PASS_COUNT>
           : pass == PASS_SCATTER ? k_select<F, LAYOUT, PASS_SCATTER>
           : pass == PASS_BOUND   ? k_select<F, LAYOUT, PASS_BOUND>
                                  : k_select<F, LAYOUT, PASS_DESC>;
}

template <int F>
SelectKernel pick_layout(int layout, int pass)
{
    return layout == RTREE_LAYOUT_AOS    ? pick_pass<F, RTREE_LAYOUT_AOS>(pass)
           : layout == RTREE_LAYOUT_LOHI ? pick_pass<F, RTREE_LAYOUT_LOHI>(pass)
                                         : pick_pass<F, RTREE_LAYOUT_SOA>(pass);
}

SelectKernel pick(int F, int layout, int pass)
{
    switch (F) {
    case 4: return pick_layout<4>(layout, pass);
    case 8: return pick_layout<8>(layout, pass);
    case 16: return pick_layout<16>(layout, pass);
    case 32: return pick_layout<32>(layout, pass);
    case 64: return pick_layout<64>(layout, pass);
    case 128: return pick_layout<128>(layout, pass);
    default: return nullptr;
    }
}

const char *pass_name(int pass)
{
    return pass == PASS_COUNT     ? "select_count"
           : pass == PASS_SCATTER ? "select_scatter"
           : pass == PASS_BOUND   ? "select_bound"
                                  : "select_desc";
}

rtree_status launch(int pass, const rtree *t, const float4 *q, int64_t Q, const SelIO &io,
                    unsigned long long *ctr, int32_t *flags, cudaStream_t s,
                    unsigned long long *stats = nullptr)
{
    SelectKernel kern = pick(t->fanout, t->layout, pass);
    if (!kern)
        return fail(RTREE_EINVAL, "unsupported fanout %d", t->fanout);
    const int cap = t->levels * (t->fanout > 32 ? t->fanout : 32);
    const size_t smem = (size_t)kWarps * cap * sizeof(int32_t);
    if (smem > 48 * 1024)
        RT_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    RT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem));
    if (per_sm < 1)
        return fail(RTREE_EOVERFLOW, "select kernel does not fit on an SM (%zu B shared)", smem);
    int64_t grid = (int64_t)per_sm * sm_count();
    const int64_t need = (Q + kWarps - 1) / kWarps;
    if (grid > need)
        grid = need;
    KernelTimer kt_(pass_name(pass), s);
    kern<<<(unsigned)grid, kThreads, smem, s>>>(t->view(), q, Q, io, ctr, flags, cap, stats);
    RT_LAUNCH();
    return RTREE_OK;
}

using WqKernel = void (*)(TreeDev, const float4 *, int64_t, SelIO, WorkQueue, int32_t *, int,
                          unsigned long long *);

template <int F, int LAYOUT>
WqKernel pick_wq_pass(int pass)
{
    return pass == PASS_COUNT     ? k_select_wq<F, LAYOUT, PASS_COUNT>
           : pass == PASS_SCATTER ? k_select_wq<F, LAYOUT, PASS_SCATTER>
                                  : k_select_wq<F, LAYOUT, PASS_DESC>;
}

template <int F>
WqKernel pick_wq_layout(int layout, int pass)
{
    return layout == RTREE_LAYOUT_AOS    ? pick_wq_pass<F, RTREE_LAYOUT_AOS>(pass)
           : layout == RTREE_LAYOUT_LOHI ? pick_wq_pass<F, RTREE_LAYOUT_LOHI>(pass)
                                         : pick_wq_pass<F, RTREE_LAYOUT_SOA>(pass);
}

WqKernel pick_wq(int F, int layout, int pass)
{
    switch (F) {
    case 4: return pick_wq_layout<4>(layout, pass);
    case 8: return pick_wq_layout<8>(layout, pass);
    case 16: return pick_wq_layout<16>(layout, pass);
    case 32: return pick_wq_layout<32>(layout, pass);
    case 64: return pick_wq_layout<64>(layout, pass);
    case 128: return pick_wq_layout<128>(layout, pass);
    default: return nullptr;
    }
}

// One pass with the persistent work-queue mapping.  io's per-query outputs
// (counts for COUNT, cursors otherwise) must be zeroed by the caller.
rtree_status launch_wq(int pass, const rtree *t, const float4 *q, int64_t Q, const SelIO &io,
                       int32_t *flags, cudaStream_t s, unsigned long long *stats = nullptr,
                       unsigned long long *ext_items = nullptr, long long ext_cap = 0,
                       unsigned long long *ext_ctl = nullptr)
{
    WqKernel kern = pick_wq(t->fanout, t->layout, pass);
    if (!kern)
        return fail(RTREE_EINVAL, "unsupported fanout %d", t->fanout);
    const int cap = t->levels * (t->fanout > 32 ? t->fanout : 32);
    const size_t smem = (size_t)kWarps * cap * sizeof(int32_t);
    if (smem > 48 * 1024)
        RT_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    RT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem));
    if (per_sm < 1)
        return fail(RTREE_EOVERFLOW, "select kernel does not fit on an SM (%zu B shared)", smem);
    const int64_t grid = (int64_t)per_sm * sm_count();  // persistent: all warps resident
    long long cap_items = ext_cap;
    DevBuf<unsigned long long> items(s), ctl(s);
    unsigned long long *items_p = ext_items, *ctl_p = ext_ctl;
    if (!items_p) {
        cap_items = Q + (Q > (1 << 20) ? Q : (1 << 20));
        RT_TRY(items.alloc(cap_items, "work queue"));
        RT_TRY(ctl.alloc(3, "work queue counters"));
        items_p = items.p;
        ctl_p = ctl.p;
    }
    long long dbg_wait = 0;
    int dbg_hold = 0;
    debug_wq_take(&dbg_wait, &dbg_hold);
    {
        KernelTimer kt_("wq_init", s);
        int64_t b = (cap_items + 255) / 256;
        k_wq_init<<<(unsigned)(b > 65536 ? 65536 : b), 256, 0, s>>>(items_p, cap_items, Q, ctl_p, io.order,
                                                                   dbg_hold ? 1 : 0);
        RT_LAUNCH();
    }
    WorkQueue wq{items_p, cap_items, ctl_p, ctl_p + 1, reinterpret_cast<long long *>(ctl_p + 2),
                 dbg_wait > 0 ? dbg_wait : kWaitCycles};
    {
        KernelTimer kt_(pass == PASS_COUNT ? "select_count" : pass == PASS_SCATTER ? "select_scatter" : "select_desc", s);
        kern<<<(unsigned)grid, kThreads, smem, s>>>(t->view(), q, Q, io, wq, flags, cap, stats);
        RT_LAUNCH();
    }
    if (pass != PASS_COUNT) {
        KernelTimer kt_("wq_check", s);
        int64_t b = (Q + 255) / 256;
        k_wq_check<<<(unsigned)(b > 65536 ? 65536 : b), 256, 0, s>>>(io, pass, Q, flags);
        RT_LAUNCH();
    }
    return RTREE_OK;
}

SelIO unlimited()
{
    SelIO io{};
    io.out_cap = io.leaf_cap = io.rng_cap = INT64_MAX;
    return io;
}

int64_t word64(const uint32_t *w) { return (int64_t)((uint64_t)w[0] | ((uint64_t)w[1] << 32)); }

rtree_status empty_result(int64_t Q, DevBuf<int64_t> &off, cudaStream_t s, rtree_result *res)
{
    RT_CUDA(cudaMemsetAsync(off.p, 0, (Q + 1) * sizeof(int64_t), s));
    DevBuf<int32_t> ids(s);
    RT_TRY(ids.alloc(1, "select ids"));
    res->offsets = off.release();
    res->ids = ids.release();
    return RTREE_OK;
}

// Sorted select, warp per query.  The bound pass stops above the leaves and
// gives each query F leaf-hit slots per intersecting leaf (whole subtrees
// exactly); the descriptor pass fills the slots and reports every query's
// exact counts, whose scan gives the final offsets; the sort reads each
// query's leaf hits from the start of its slots.  Against an exact count
// pass this skips the leaf level once (three quarters of the node visits).
rtree_status range_select_bounded(const rtree *t, const float4 *queries, int64_t Q, int order,
                                  cudaStream_t s, rtree_result *res, DevBuf<int64_t> &off)
{
    DevBuf<int32_t> cnt(s), cnt_leaf(s), cnt_rng(s), flags(s);
    DevBuf<unsigned long long> ctr(s);
    DevBuf<int64_t> off_leaf(s), off_rng(s);
    DevBuf<uint32_t> perm(s);
    RT_TRY(cnt.alloc(Q, "select counts"));
    RT_TRY(cnt_leaf.alloc(Q, "select counts"));
    RT_TRY(cnt_rng.alloc(Q, "select counts"));
    RT_TRY(flags.alloc(2, "select flags"));  // [0] select passes, [1] sort
    RT_TRY(ctr.alloc(2, "select work counters"));
    RT_TRY(off_leaf.alloc(Q + 1, "select offsets"));
    RT_TRY(off_rng.alloc(Q + 1, "select offsets"));
    RT_CUDA(cudaMemsetAsync(flags.p, 0, 2 * sizeof(int32_t), s));
    RT_CUDA(cudaMemsetAsync(ctr.p, 0, 2 * sizeof(unsigned long long), s));
    if (order == RTREE_ORDER_HILBERT) {
        RT_TRY(perm.alloc(Q, "query order"));
        RT_TRY(hilbert_order(t, queries, Q, perm.p, s));
    }
    SelIO io = unlimited();
    io.counts = cnt.p;
    io.counts_leaf = cnt_leaf.p;
    io.counts_rng = cnt_rng.p;
    io.order = perm.p;
    RT_TRY(launch(PASS_BOUND, t, queries, Q, io, ctr.p, flags.p, s));
    RT_TRY(scan_exclusive(cnt_leaf.p, off_leaf.p, Q, s));
    RT_TRY(scan_exclusive(cnt_rng.p, off_rng.p, Q, s));
    // host read 1 of 2: the sizes of the descriptor pass's outputs and the flags
    int64_t h[2] = {0, 0};
    int32_t hflags = 0;
    {
        PostList pl{};
        pl.src[0] = off_leaf.p + Q;
        pl.words[0] = 2;
        pl.at[0] = 0;
        pl.src[1] = off_rng.p + Q;
        pl.words[1] = 2;
        pl.at[1] = 2;
        pl.src[2] = flags.p;
        pl.words[2] = 1;
        pl.at[2] = 4;
        pl.n = 3;
        uint32_t w[5];
        RT_TRY(read_words(pl, s, w, 5));
        h[0] = word64(w);
        h[1] = word64(w + 2);
        hflags = (int32_t)w[4];
    }
    if (hflags)
        return fail(RTREE_EINTERNAL, "select bound pass reported device flags 0x%x", hflags);

    DevBuf<int32_t> leaf(s);
    DevBuf<int2> rng(s);
    RT_TRY(leaf.alloc(h[0], "select leaf hits"));
    RT_TRY(rng.alloc(h[1], "select whole subtrees"));
    SelIO so = unlimited();
    so.off_leaf = off_leaf.p;
    so.off_rng = off_rng.p;
    so.leaf_out = leaf.p;
    so.rng_out = rng.p;
    so.order = perm.p;
    so.counts = cnt.p;            // exact ids per query
    so.counts_leaf = cnt_leaf.p;  // exact leaf hits (the bounds are scanned already)
    RT_TRY(launch(PASS_DESC, t, queries, Q, so, ctr.p + 1, flags.p, s));
    RT_TRY(scan_exclusive(cnt.p, off.p, Q, s));
    // host read 2 of 2: the total (it sizes the result and is returned)
    int64_t total = 0;
    {
        PostList pl{};
        pl.src[0] = off.p + Q;
        pl.words[0] = 2;
        pl.at[0] = 0;
        pl.src[1] = flags.p;
        pl.words[1] = 1;
        pl.at[1] = 2;
        pl.n = 2;
        uint32_t w[3];
        RT_TRY(read_words(pl, s, w, 3));
        total = word64(w);
        if (w[2])
            return fail(RTREE_EINTERNAL, "select descriptor pass reported device flags 0x%x", w[2]);
    }
    DevBuf<int32_t> ids(s);
    RT_TRY(ids.alloc(total, "select ids"));
    SortSources src{};
    src.leaf = leaf.p;
    src.off_leaf = off_leaf.p;
    src.leaf_len = cnt_leaf.p;
    src.rng = rng.p;
    src.off_rng = off_rng.p;
    src.tree_ids = t->ids;
    RT_TRY(segmented_sort_gather(ids.p, off.p, Q, total, src, s, flags.p + 1));
    // the sort runs on in the order of s; its flags reach the result's status
    RT_TRY(post_result_status(flags.p, s, res));
    res->total = total;
    res->offsets = off.release();
    res->ids = ids.release();
    return RTREE_OK;
}

}  // namespace

rtree_status range_select(const rtree *t, const float4 *queries, int64_t Q, bool sorted,
                          int mapping, int order, cudaStream_t s, rtree_result *res)
{
    const bool wq = mapping == RTREE_MAP_WORK_QUEUE;
    res->rows = Q;
    res->total = 0;
    DevBuf<int64_t> off(s);
    RT_TRY(off.alloc(Q + 1, "select offsets"));
    if (Q == 0 || t->nodes == 0)
        return empty_result(Q, off, s, res);
    if (!pick(t->fanout, t->layout, PASS_COUNT))
        return fail(RTREE_EINVAL, "unsupported fanout %d", t->fanout);
    if (sorted && !wq)
        return range_select_bounded(t, queries, Q, order, s, res, off);

    DevBuf<int32_t> cnt(s), cnt_leaf(s), cnt_rng(s), flags(s);
    DevBuf<unsigned long long> ctr(s);
    RT_TRY(cnt.alloc(Q, "select counts"));
    RT_TRY(flags.alloc(2, "select flags"));  // [0] select passes, [1] sort
    RT_TRY(ctr.alloc(2, "select work counters"));
    RT_CUDA(cudaMemsetAsync(flags.p, 0, 2 * sizeof(int32_t), s));
    RT_CUDA(cudaMemsetAsync(ctr.p, 0, 2 * sizeof(unsigned long long), s));
    DevBuf<uint32_t> perm(s);
    if (order == RTREE_ORDER_HILBERT) {
        RT_TRY(perm.alloc(Q, "query order"));
        RT_TRY(hilbert_order(t, queries, Q, perm.p, s));
    }
    SelIO io = unlimited();
    io.counts = cnt.p;
    io.order = perm.p;
    if (sorted) {
        RT_TRY(cnt_leaf.alloc(Q, "select counts"));
        RT_TRY(cnt_rng.alloc(Q, "select counts"));
        io.counts_leaf = cnt_leaf.p;
        io.counts_rng = cnt_rng.p;
    }
    if (wq) {  // several warps add into one query's counts
        RT_CUDA(cudaMemsetAsync(cnt.p, 0, Q * sizeof(int32_t), s));
        if (sorted) {
            RT_CUDA(cudaMemsetAsync(cnt_leaf.p, 0, Q * sizeof(int32_t), s));
            RT_CUDA(cudaMemsetAsync(cnt_rng.p, 0, Q * sizeof(int32_t), s));
        }
        RT_TRY(launch_wq(PASS_COUNT, t, queries, Q, io, flags.p, s));
    } else {
        RT_TRY(launch(PASS_COUNT, t, queries, Q, io, ctr.p, flags.p, s));
    }
    RT_TRY(scan_exclusive(cnt.p, off.p, Q, s));
    DevBuf<int64_t> off_leaf(s), off_rng(s);
    if (sorted) {
        RT_TRY(off_leaf.alloc(Q + 1, "select offsets"));
        RT_TRY(off_rng.alloc(Q + 1, "select offsets"));
        RT_TRY(scan_exclusive(cnt_leaf.p, off_leaf.p, Q, s));
        RT_TRY(scan_exclusive(cnt_rng.p, off_rng.p, Q, s));
    }
    // the one host read: the total, the descriptor sizes and the flags
    int64_t h[3] = {0, 0, 0};
    int32_t hflags = 0;
    {
        PostList pl{};
        pl.src[0] = off.p + Q;
        pl.words[0] = 2;
        pl.at[0] = 0;
        pl.src[1] = flags.p;
        pl.words[1] = 1;
        pl.at[1] = 2;
        pl.n = 2;
        if (sorted) {
            pl.src[2] = off_leaf.p + Q;
            pl.words[2] = 2;
            pl.at[2] = 3;
            pl.src[3] = off_rng.p + Q;
            pl.words[3] = 2;
            pl.at[3] = 5;
            pl.n = 4;
        }
        uint32_t w[7] = {};
        RT_TRY(read_words(pl, s, w, sorted ? 7 : 3));
        h[0] = word64(w);
        hflags = (int32_t)w[2];
        if (sorted) {
            h[1] = word64(w + 3);
            h[2] = word64(w + 5);
        }
    }
    if (hflags & FLAG_TIMEOUT)
        return fail(RTREE_ETIMEOUT, "select count pass: a work-queue wait exceeded its limit");
    if (hflags)
        return fail(RTREE_EINTERNAL, "select count pass reported device flags 0x%x", hflags);
    const int64_t total = h[0];
    DevBuf<int32_t> cursors(s);
    if (wq) {
        RT_TRY(cursors.alloc(2 * Q, "select cursors"));
        RT_CUDA(cudaMemsetAsync(cursors.p, 0, 2 * Q * sizeof(int32_t), s));
    }

    DevBuf<int32_t> ids(s);
    RT_TRY(ids.alloc(total, "select ids"));
    if (!sorted) {
        SelIO so = unlimited();
        so.offsets = off.p;
        so.out = ids.p;
        so.order = perm.p;
        if (wq) {
            so.cur_ids = cursors.p;
            RT_TRY(launch_wq(PASS_SCATTER, t, queries, Q, so, flags.p, s));
        } else {
            RT_TRY(launch(PASS_SCATTER, t, queries, Q, so, ctr.p + 1, flags.p, s));
        }
    } else {
        DevBuf<int32_t> leaf(s);
        DevBuf<int2> rng(s);
        RT_TRY(leaf.alloc(h[1], "select leaf hits"));
        RT_TRY(rng.alloc(h[2], "select whole subtrees"));
        SelIO so = unlimited();
        so.off_leaf = off_leaf.p;
        so.off_rng = off_rng.p;
        so.leaf_out = leaf.p;
        so.rng_out = rng.p;
        so.order = perm.p;
        if (wq) {
            so.cur_leaf = cursors.p;
            so.cur_rng = cursors.p + Q;
            RT_TRY(launch_wq(PASS_DESC, t, queries, Q, so, flags.p, s));
        } else {
            RT_TRY(launch(PASS_DESC, t, queries, Q, so, ctr.p + 1, flags.p, s));
        }
        SortSources src{};
        src.leaf = leaf.p;
        src.off_leaf = off_leaf.p;
        src.rng = rng.p;
        src.off_rng = off_rng.p;
        src.tree_ids = t->ids;
        RT_TRY(segmented_sort_gather(ids.p, off.p, Q, total, src, s, flags.p + 1));
    }
    // the second pass (and sort) run on in the order of s; their flags reach
    // the result's status
    RT_TRY(post_result_status(flags.p, s, res));
    res->total = total;
    res->offsets = off.release();
    res->ids = ids.release();
    return RTREE_OK;
}

// Results in host memory.  One count pass over the whole batch fixes the
// offsets; a small device kernel cuts the batch into chunks of about equal
// id counts and posts the totals and chunk bounds to a mailbox (so the host
// reads them without waiting behind copies still queued by earlier calls).
// Each chunk's second pass (descriptors, then the segmented sort; or the
// scatter pass unsorted) runs on `s`, and when it is done its ids are copied
// to the caller's buffer on a stream of the call's own while the next chunk
// runs; the offsets go first on that stream.  Chunks of about 128M ids (at
// most 32 of them) balance the exposed ends (the first chunk's select, the
// last chunk's copy) against per-chunk launch costs.  The call returns once
// everything is enqueued; range_select_host_finish waits for the copies.
constexpr int kHostMaxChunks = 32;
constexpr int64_t kHostChunkIds = int64_t(128) << 20;

// Mailbox layout of the count pass's summary (int64 words).
enum { MB_TOTAL = 0, MB_LEAF, MB_RNG, MB_FLAGS, MB_CHUNKS, MB_BOUND,
       MB_BOFF = MB_BOUND + kHostMaxChunks + 1, MB_WORDS = MB_BOFF + kHostMaxChunks + 1 };
static_assert(2 * MB_WORDS <= kMailboxWords, "mailbox too small");

// Thread k finds chunk bound k: the first query whose ids start at or after
// k * total / chunks (a lower bound over the offsets).
__global__ void k_chunk_plan(const int64_t *__restrict__ off, const int64_t *__restrict__ off_leaf,
                             const int64_t *__restrict__ off_rng, const int32_t *__restrict__ flags,
                             int64_t Q, int64_t *__restrict__ mb)
{
    const int64_t total = off[Q];
    int64_t nc = total / kHostChunkIds + 1;
    nc = nc < kHostMaxChunks ? nc : kHostMaxChunks;
    nc = nc < Q ? nc : Q;
    const int k = threadIdx.x;
    if (k == 0) {
        mb[MB_TOTAL] = total;
        mb[MB_LEAF] = off_leaf ? off_leaf[Q] : 0;
        mb[MB_RNG] = off_rng ? off_rng[Q] : 0;
        mb[MB_FLAGS] = flags[0];
        mb[MB_CHUNKS] = nc;
    }
    if (k <= nc) {
        int64_t b = Q;
        if (k == 0) {
            b = 0;
        } else if (k < nc) {
            const int64_t want = total / nc * k;
            int64_t lo = 0, hi = Q;
            while (lo < hi) {
                const int64_t mid = lo + (hi - lo) / 2;
                if (off[mid] < want)
                    lo = mid + 1;
                else
                    hi = mid;
            }
            b = lo;
        }
        mb[MB_BOUND + k] = b;
        mb[MB_BOFF + k] = off[b];
    }
}

rtree_status range_select_host_begin(const rtree *t, const float4 *queries, int64_t Q, bool sorted,
                                     int mapping, int order, cudaStream_t s, int64_t *h_off,
                                     int32_t *h_ids, int64_t capacity, int64_t *h_total,
                                     rtree_pending **pending)
{
    *pending = nullptr;
    *h_total = 0;
    if (Q == 0 || t->nodes == 0) {
        memset(h_off, 0, (size_t)(Q + 1) * sizeof(int64_t));
        return RTREE_OK;
    }
    if (!pick(t->fanout, t->layout, PASS_COUNT))
        return fail(RTREE_EINVAL, "unsupported fanout %d", t->fanout);
    const bool wq = mapping == RTREE_MAP_WORK_QUEUE;
    DevBuf<int32_t> cnt(s), cnt_leaf(s), cnt_rng(s), flags(s);
    DevBuf<unsigned long long> ctr(s);
    DevBuf<int64_t> off(s), off_leaf(s), off_rng(s);
    DevBuf<uint32_t> perm(s);
    RT_TRY(cnt.alloc(Q, "select counts"));
    RT_TRY(off.alloc(Q + 1, "select offsets"));
    RT_TRY(flags.alloc(2, "select flags"));
    RT_TRY(ctr.alloc(1 + kHostMaxChunks, "select work counters"));
    RT_CUDA(cudaMemsetAsync(flags.p, 0, 2 * sizeof(int32_t), s));
    RT_CUDA(cudaMemsetAsync(ctr.p, 0, (1 + kHostMaxChunks) * sizeof(unsigned long long), s));
    if (order == RTREE_ORDER_HILBERT) {
        RT_TRY(perm.alloc(Q, "query order"));
        RT_TRY(hilbert_order(t, queries, Q, perm.p, s));
    }
    SelIO io = unlimited();
    io.counts = cnt.p;
    io.order = perm.p;
    if (sorted) {
        RT_TRY(cnt_leaf.alloc(Q, "select counts"));
        RT_TRY(cnt_rng.alloc(Q, "select counts"));
        RT_TRY(off_leaf.alloc(Q + 1, "select offsets"));
        RT_TRY(off_rng.alloc(Q + 1, "select offsets"));
        io.counts_leaf = cnt_leaf.p;
        io.counts_rng = cnt_rng.p;
    }
    if (wq) {
        RT_CUDA(cudaMemsetAsync(cnt.p, 0, Q * sizeof(int32_t), s));
        if (sorted) {
            RT_CUDA(cudaMemsetAsync(cnt_leaf.p, 0, Q * sizeof(int32_t), s));
            RT_CUDA(cudaMemsetAsync(cnt_rng.p, 0, Q * sizeof(int32_t), s));
        }
        RT_TRY(launch_wq(PASS_COUNT, t, queries, Q, io, flags.p, s));
    } else {
        RT_TRY(launch(PASS_COUNT, t, queries, Q, io, ctr.p, flags.p, s));
    }
    RT_TRY(scan_exclusive(cnt.p, off.p, Q, s));
    if (sorted) {
        RT_TRY(scan_exclusive(cnt_leaf.p, off_leaf.p, Q, s));
        RT_TRY(scan_exclusive(cnt_rng.p, off_rng.p, Q, s));
    }
    MailboxRef plan;
    RT_TRY(mailbox_get(&plan.m));
    int64_t *mbd = reinterpret_cast<int64_t *>(plan.m.d);
    k_chunk_plan<<<1, 64, 0, s>>>(off.p, sorted ? off_leaf.p : nullptr, sorted ? off_rng.p : nullptr,
                                  flags.p, Q, mbd);
    RT_LAUNCH();
    RT_CUDA(cudaEventRecord(plan.m.ev, s));
    RT_TRY(mailbox_wait(plan.m));
    const volatile int64_t *mb = reinterpret_cast<const volatile int64_t *>(plan.m.h);
    const int32_t hflags = (int32_t)mb[MB_FLAGS];
    if (hflags & FLAG_TIMEOUT)
        return fail(RTREE_ETIMEOUT, "select count pass: a work-queue wait exceeded its limit");
    if (hflags)
        return fail(RTREE_EINTERNAL, "select count pass reported device flags 0x%x", hflags);
    const int64_t total = mb[MB_TOTAL];
    *h_total = total;
    if (total > capacity || total == 0) {  // the offsets are the whole answer
        RT_CUDA(cudaMemcpyAsync(h_off, off.p, (Q + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        RT_CUDA(cudaStreamSynchronize(s));
        if (total > capacity)
            return fail(RTREE_EOVERFLOW, "rtree_range_select_host: %lld ids, capacity %lld",
                        (long long)total, (long long)capacity);
        return RTREE_OK;
    }
    const int kChunks = (int)mb[MB_CHUNKS];
    int64_t bound[kHostMaxChunks + 1], boff[kHostMaxChunks + 1];
    if (kChunks < 1 || kChunks > kHostMaxChunks)
        return fail(RTREE_EINTERNAL, "select: bad chunk count %d", kChunks);
    for (int k = 0; k <= kChunks; ++k) {
        bound[k] = mb[MB_BOUND + k];
        boff[k] = mb[MB_BOFF + k];
    }
    const int64_t leaf_total = mb[MB_LEAF], rng_total = mb[MB_RNG];

    DevBuf<int32_t> ids(s), cursors(s), leaf(s);
    DevBuf<int2> rng(s);
    DevBuf<uint32_t> cperm(s);
    RT_TRY(ids.alloc(total, "select ids"));
    if (sorted) {
        RT_TRY(leaf.alloc(leaf_total, "select leaf hits"));
        RT_TRY(rng.alloc(rng_total, "select whole subtrees"));
    }
    if (wq) {
        RT_TRY(cursors.alloc(2 * Q, "select cursors"));
        RT_CUDA(cudaMemsetAsync(cursors.p, 0, 2 * Q * sizeof(int32_t), s));
    }
    int64_t max_chunk = 0;
    for (int k = 0; k < kChunks; ++k)
        max_chunk = bound[k + 1] - bound[k] > max_chunk ? bound[k + 1] - bound[k] : max_chunk;
    if (order == RTREE_ORDER_HILBERT)
        RT_TRY(cperm.alloc(max_chunk, "query order"));

    struct Pending {  // owns the in-flight state until it is handed out
        rtree_pending *p = new rtree_pending();
        ~Pending()
        {
            if (p)
                range_select_host_finish(p);
        }
    } pd;
    rtree_pending *p = pd.p;
    p->device = t->device;
    p->alloc = t->alloc;
    p->custom_alloc = t->custom_alloc;
    RT_CUDA(cudaStreamCreateWithFlags(&p->cs, cudaStreamNonBlocking));
    for (int k = 0; k <= kChunks; ++k)
        RT_CUDA(cudaEventCreateWithFlags(&p->ev[k], cudaEventDisableTiming));
    RT_TRY(mailbox_get(&p->flags));
    // the offsets, then each chunk's ids, go to the host on the call's stream
    RT_CUDA(cudaEventRecord(p->ev[kChunks], s));
    RT_CUDA(cudaStreamWaitEvent(p->cs, p->ev[kChunks], 0));
    RT_CUDA(cudaMemcpyAsync(h_off, off.p, (Q + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, p->cs));
    for (int k = 0; k < kChunks; ++k) {
        const int64_t c0 = bound[k], qc = bound[k + 1] - bound[k];
        if (qc == 0)
            continue;
        const float4 *qk = queries + c0;
        SelIO so = unlimited();
        if (order == RTREE_ORDER_HILBERT) {
            RT_TRY(hilbert_order(t, qk, qc, cperm.p, s));
            so.order = cperm.p;
        }
        if (!sorted) {
            so.offsets = off.p + c0;
            so.out = ids.p;
            if (wq) {
                so.cur_ids = cursors.p + c0;
                RT_TRY(launch_wq(PASS_SCATTER, t, qk, qc, so, flags.p, s));
            } else {
                RT_TRY(launch(PASS_SCATTER, t, qk, qc, so, ctr.p + 1 + k, flags.p, s));
            }
        } else {
            so.off_leaf = off_leaf.p + c0;
            so.off_rng = off_rng.p + c0;
            so.leaf_out = leaf.p;
            so.rng_out = rng.p;
            if (wq) {
                so.cur_leaf = cursors.p + c0;
                so.cur_rng = cursors.p + Q + c0;
                RT_TRY(launch_wq(PASS_DESC, t, qk, qc, so, flags.p, s));
            } else {
                RT_TRY(launch(PASS_DESC, t, qk, qc, so, ctr.p + 1 + k, flags.p, s));
            }
            SortSources src{};
            src.leaf = leaf.p;
            src.off_leaf = off_leaf.p + c0;
            src.rng = rng.p;
            src.off_rng = off_rng.p + c0;
            src.tree_ids = t->ids;
            RT_TRY(segmented_sort_gather(ids.p, off.p + c0, qc, boff[k + 1] - boff[k], src, s,
                                         flags.p + 1, total));
        }
        const int64_t a = boff[k], b = boff[k + 1];
        RT_CUDA(cudaEventRecord(p->ev[k], s));
        RT_CUDA(cudaStreamWaitEvent(p->cs, p->ev[k], 0));
        if (b > a)
            RT_CUDA(cudaMemcpyAsync(h_ids + a, ids.p + a, (b - a) * sizeof(int32_t), cudaMemcpyDeviceToHost,
                                    p->cs));
    }
    PostList fl{};
    fl.src[0] = flags.p;
    fl.words[0] = 2;
    fl.at[0] = 0;
    fl.n = 1;
    RT_TRY(mailbox_post(p->flags, fl, s));
    p->ids = ids.release();
    p->off = off.release();
    pd.p = nullptr;
    *pending = p;
    return RTREE_OK;
}

rtree_status range_select_host_finish(rtree_pending *p)
{
    DeviceGuard guard(p->device);
    cudaError_t e = cudaSuccess;
    if (p->cs)
        e = cudaStreamSynchronize(p->cs);
    int32_t hf[2] = {0, 0};
    if (p->flags.h) {
        const cudaError_t e2 = cudaEventSynchronize(p->flags.ev);
        e = e != cudaSuccess ? e : e2;
        const volatile int32_t *f = reinterpret_cast<const volatile int32_t *>(p->flags.h);
        hf[0] = f[0];
        hf[1] = f[1];
    }
    if (p->cs) {
        AllocScope scope(p->custom_alloc ? &p->alloc : nullptr);
        dfree(p->ids, p->cs);
        dfree(p->off, p->cs);
        cudaStreamDestroy(p->cs);
    }
    for (auto ev : p->ev)
        if (ev)
            cudaEventDestroy(ev);
    mailbox_put(&p->flags);
    delete p;
    if (e != cudaSuccess)
        return fail(RTREE_ECUDA, "host-result select: %s", cudaGetErrorString(e));
    if (hf[1])
        return fail(RTREE_EINTERNAL, "segmented sort reported device flags 0x%x", hf[1]);
    if (hf[0] & FLAG_TIMEOUT)
        return fail(RTREE_ETIMEOUT, "select second pass: a work-queue wait exceeded its limit");
    if (hf[0])
        return fail(RTREE_EINTERNAL, "select second pass reported device flags 0x%x", hf[0]);
    return RTREE_OK;
}

rtree_status select_enqueue(const rtree *t, const float4 *queries, int64_t Q, int mapping,
                            const SelectBuffers &b, cudaStream_t s)
{
    const bool wq = mapping == RTREE_MAP_WORK_QUEUE;
    RT_CUDA(cudaMemsetAsync(b.flags, 0, 2 * sizeof(int32_t), s));
    RT_CUDA(cudaMemsetAsync(b.ctr, 0, 2 * sizeof(unsigned long long), s));
    if (Q == 0 || t->nodes == 0) {
        RT_CUDA(cudaMemsetAsync(b.off, 0, (Q + 1) * sizeof(int64_t), s));
        RT_CUDA(cudaMemsetAsync(b.off_leaf, 0, (Q + 1) * sizeof(int64_t), s));
        RT_CUDA(cudaMemsetAsync(b.off_rng, 0, (Q + 1) * sizeof(int64_t), s));
        return RTREE_OK;
    }
    SelIO io = unlimited();
    io.counts = b.cnt;
    io.counts_leaf = b.cnt_leaf;
    io.counts_rng = b.cnt_rng;
    if (wq) {
        RT_CUDA(cudaMemsetAsync(b.cnt, 0, Q * sizeof(int32_t), s));
        RT_CUDA(cudaMemsetAsync(b.cnt_leaf, 0, Q * sizeof(int32_t), s));
        RT_CUDA(cudaMemsetAsync(b.cnt_rng, 0, Q * sizeof(int32_t), s));
        RT_TRY(launch_wq(PASS_COUNT, t, queries, Q, io, b.flags, s, nullptr, b.wq_items, b.wq_cap,
                         b.wq_ctl));
    } else {
        // warp per query: the bound pass (stopped above the leaves) sizes the
        // leaf-hit slots; the descriptor pass reports the exact counts
        RT_TRY(launch(PASS_BOUND, t, queries, Q, io, b.ctr, b.flags, s));
    }
    if (wq)
        RT_TRY(scan_exclusive(b.cnt, b.off, Q, s));
    RT_TRY(scan_exclusive(b.cnt_leaf, b.off_leaf, Q, s));
    RT_TRY(scan_exclusive(b.cnt_rng, b.off_rng, Q, s));
    SelIO so = unlimited();
    so.off_leaf = b.off_leaf;
    so.off_rng = b.off_rng;
    so.leaf_out = b.leaf;
    so.rng_out = b.rng;
    so.leaf_cap = b.leaf_cap;
    so.rng_cap = b.rng_cap;
    if (wq) {
        RT_CUDA(cudaMemsetAsync(b.cursors, 0, 2 * Q * sizeof(int32_t), s));
        so.cur_leaf = b.cursors;
        so.cur_rng = b.cursors + Q;
        RT_TRY(launch_wq(PASS_DESC, t, queries, Q, so, b.flags, s, nullptr, b.wq_items, b.wq_cap,
                         b.wq_ctl));
    } else {
        so.counts = b.cnt;            // exact ids per query
        so.counts_leaf = b.cnt_leaf;  // exact leaf hits (the slot bounds are scanned already)
        RT_TRY(launch(PASS_DESC, t, queries, Q, so, b.ctr + 1, b.flags, s));
        RT_TRY(scan_exclusive(b.cnt, b.off, Q, s));
    }
    SortSources src{};
    src.leaf = b.leaf;
    src.off_leaf = b.off_leaf;
    src.leaf_len = wq ? nullptr : b.cnt_leaf;
    src.rng = b.rng;
    src.off_rng = b.off_rng;
    src.tree_ids = t->ids;
    src.leaf_cap = b.leaf_cap;
    src.rng_cap = b.rng_cap;
    return segmented_sort_gather(b.ids, b.off, Q, b.ids_cap, src, s, b.flags + 1);
}

rtree_status select_pass(const rtree *t, const float4 *queries, int64_t Q, int32_t *counts,
                         const int64_t *offsets, int32_t *out, unsigned long long *ctr,
                         int32_t *flags, cudaStream_t s)
{
    SelIO io = unlimited();
    io.counts = counts;
    io.offsets = offsets;
    io.out = out;
    return launch(counts ? PASS_COUNT : PASS_SCATTER, t, queries, Q, io, ctr, flags, s);
}

rtree_status select_stats(const rtree *t, const float4 *queries, int64_t Q, cudaStream_t s,
                          int64_t out[8])
{
    for (int i = 0; i < 8; ++i)
        out[i] = 0;
    out[0] = Q;
    if (Q == 0 || t->nodes == 0)
        return RTREE_OK;
    DevBuf<int32_t> cnt(s), flags(s);
    DevBuf<unsigned long long> ctr(s), st(s);
    RT_TRY(cnt.alloc(Q, "select counts"));
    RT_TRY(flags.alloc(1, "select flags"));
    RT_TRY(ctr.alloc(1, "select work counter"));
    RT_TRY(st.alloc(8, "select statistics"));
    RT_CUDA(cudaMemsetAsync(flags.p, 0, sizeof(int32_t), s));
    RT_CUDA(cudaMemsetAsync(ctr.p, 0, sizeof(unsigned long long), s));
    RT_CUDA(cudaMemsetAsync(st.p, 0, 8 * sizeof(unsigned long long), s));
    SelIO io = unlimited();
    io.counts = cnt.p;
    RT_TRY(launch(PASS_COUNT, t, queries, Q, io, ctr.p, flags.p, s, st.p));
    unsigned long long h[8];
    RT_CUDA(cudaMemcpyAsync(h, st.p, sizeof(h), cudaMemcpyDeviceToHost, s));
    RT_CUDA(cudaStreamSynchronize(s));
    for (int i = 0; i < 6; ++i)
        out[i] = (int64_t)h[i];
    return RTREE_OK;
}

}  // namespace rt
