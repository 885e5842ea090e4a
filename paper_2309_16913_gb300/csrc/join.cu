// join.cu -- R-tree join (Section 4), synchronized top-down traversal.
//
// Both trees are walked from their roots together (Brinkhoff, Kriegel and
// Seeger 1993): a node pair (a, b) whose entries intersect yields child
// pairs, and leaf pairs yield (r_id, s_id).  The frontier is processed one
// level at a time; every node pair is tested by one warp with the
// one-to-many comparison of Section 4.1: the inner node's children sit one
// per lane (G = min(32, F_s) lanes per outer child, so 32/G outer children
// are tested per step), each outer child's MBR is broadcast to its lanes,
// and __ballot_sync over the four comparisons gives the qualifying inner
// children, compacted with popc(mask & lanemask_lt) (queue insertion, step 4).
// Where the heights differ, only the taller tree descends: its children are
// tested against the other node's bounding box.
//
// For trees whose node entries ascend by lx, equal-height pairs can use the
// prunings of Section 4.2 instead (k_join_pruned): O3 ends the outer loop at
// the first outer child whose lx lies right of every inner child, and O4/O5
// bound each outer child's inner scan by the number f of inner children that
// start left of its hx, found by the batched search of the many-to-many
// comparison.  The f candidate pairs of all lanes are then packed densely
// onto the warp, so a node pair costs ceil(sum f / 32) tests instead of one
// per outer child.
//
// Output is written in two passes per level (count, scan, scatter).  The
// final (r_id, s_id) pairs are sorted lexicographically by two stable radix
// sorts (by s, then by r).
#include <algorithm>

#include "internal.cuh"

namespace rt {
namespace {

enum { J_BOTH = 0, J_A = 1, J_B = 2, J_LEAF = 3 };
enum { PASS_COUNT = 0, PASS_SCATTER = 1 };
constexpr int kThreads = 256;
constexpr uint32_t kSign = 0x80000000u;

template <int MODE, int PASS>
__global__ void __launch_bounds__(kThreads)
    k_join(TreeDev ta, TreeDev tb, const int2 *__restrict__ pairs, int64_t np,
           int32_t *__restrict__ counts, const int64_t *__restrict__ offs, int2 *__restrict__ out)
{
    const int lane = threadIdx.x & 31;
    const unsigned lt = lanemask_lt();
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int Fa = ta.fanout, Fb = tb.fanout;
    for (int64_t p = warp; p < np; p += nwarps) {
        const int2 pr = pairs[p];
        const int a = pr.x, b = pr.y;
        const int4 ma = __ldg(ta.meta + a), mb = __ldg(tb.meta + b);
        int64_t base = 0;
        if (PASS == PASS_SCATTER)
            base = offs[p];
        int cur = 0;
        if (MODE == J_A) {
            const float4 bb = __ldg(tb.nbox + b);
            for (int i0 = 0; i0 < ma.y; i0 += 32) {
                const int i = i0 + lane;
                const bool hit = i < ma.y && meets(load_entry(ta.mbr, ta.layout, Fa, a, i), bb);
                const unsigned m = __ballot_sync(RT_FULL, hit);
                if (PASS == PASS_SCATTER && hit)
                    out[base + cur + __popc(m & lt)] = make_int2(ma.x + i, b);
                cur += __popc(m);
            }
        } else if (MODE == J_B) {
            const float4 ab = __ldg(ta.nbox + a);
            for (int j0 = 0; j0 < mb.y; j0 += 32) {
                const int j = j0 + lane;
                const bool hit = j < mb.y && meets(ab, load_entry(tb.mbr, tb.layout, Fb, b, j));
                const unsigned m = __ballot_sync(RT_FULL, hit);
                if (PASS == PASS_SCATTER && hit)
                    out[base + cur + __popc(m & lt)] = make_int2(a, mb.x + j);
                cur += __popc(m);
            }
        } else {
            const int G = Fb < 32 ? Fb : 32;
            const int KO = 32 / G;
            const int grp = lane / G, sub = lane % G;
            for (int j0 = 0; j0 < mb.y; j0 += G) {
                const int j = j0 + sub;
                const bool vj = j < mb.y;
                const float4 ib = vj ? load_entry(tb.mbr, tb.layout, Fb, b, j) : empty_box();
                for (int i0 = 0; i0 < ma.y; i0 += KO) {
                    const int i = i0 + grp;
                    const bool vi = i < ma.y;
                    const float4 ob = vi ? load_entry(ta.mbr, ta.layout, Fa, a, i) : empty_box();
                    const bool hit = vi && vj && meets(ob, ib);
                    const unsigned m = __ballot_sync(RT_FULL, hit);
                    if (PASS == PASS_SCATTER && hit) {
                        int2 v;
                        if (MODE == J_LEAF)
                            v = make_int2(__ldg(ta.ids + ma.x + i), __ldg(tb.ids + mb.x + j));
                        else
                            v = make_int2(ma.x + i, mb.x + j);
                        out[base + cur + __popc(m & lt)] = v;
                    }
                    cur += __popc(m);
                }
            }
        }
        if (PASS == PASS_COUNT && lane == 0)
            counts[p] = cur;
    }
}

constexpr int kMaxFanout = 128;

__device__ __forceinline__ float entry_lx(const TreeDev &t, int64_t g, int j)
{
    if (t.layout == RTREE_LAYOUT_AOS)
        return __ldg(reinterpret_cast<const float *>(t.mbr) + (g * t.fanout + j) * 4);
    if (t.layout == RTREE_LAYOUT_LOHI)
        return __ldg(t.mbr + g * 4 * t.fanout + 2 * j);
    return __ldg(t.mbr + g * 4 * t.fanout + j);
}

// Equal-height node pairs of two sorted-children trees, one pair per warp.
template <bool LEAF, int PASS>
__global__ void __launch_bounds__(kThreads)
    k_join_pruned(TreeDev ta, TreeDev tb, const int2 *__restrict__ pairs, int64_t np,
                  int32_t *__restrict__ counts, const int64_t *__restrict__ offs,
                  int2 *__restrict__ out)
{
    __shared__ float s_lx[kThreads / 32][kMaxFanout];
    const int lane = threadIdx.x & 31;
    const unsigned lt = lanemask_lt();
    float *lxs = s_lx[threadIdx.x >> 5];
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t p = warp; p < np; p += nwarps) {
        const int2 pr = pairs[p];
        const int a = pr.x, b = pr.y;
        const int4 ma = __ldg(ta.meta + a), mb = __ldg(tb.meta + b);
        const float4 bb = __ldg(tb.nbox + b);  // inner node MBR: max over children of hx is bb.z
        const int nin = mb.y;
        int64_t base = 0;
        if (PASS == PASS_SCATTER)
            base = offs[p];
        __syncwarp();  // the previous pair's searches are done with lxs
        for (int j = lane; j < nin; j += 32)
            lxs[j] = entry_lx(tb, b, j);
        __syncwarp();
        int P2 = 1, rounds = 1;  // inner count rounded up to a power of two; log2(P2)+1 rounds
        while (P2 < nin) {
            P2 <<= 1;
            ++rounds;
        }
        int cur = 0;
        for (int i0 = 0; i0 < ma.y; i0 += 32) {
            const int i = i0 + lane;
            const bool vi = i < ma.y;
            const float4 ob = vi ? load_entry(ta.mbr, ta.layout, ta.fanout, a, i) : empty_box();
            const bool keyok = vi && ob.x <= bb.z;   // O3 key test against all inner children
            const bool cand = keyok && meets(ob, bb);  // search-space restriction
            int f = 0;
            if (cand) {  // O5: first inner index whose lx exceeds ob.hx
                int g = P2 >> 1, step = (P2 >> 2) > 1 ? (P2 >> 2) : 1;
                f = nin;
                for (int r = 0; r < rounds; ++r) {
                    const bool pass = g < nin && ob.z >= lxs[g];
                    if (!pass && g < f)
                        f = g;
                    g = pass ? g + step : g - step;
                    step = (step >> 1) > 1 ? (step >> 1) : 1;
                }
            }
            int incl = f;  // inclusive scan of the bounds over the lanes
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int u = __shfl_up_sync(RT_FULL, incl, o);
                if (lane >= o)
                    incl += u;
            }
            const int excl = incl - f;
            const int T = __shfl_sync(RT_FULL, incl, 31);
            for (int k0 = 0; k0 < T; k0 += 32) {
                const int k = k0 + lane;
                int own = 0;  // the lane whose run [excl, incl) holds k
#pragma unroll
                for (int st = 16; st > 0; st >>= 1) {
                    const int v = __shfl_sync(RT_FULL, incl, own + st - 1);
                    if (v <= k)
                        own += st;
                }
                const int ex = __shfl_sync(RT_FULL, excl, own);
                const float4 o = make_float4(__shfl_sync(RT_FULL, ob.x, own),
                                             __shfl_sync(RT_FULL, ob.y, own),
                                             __shfl_sync(RT_FULL, ob.z, own),
                                             __shfl_sync(RT_FULL, ob.w, own));
                const int j = k - ex;
                bool hit = false;
                if (k < T)
                    hit = meets(o, load_entry(tb.mbr, tb.layout, tb.fanout, b, j));
                const unsigned m = __ballot_sync(RT_FULL, hit);
                if (PASS == PASS_SCATTER && hit) {
                    const int io = i0 + own;
                    int2 v;
                    if (LEAF)
                        v = make_int2(__ldg(ta.ids + ma.x + io), __ldg(tb.ids + mb.x + j));
                    else
                        v = make_int2(ma.x + io, mb.x + j);
                    out[base + cur + __popc(m & lt)] = v;
                }
                cur += __popc(m);
            }
            // O3: outer children ascend by lx, so after one fails the key test
            // every later one fails it too
            if (__ballot_sync(RT_FULL, vi && !keyok) != 0)
                break;
        }
        if (PASS == PASS_COUNT && lane == 0)
            counts[p] = cur;
    }
}

// ------------------------------------------------ persistent queued form
// The same traversal with node pairs pulled from a device work queue
// instead of one launch per level: warps of a persistent grid take items
// (node pairs, one 64-bit word each) by ticket, test them with the
// one-to-many comparison, and publish the qualifying child pairs to new
// slots of the queue; leaf pairs yield (r_id, s_id).  `pending` counts items
// published but not finished; a warp waits for its ticket's slot to be
// filled or for pending to reach zero, which ends the pass.  Every wait is
// bounded (flag 4, reported as RTREE_ETIMEOUT).  Two passes over the same
// traversal: the count pass adds up the result pairs, the scatter pass
// writes them through an atomic cursor (the pairs are sorted afterwards).
enum { JQ_QUEUE_FULL = 1, JQ_OUT_FULL = 2, JQ_TIMEOUT = 4, JQ_MISMATCH = 8 };
constexpr unsigned long long kJEmpty = ~0ull;
constexpr long long kJoinWaitCycles = 2000000000LL;  // about one second
constexpr int kTickets = 4;  // queue slots a warp takes at once

// Level bases of one tree (node index where each level starts, root first).
struct Levels {
    int32_t base[RT_MAX_LEVELS];
    int32_t n;
};

struct JoinQueue {
    unsigned long long *items;
    long long cap;
    unsigned long long *head;
    unsigned long long *tail;
    long long *pending;
};

// Height of node g above the leaves (0 = leaf level).
__device__ __forceinline__ int height_of(const Levels &L, int g)
{
    int l = 0;
    for (int e = 1; e < L.n; ++e)
        if (g >= L.base[e])
            l = e;
    return L.n - 1 - l;
}

__device__ __forceinline__ unsigned long long pack_pair(int a, int b)
{
    return (unsigned long long)(unsigned)a | ((unsigned long long)(unsigned)b << 32);
}

// Per-warp staging of one item's output: child node pairs to publish and
// result pairs to write, flushed with one atomic reservation each, so that
// the queue's and the output's counters see few atomics per item.
constexpr int kStage = 128;
struct JoinStage {
    unsigned long long push[kThreads / 32][kStage];
    int2 pairs[kThreads / 32][kStage];
};

// Publishes the np staged child pairs: pending is raised before the slots
// are reserved and written, so the pass cannot end while they are
// outstanding.
__device__ __forceinline__ void jq_flush_push(const JoinQueue &q, int32_t *flags, const unsigned long long *buf,
                                              int np, int lane)
{
    if (np == 0)
        return;
    unsigned long long pos = 0;
    if (lane == 0) {
        atomicAdd(reinterpret_cast<unsigned long long *>(q.pending), (unsigned long long)np);
        pos = atomicAdd(q.tail, (unsigned long long)np);
    }
    pos = __shfl_sync(RT_FULL, pos, 0);
    for (int e = lane; e < np; e += 32) {
        const unsigned long long at = pos + e;
        if ((long long)at < q.cap) {
            volatile unsigned long long *slot = q.items + at;
            *slot = buf[e];
        } else {  // dropped: the traversal is incomplete, the host redoes it by levels
            atomicOr(flags, JQ_QUEUE_FULL);
            atomicAdd(reinterpret_cast<unsigned long long *>(q.pending), ~0ull);
        }
    }
    __syncwarp();
}

__device__ __forceinline__ void jq_flush_pairs(unsigned long long *out_count, int2 *out, long long out_cap,
                                               int32_t *flags, const int2 *buf, int n, int lane)
{
    if (n == 0)
        return;
    unsigned long long base = 0;
    if (lane == 0)
        base = atomicAdd(out_count, (unsigned long long)n);
    base = __shfl_sync(RT_FULL, base, 0);
    for (int e = lane; e < n; e += 32) {
        if ((long long)(base + e) < out_cap)
            out[base + e] = buf[e];
        else
            atomicOr(flags, JQ_OUT_FULL);
    }
    __syncwarp();
}

// Emits one ballot round: result pairs (leaf) are counted (count pass) or
// staged for writing; child node pairs are staged for publishing.
template <int PASS>
__device__ __forceinline__ void jq_emit(const JoinQueue &q, unsigned long long *out_count, int2 *out,
                                        long long out_cap, int32_t *flags, unsigned m, bool hit, int2 v,
                                        bool leaf, int lane, unsigned lt, unsigned long long &leaf_cnt,
                                        unsigned long long *push, int &np, int2 *pbuf, int &npairs)
{
    const int n = __popc(m);
    if (n == 0)
        return;
    if (leaf) {
        if (PASS == PASS_COUNT) {
            leaf_cnt += n;
            return;
        }
        if (npairs + n > kStage) {
            jq_flush_pairs(out_count, out, out_cap, flags, pbuf, npairs, lane);
            npairs = 0;
        }
        if (hit)
            pbuf[npairs + __popc(m & lt)] = v;
        npairs += n;
        __syncwarp();
        return;
    }
    if (np + n > kStage) {
        jq_flush_push(q, flags, push, np, lane);
        np = 0;
    }
    if (hit)
        push[np + __popc(m & lt)] = pack_pair(v.x, v.y);
    np += n;
    __syncwarp();
}

template <int PASS, bool PRUNE>
__global__ void __launch_bounds__(kThreads)
    k_join_wq(TreeDev ta, TreeDev tb, Levels la, Levels lb, JoinQueue q, long long wait_cycles,
              unsigned long long *__restrict__ out_count, int2 *__restrict__ out, long long out_cap,
              int32_t *__restrict__ flags)
{
    __shared__ float s_lx[kThreads / 32][kMaxFanout];
    __shared__ JoinStage stage;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned lt = lanemask_lt();
    float *lxs = s_lx[wid];
    unsigned long long *push = stage.push[wid];
    int2 *pbuf = stage.pairs[wid];
    const int Fa = ta.fanout, Fb = tb.fanout;
    unsigned long long warp_pairs = 0;  // count pass: result pairs found by this warp
    unsigned long long ticket = 0, ticket_end = 0;  // tickets are taken kTickets at a time
    for (;;) {
        if (ticket == ticket_end) {
            if (lane == 0)
                ticket = atomicAdd(q.head, (unsigned long long)kTickets);
            ticket = __shfl_sync(RT_FULL, ticket, 0);
            ticket_end = ticket + kTickets;
        }
        const unsigned long long my = ticket++;
        if ((long long)my >= q.cap)
            break;
        unsigned long long word = kJEmpty;
        if (lane == 0) {
            const long long t0 = clock64();
            const volatile unsigned long long *slot = q.items + my;
            const volatile long long *pend = q.pending;
            unsigned ns = 32;
            for (;;) {
                word = *slot;
                if (word != kJEmpty)
                    break;
                if (*pend == 0)
                    break;
                if (clock64() - t0 > wait_cycles) {
                    atomicOr(flags, JQ_TIMEOUT);
                    break;
                }
                __nanosleep(ns);
                if (ns < 2048)
                    ns <<= 1;
            }
            __threadfence();
        }
        word = __shfl_sync(RT_FULL, word, 0);
        if (word == kJEmpty)
            break;
        const int a = (int)(word & 0xffffffffull), b = (int)(word >> 32);
        const int ha = height_of(la, a), hb = height_of(lb, b);
        const int4 ma = __ldg(ta.meta + a), mb = __ldg(tb.meta + b);
        unsigned long long leaf_cnt = 0;
        int np = 0, npairs = 0;
        if (ha > hb) {  // only r descends
            const float4 bb = __ldg(tb.nbox + b);
            for (int i0 = 0; i0 < ma.y; i0 += 32) {
                const int i = i0 + lane;
                const bool hit = i < ma.y && meets(load_entry(ta.mbr, ta.layout, Fa, a, i), bb);
                const unsigned m = __ballot_sync(RT_FULL, hit);
                jq_emit<PASS>(q, out_count, out, out_cap, flags, m, hit, make_int2(ma.x + i, b), false, lane,
                              lt, leaf_cnt, push, np, pbuf, npairs);
            }
        } else if (hb > ha) {  // only s descends
            const float4 ab = __ldg(ta.nbox + a);
            for (int j0 = 0; j0 < mb.y; j0 += 32) {
                const int j = j0 + lane;
                const bool hit = j < mb.y && meets(ab, load_entry(tb.mbr, tb.layout, Fb, b, j));
                const unsigned m = __ballot_sync(RT_FULL, hit);
                jq_emit<PASS>(q, out_count, out, out_cap, flags, m, hit, make_int2(a, mb.x + j), false, lane,
                              lt, leaf_cnt, push, np, pbuf, npairs);
            }
        } else if (!PRUNE) {  // equal heights: one-to-many comparison
            const bool leaf = ha == 0;
            const int G = Fb < 32 ? Fb : 32;
            const int KO = 32 / G;
            const int grp = lane / G, sub = lane % G;
            for (int j0 = 0; j0 < mb.y; j0 += G) {
                const int j = j0 + sub;
                const bool vj = j < mb.y;
                const float4 ib = vj ? load_entry(tb.mbr, tb.layout, Fb, b, j) : empty_box();
                for (int i0 = 0; i0 < ma.y; i0 += KO) {
                    const int i = i0 + grp;
                    const bool vi = i < ma.y;
                    const float4 ob = vi ? load_entry(ta.mbr, ta.layout, Fa, a, i) : empty_box();
                    const bool hit = vi && vj && meets(ob, ib);
                    const unsigned m = __ballot_sync(RT_FULL, hit);
                    int2 v = make_int2(ma.x + i, mb.x + j);
                    if (leaf && hit && PASS == PASS_SCATTER)
                        v = make_int2(__ldg(ta.ids + ma.x + i), __ldg(tb.ids + mb.x + j));
                    jq_emit<PASS>(q, out_count, out, out_cap, flags, m, hit, v, leaf, lane, lt, leaf_cnt, push, np,
                                  pbuf, npairs);
                }
            }
        } else {  // equal heights of sorted trees: O3 and O5 as in k_join_pruned
            const bool leaf = ha == 0;
            const float4 bb = __ldg(tb.nbox + b);
            const int nin = mb.y;
            __syncwarp();
            for (int j = lane; j < nin; j += 32)
                lxs[j] = entry_lx(tb, b, j);
            __syncwarp();
            int P2 = 1, rounds = 1;
            while (P2 < nin) {
                P2 <<= 1;
                ++rounds;
            }
            for (int i0 = 0; i0 < ma.y; i0 += 32) {
                const int i = i0 + lane;
                const bool vi = i < ma.y;
                const float4 ob = vi ? load_entry(ta.mbr, ta.layout, Fa, a, i) : empty_box();
                const bool keyok = vi && ob.x <= bb.z;
                const bool cand = keyok && meets(ob, bb);
                int f = 0;
                if (cand) {
                    int g = P2 >> 1, step = (P2 >> 2) > 1 ? (P2 >> 2) : 1;
                    f = nin;
                    for (int r = 0; r < rounds; ++r) {
                        const bool pass = g < nin && ob.z >= lxs[g];
                        if (!pass && g < f)
                            f = g;
                        g = pass ? g + step : g - step;
                        step = (step >> 1) > 1 ? (step >> 1) : 1;
                    }
                }
                int incl = f;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int u = __shfl_up_sync(RT_FULL, incl, o);
                    if (lane >= o)
                        incl += u;
                }
                const int excl = incl - f;
                const int T = __shfl_sync(RT_FULL, incl, 31);
                for (int k0 = 0; k0 < T; k0 += 32) {
                    const int k = k0 + lane;
                    int own = 0;
#pragma unroll
                    for (int st = 16; st > 0; st >>= 1) {
                        const int v = __shfl_sync(RT_FULL, incl, own + st - 1);
                        if (v <= k)
                            own += st;
                    }
                    const int ex = __shfl_sync(RT_FULL, excl, own);
                    const float4 o = make_float4(__shfl_sync(RT_FULL, ob.x, own), __shfl_sync(RT_FULL, ob.y, own),
                                                 __shfl_sync(RT_FULL, ob.z, own), __shfl_sync(RT_FULL, ob.w, own));
                    const int j = k - ex;
                    bool hit = false;
                    if (k < T)
                        hit = meets(o, load_entry(tb.mbr, tb.layout, Fb, b, j));
                    const unsigned m = __ballot_sync(RT_FULL, hit);
                    const int io = i0 + own;
                    int2 v = make_int2(ma.x + io, mb.x + j);
                    if (leaf && hit && PASS == PASS_SCATTER)
                        v = make_int2(__ldg(ta.ids + ma.x + io), __ldg(tb.ids + mb.x + j));
                    jq_emit<PASS>(q, out_count, out, out_cap, flags, m, hit, v, leaf, lane, lt, leaf_cnt, push, np,
                                  pbuf, npairs);
                }
                if (__ballot_sync(RT_FULL, vi && !keyok) != 0)
                    break;
            }
        }
        warp_pairs += leaf_cnt;
        jq_flush_push(q, flags, push, np, lane);
        if (PASS == PASS_SCATTER)
            jq_flush_pairs(out_count, out, out_cap, flags, pbuf, npairs, lane);
        __syncwarp();
        if (lane == 0) {
            __threadfence();
            atomicAdd(reinterpret_cast<unsigned long long *>(q.pending), ~0ull);  // -1: this item is done
        }
    }
    if (PASS == PASS_COUNT && lane == 0 && warp_pairs)
        atomicAdd(out_count, warp_pairs);
}

// Resets the queue to the one item (root, root) and zeroes the counter;
// hold adds items counted as pending but never published (0 in normal use).
__global__ void k_jq_init(unsigned long long *__restrict__ items, long long cap,
                          unsigned long long *__restrict__ ctl, unsigned long long *__restrict__ counter,
                          int hold)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < cap;
         i += (long long)gridDim.x * blockDim.x)
        items[i] = i == 0 ? pack_pair(0, 0) : kJEmpty;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctl[0] = 0;  // head
        ctl[1] = 1;  // tail
        ctl[2] = 1 + hold;  // pending
        *counter = 0;
    }
}

__global__ void k_jq_check(const unsigned long long *__restrict__ cursor, const unsigned long long *__restrict__ want,
                           int32_t *__restrict__ flags)
{
    if (*cursor != *want)
        atomicOr(flags, JQ_MISMATCH);
}

using JoinKernel = void (*)(TreeDev, TreeDev, const int2 *, int64_t, int32_t *, const int64_t *,
                            int2 *);

JoinKernel pick(int mode, int pass, bool prune)
{
    if (prune && mode == J_BOTH)
        return pass == PASS_COUNT ? k_join_pruned<false, PASS_COUNT> : k_join_pruned<false, PASS_SCATTER>;
    if (prune && mode == J_LEAF)
        return pass == PASS_COUNT ? k_join_pruned<true, PASS_COUNT> : k_join_pruned<true, PASS_SCATTER>;
    switch (mode) {
    case J_BOTH: return pass == PASS_COUNT ? k_join<J_BOTH, PASS_COUNT> : k_join<J_BOTH, PASS_SCATTER>;
    case J_A: return pass == PASS_COUNT ? k_join<J_A, PASS_COUNT> : k_join<J_A, PASS_SCATTER>;
    case J_B: return pass == PASS_COUNT ? k_join<J_B, PASS_COUNT> : k_join<J_B, PASS_SCATTER>;
    default: return pass == PASS_COUNT ? k_join<J_LEAF, PASS_COUNT> : k_join<J_LEAF, PASS_SCATTER>;
    }
}

unsigned grid_for(int64_t np)
{
    int64_t g = (np * 32 + kThreads - 1) / kThreads;
    const int64_t cap = (int64_t)sm_count() * 8;
    if (g > cap)
        g = cap;
    return (unsigned)(g < 1 ? 1 : g);
}

__global__ void k_split_pairs(const int2 *__restrict__ p, int64_t n, uint32_t *__restrict__ key,
                              uint32_t *__restrict__ val)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int2 v = p[i];
        key[i] = (uint32_t)v.y ^ kSign;  // s first (least significant)
        val[i] = (uint32_t)v.x;
    }
}

__global__ void k_flip(const uint32_t *__restrict__ in, int64_t n, uint32_t *__restrict__ out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = in[i] ^ kSign;
}

__global__ void k_merge_pairs(const uint32_t *__restrict__ r, const uint32_t *__restrict__ s,
                              int64_t n, int2 *__restrict__ out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = make_int2((int)(r[i] ^ kSign), (int)(s[i] ^ kSign));
}

unsigned blocks_for(int64_t n)
{
    int64_t b = (n + 255) / 256;
    return (unsigned)(b < 1 ? 1 : (b > 65536 ? 65536 : b));
}

// Sorts (r, s) pairs lexicographically: stable sort by s, then by r.
rtree_status sort_pairs(int2 *pairs, int64_t n, cudaStream_t s)
{
    if (n <= 1)
        return RTREE_OK;
    DevBuf<uint32_t> k0(s), v0(s), k1(s), v1(s);
    RT_TRY(k0.alloc(n, "join sort"));
    RT_TRY(v0.alloc(n, "join sort"));
    RT_TRY(k1.alloc(n, "join sort"));
    RT_TRY(v1.alloc(n, "join sort"));
    {
        KernelTimer kt_("split_pairs", s);
        k_split_pairs<<<blocks_for(n), 256, 0, s>>>(pairs, n, k0.p, v0.p);
        RT_LAUNCH();
    }
    RT_TRY(radix_sort_pairs(k0.p, v0.p, k1.p, v1.p, n, 0, 32, s));  // by s; v1 = r
    {
        KernelTimer kt_("flip", s);
        k_flip<<<blocks_for(n), 256, 0, s>>>(v1.p, n, k0.p);  // r keys
        RT_LAUNCH();
    }
    RT_TRY(radix_sort_pairs(k0.p, k1.p, v0.p, v1.p, n, 0, 32, s));  // by r; v1 = s keys
    {
        KernelTimer kt_("merge_pairs", s);
        k_merge_pairs<<<blocks_for(n), 256, 0, s>>>(v0.p, v1.p, n, pairs);
        RT_LAUNCH();
    }
    return RTREE_OK;
}

using JoinWqKernel = void (*)(TreeDev, TreeDev, Levels, Levels, JoinQueue, long long, unsigned long long *,
                              int2 *, long long, int32_t *);

Levels levels_of(const rtree *t)
{
    Levels L{};
    L.n = t->levels;
    for (int e = 0; e < t->levels; ++e)
        L.base[e] = (int32_t)t->level_base[e];
    return L;
}

}  // namespace

rtree_status tree_join_queue(const rtree *R, const rtree *S, bool prune, cudaStream_t s, rtree_result *res,
                             bool *redo_by_levels)
{
    *redo_by_levels = false;
    res->rows = 0;
    res->total = 0;
    res->offsets = nullptr;
    if (R->nodes == 0 || S->nodes == 0) {
        DevBuf<int32_t> ids(s);
        RT_TRY(ids.alloc(2, "join pairs"));
        res->ids = ids.release();
        return RTREE_OK;
    }
    const TreeDev ta = R->view(), tb = S->view();
    const Levels la = levels_of(R), lb = levels_of(S);
    const long long cap = std::max<long long>(1ll << 22, 8ll * (R->nodes + S->nodes));
    DevBuf<unsigned long long> items(s), ctl(s), counter(s);
    DevBuf<int32_t> flags(s);
    RT_TRY(items.alloc(cap, "join work queue"));
    RT_TRY(ctl.alloc(3, "join work queue counters"));
    RT_TRY(counter.alloc(2, "join pair counters"));  // [0] count pass total, [1] scatter cursor
    RT_TRY(flags.alloc(2, "join flags"));
    RT_CUDA(cudaMemsetAsync(flags.p, 0, 2 * sizeof(int32_t), s));
    const JoinQueue q{items.p, cap, ctl.p, ctl.p + 1, reinterpret_cast<long long *>(ctl.p + 2)};
    JoinWqKernel kc = prune ? k_join_wq<PASS_COUNT, true> : k_join_wq<PASS_COUNT, false>;
    JoinWqKernel ks = prune ? k_join_wq<PASS_SCATTER, true> : k_join_wq<PASS_SCATTER, false>;
    int per_sm = 0;
    RT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kc, kThreads, 0));
    const unsigned grid = (unsigned)((per_sm > 0 ? per_sm : 1) * sm_count());  // persistent: all resident
    const unsigned init_blocks = (unsigned)std::min<long long>((cap + 255) / 256, 65536);
    long long dbg_wait = 0;
    int dbg_hold = 0;
    debug_wq_take(&dbg_wait, &dbg_hold);
    {
        KernelTimer kt_("jq_init", s);
        k_jq_init<<<init_blocks, 256, 0, s>>>(items.p, cap, ctl.p, counter.p, dbg_hold ? 1 : 0);
        RT_LAUNCH();
    }
    {
        KernelTimer kt_(prune ? "join_pruned_queue_count" : "join_queue_count", s);
        kc<<<grid, kThreads, 0, s>>>(ta, tb, la, lb, q, dbg_wait > 0 ? dbg_wait : kJoinWaitCycles, counter.p,
                                     nullptr, 0, flags.p);
        RT_LAUNCH();
    }
    // the one host read: the number of pairs (it sizes the result) and the flags
    int64_t total = 0;
    {
        PostList pl{};
        pl.src[0] = counter.p;
        pl.words[0] = 2;
        pl.at[0] = 0;
        pl.src[1] = flags.p;
        pl.words[1] = 1;
        pl.at[1] = 2;
        pl.n = 2;
        uint32_t w[3];
        RT_TRY(read_words(pl, s, w, 3));
        total = (int64_t)((uint64_t)w[0] | ((uint64_t)w[1] << 32));
        if (w[2] & JQ_TIMEOUT)
            return fail(RTREE_ETIMEOUT, "join: a work-queue wait exceeded its limit");
        if (w[2] & JQ_QUEUE_FULL) {  // more node pairs than the queue holds
            *redo_by_levels = true;
            return RTREE_OK;
        }
        if (w[2])
            return fail(RTREE_EINTERNAL, "join count pass reported device flags 0x%x", w[2]);
    }
    if (total >= (int64_t)INT32_MAX)
        return fail(RTREE_EOVERFLOW, "join result of %lld pairs exceeds the 2^31-1 pairs the pair sort takes",
                    (long long)total);
    DevBuf<int2> pairs(s);
    RT_TRY(pairs.alloc(total, "join pairs"));
    {
        KernelTimer kt_("jq_init", s);
        k_jq_init<<<init_blocks, 256, 0, s>>>(items.p, cap, ctl.p, counter.p + 1, 0);
        RT_LAUNCH();
    }
    {
        KernelTimer kt_(prune ? "join_pruned_queue_scatter" : "join_queue_scatter", s);
        ks<<<grid, kThreads, 0, s>>>(ta, tb, la, lb, q, kJoinWaitCycles, counter.p + 1, pairs.p, total,
                                     flags.p);
        RT_LAUNCH();
    }
    {
        KernelTimer kt_("jq_check", s);
        k_jq_check<<<1, 1, 0, s>>>(counter.p + 1, counter.p, flags.p);
        RT_LAUNCH();
    }
    RT_TRY(sort_pairs(pairs.p, total, s));
    // the scatter pass and the sort run on in the order of s; their flags
    // reach the result's status
    RT_TRY(post_result_status(flags.p, s, res));
    res->total = total;
    res->ids = reinterpret_cast<int32_t *>(pairs.release());
    return RTREE_OK;
}

rtree_status tree_join(const rtree *R, const rtree *S, bool prune, cudaStream_t s,
                       rtree_result *res, int64_t *stats)
{
    res->rows = 0;
    res->total = 0;
    res->offsets = nullptr;
    if (R->nodes == 0 || S->nodes == 0) {
        DevBuf<int32_t> ids(s);
        RT_TRY(ids.alloc(2, "join pairs"));
        RT_CUDA(cudaStreamSynchronize(s));
        res->ids = ids.release();
        return RTREE_OK;
    }
    const TreeDev ta = R->view(), tb = S->view();
    DevBuf<int2> front(s);
    RT_TRY(front.alloc(1, "join frontier"));
    const int2 root = make_int2(0, 0);
    RT_CUDA(cudaMemcpyAsync(front.p, &root, sizeof(int2), cudaMemcpyHostToDevice, s));
    int64_t np = 1;
    int da = 0, db = 0;
    for (;;) {
        const int ra = R->levels - 1 - da, rb = S->levels - 1 - db;
        const int mode = (ra == 0 && rb == 0) ? J_LEAF : (ra > rb ? J_A : (rb > ra ? J_B : J_BOTH));
        if (stats)
            stats[mode] += np;  // node pairs tested in this mode
        DevBuf<int32_t> cnt(s);
        DevBuf<int64_t> off(s);
        RT_TRY(cnt.alloc(np, "join counts"));
        RT_TRY(off.alloc(np + 1, "join offsets"));
        {
            KernelTimer kt_(prune ? "join_pruned_count" : "join_count", s);
            pick(mode, PASS_COUNT, prune)<<<grid_for(np), kThreads, 0, s>>>(ta, tb, front.p, np, cnt.p,
                                                                     nullptr, nullptr);
            RT_LAUNCH();
        }
        RT_TRY(scan_exclusive(cnt.p, off.p, np, s));
        int64_t total = 0;
        RT_CUDA(cudaMemcpyAsync(&total, off.p + np, sizeof(total), cudaMemcpyDeviceToHost, s));
        RT_CUDA(cudaStreamSynchronize(s));
        DevBuf<int2> next(s);
        RT_TRY(next.alloc(total, mode == J_LEAF ? "join pairs" : "join frontier"));
        if (total > 0) {
            KernelTimer kt_(prune ? "join_pruned_scatter" : "join_scatter", s);
            pick(mode, PASS_SCATTER, prune)<<<grid_for(np), kThreads, 0, s>>>(ta, tb, front.p, np,
                                                                       nullptr, off.p, next.p);
            RT_LAUNCH();
        }
        if (mode == J_LEAF || total == 0) {
            if (stats)
                stats[4] = mode == J_LEAF ? total : 0;
            RT_TRY(sort_pairs(next.p, total, s));
            RT_CUDA(cudaStreamSynchronize(s));
            res->total = total;
            res->ids = reinterpret_cast<int32_t *>(next.release());
            return RTREE_OK;
        }
        if (mode == J_A || mode == J_BOTH)
            ++da;
        if (mode == J_B || mode == J_BOTH)
            ++db;
        std::swap(front.p, next.p);
        np = total;
    }
}

}  // namespace rt
