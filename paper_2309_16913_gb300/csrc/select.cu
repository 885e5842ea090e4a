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
// Pass kinds:
//   COUNT    per query: ids found, and (optionally) how many came one by one
//            from leaves and how many whole subtrees were taken;
//   SCATTER  writes the ids themselves in traversal order (unsorted output);
//   DESC     writes the leaf hits and, for every whole subtree, its (lo, hi)
//            range of the tree's id array; the sorted output is then built
//            by the segmented sort, which reads the ranges directly.
#include "internal.cuh"

namespace rt {
namespace {

constexpr int kWarps = 8;
constexpr int kThreads = kWarps * 32;
enum { PASS_COUNT = 0, PASS_SCATTER = 1, PASS_DESC = 2 };
enum { FLAG_STACK = 1, FLAG_COUNT_MISMATCH = 2 };

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

template <int F, int LAYOUT, int PASS>
__global__ void __launch_bounds__(kThreads)
    k_select(TreeDev t, const float4 *__restrict__ queries, int64_t Q, SelIO io,
             unsigned long long *__restrict__ next_query, int32_t *__restrict__ flags, int cap,
             unsigned long long *__restrict__ stats)
{
    constexpr int G = F < 32 ? F : 32;  // lanes per node
    constexpr int K = 32 / G;           // nodes per warp step
    constexpr int C = F / G;            // children per lane
    extern __shared__ int32_t smem[];
    const int lane = threadIdx.x & 31;
    int32_t *st = smem + (threadIdx.x >> 5) * cap;
    const int grp = lane / G, sub = lane % G;
    const unsigned lt = lanemask_lt();

    for (;;) {
        unsigned long long qi = 0;
        if (lane == 0)
            qi = atomicAdd(next_query, 1ull);
        qi = __shfl_sync(RT_FULL, qi, 0);
        if (qi >= (unsigned long long)Q)
            break;
        const float4 q = __ldg(queries + qi);
        // output cursors: ids (SCATTER), leaf hits and ranges (DESC)
        int64_t base = 0, lim = 0, lbase = 0, llim = 0, rbase = 0, rlim = 0;
        if (PASS == PASS_SCATTER) {
            base = __ldg(io.offsets + qi);
            lim = __ldg(io.offsets + qi + 1);  // writes never pass the segment end
        }
        if (PASS == PASS_DESC) {
            lbase = __ldg(io.off_leaf + qi);
            llim = __ldg(io.off_leaf + qi + 1);
            rbase = __ldg(io.off_rng + qi);
            rlim = __ldg(io.off_rng + qi + 1);
        }
        int64_t cur = 0;   // ids found so far, warp-uniform
        int64_t lcur = 0;  // leaf hits so far
        int64_t rcur = 0;  // whole subtrees so far
        int top = 0;
        if (t.nodes > 0) {
            if (lane == 0)
                st[0] = 0;
            top = 1;
        }
        __syncwarp();
        bool overflow = false;
        unsigned long long n_visit = 0, n_leaf = 0;
        int steps = 0;  // a query visits each node at most once
        while (top > 0) {
            if (++steps > t.nodes) {
                overflow = true;
                break;
            }
            const int k = top < K ? top : K;
            const int node = grp < k ? st[top - 1 - grp] : -1;
            top -= k;
            __syncwarp();
            if (stats) {
                n_visit += k;
                n_leaf += __popc(__ballot_sync(RT_FULL, node >= t.leaf_base && sub == 0));
            }
            // Entry loads do not wait for the node's metadata: unused slots
            // hold the empty box, and the count only masks them afterwards.
            float4 b[C];
#pragma unroll
            for (int c = 0; c < C; ++c)
                b[c] = node >= 0 ? load_entry_t<F, LAYOUT>(t.mbr, node, sub + c * G) : empty_box();
            const int4 m = node >= 0 ? __ldg(t.meta + node) : make_int4(0, 0, 0, 0);
            const bool leaf = node >= t.leaf_base;
#pragma unroll
            for (int c = 0; c < C; ++c) {
                const int j = sub + c * G;
                const bool hit = node >= 0 && j < m.y && meets(b[c], q);
                const bool cont = hit && !leaf && inside(b[c], q);
                const bool push = hit && !leaf && !cont;
                const bool emit = hit && leaf;
                const unsigned mp = __ballot_sync(RT_FULL, push);
                if (push) {
                    const int pos = top + __popc(mp & lt);
                    if (pos < cap)
                        st[pos] = m.x + j;
                }
                top += __popc(mp);
                const unsigned me = __ballot_sync(RT_FULL, emit);
                if (PASS == PASS_SCATTER && emit) {
                    const int64_t o = base + cur + __popc(me & lt);
                    if (o < lim)
                        io.out[o] = __ldg(t.ids + m.x + j);
                }
                if (PASS == PASS_DESC && emit) {
                    const int64_t o = lbase + lcur + __popc(me & lt);
                    if (o < llim)
                        io.leaf_out[o] = __ldg(t.ids + m.x + j);
                }
                cur += __popc(me);
                lcur += __popc(me);
                const unsigned mc = __ballot_sync(RT_FULL, cont);
                if (mc) {
                    int lo = 0, hi = 0;
                    if (cont) {
                        const int4 cm = __ldg(t.meta + m.x + j);
                        lo = cm.z;
                        hi = cm.w;
                    }
                    if (PASS == PASS_DESC && cont) {
                        const int64_t o = rbase + rcur + __popc(mc & lt);
                        if (o < rlim)
                            io.rng_out[o] = make_int2(lo, hi);
                    }
                    rcur += __popc(mc);
                    if (PASS == PASS_SCATTER) {
                        unsigned mm = mc;
                        while (mm) {
                            const int src = __ffs(mm) - 1;
                            mm &= mm - 1;
                            const int l = __shfl_sync(RT_FULL, lo, src);
                            const int h = __shfl_sync(RT_FULL, hi, src);
                            const int64_t room = lim - (base + cur);
                            const int hh = (int64_t)(h - l) <= room ? h : l + (int)(room > 0 ? room : 0);
                            warp_copy(io.out + base + cur, t.ids, l, hh, lane);
                            cur += h - l;
                        }
                    } else {
                        cur += __reduce_add_sync(RT_FULL, (unsigned)(hi - lo));
                    }
                }
            }
            if (top > cap) {  // cannot happen with cap = H*max(32,F); guarded anyway
                overflow = true;
                top = 0;
            }
            __syncwarp();
        }
        if (stats && lane == 0) {
            atomicAdd(stats + 0, 1ull);
            atomicAdd(stats + 1, n_visit);
            atomicAdd(stats + 2, n_leaf);
            atomicAdd(stats + 3, (unsigned long long)rcur);
            atomicAdd(stats + 4, (unsigned long long)cur);
            atomicAdd(stats + 5, (unsigned long long)(cur - lcur));
        }
        if (lane == 0) {
            if (overflow)
                atomicOr(flags, FLAG_STACK);
            if (PASS == PASS_COUNT) {
                io.counts[qi] = (int32_t)cur;
                if (io.counts_leaf)
                    io.counts_leaf[qi] = (int32_t)lcur;
                if (io.counts_rng)
                    io.counts_rng[qi] = (int32_t)rcur;
            } else if (PASS == PASS_SCATTER) {
                if (cur != lim - base)
                    atomicOr(flags, FLAG_COUNT_MISMATCH);
            } else {
                if (lcur != llim - lbase || rcur != rlim - rbase)
                    atomicOr(flags, FLAG_COUNT_MISMATCH);
            }
        }
    }
}

using SelectKernel = void (*)(TreeDev, const float4 *, int64_t, SelIO, unsigned long long *,
                              int32_t *, int, unsigned long long *);

template <int F, int LAYOUT>
SelectKernel pick_pass(int pass)
{
    return pass == PASS_COUNT     ? k_select<F, LAYOUT, PASS_COUNT>
           : pass == PASS_SCATTER ? k_select<F, LAYOUT, PASS_SCATTER>
                                  : k_select<F, LAYOUT, PASS_DESC>;
}

template <int F>
SelectKernel pick_layout(int layout, int pass)
{
    return layout == RTREE_LAYOUT_AOS ? pick_pass<F, RTREE_LAYOUT_AOS>(pass)
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
    return pass == PASS_COUNT ? "select_count" : pass == PASS_SCATTER ? "select_scatter" : "select_desc";
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

rtree_status empty_result(int64_t Q, DevBuf<int64_t> &off, cudaStream_t s, rtree_result *res)
{
    RT_CUDA(cudaMemsetAsync(off.p, 0, (Q + 1) * sizeof(int64_t), s));
    DevBuf<int32_t> ids(s);
    RT_TRY(ids.alloc(1, "select ids"));
    RT_CUDA(cudaStreamSynchronize(s));
    res->offsets = off.release();
    res->ids = ids.release();
    return RTREE_OK;
}

}  // namespace

rtree_status range_select(const rtree *t, const float4 *queries, int64_t Q, bool sorted,
                          int mapping, cudaStream_t s, rtree_result *res)
{
    (void)mapping;
    res->rows = Q;
    res->total = 0;
    DevBuf<int64_t> off(s);
    RT_TRY(off.alloc(Q + 1, "select offsets"));
    if (Q == 0 || t->nodes == 0)
        return empty_result(Q, off, s, res);
    if (!pick(t->fanout, t->layout, PASS_COUNT))
        return fail(RTREE_EINVAL, "unsupported fanout %d", t->fanout);

    DevBuf<int32_t> cnt(s), cnt_leaf(s), cnt_rng(s), flags(s);
    DevBuf<unsigned long long> ctr(s);
    RT_TRY(cnt.alloc(Q, "select counts"));
    RT_TRY(flags.alloc(1, "select flags"));
    RT_TRY(ctr.alloc(2, "select work counters"));
    RT_CUDA(cudaMemsetAsync(flags.p, 0, sizeof(int32_t), s));
    RT_CUDA(cudaMemsetAsync(ctr.p, 0, 2 * sizeof(unsigned long long), s));
    SelIO io{};
    io.counts = cnt.p;
    if (sorted) {
        RT_TRY(cnt_leaf.alloc(Q, "select counts"));
        RT_TRY(cnt_rng.alloc(Q, "select counts"));
        io.counts_leaf = cnt_leaf.p;
        io.counts_rng = cnt_rng.p;
    }
    RT_TRY(launch(PASS_COUNT, t, queries, Q, io, ctr.p, flags.p, s));
    RT_TRY(scan_exclusive(cnt.p, off.p, Q, s));
    DevBuf<int64_t> off_leaf(s), off_rng(s);
    if (sorted) {
        RT_TRY(off_leaf.alloc(Q + 1, "select offsets"));
        RT_TRY(off_rng.alloc(Q + 1, "select offsets"));
        RT_TRY(scan_exclusive(cnt_leaf.p, off_leaf.p, Q, s));
        RT_TRY(scan_exclusive(cnt_rng.p, off_rng.p, Q, s));
    }
    int64_t h[3] = {0, 0, 0};
    int32_t hflags = 0;
    RT_CUDA(cudaMemcpyAsync(&h[0], off.p + Q, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    if (sorted) {
        RT_CUDA(cudaMemcpyAsync(&h[1], off_leaf.p + Q, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        RT_CUDA(cudaMemcpyAsync(&h[2], off_rng.p + Q, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    }
    RT_CUDA(cudaMemcpyAsync(&hflags, flags.p, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    RT_CUDA(cudaStreamSynchronize(s));
    if (hflags)
        return fail(RTREE_EINTERNAL, "select count pass reported device flags 0x%x", hflags);
    const int64_t total = h[0];

    DevBuf<int32_t> ids(s);
    RT_TRY(ids.alloc(total, "select ids"));
    if (!sorted) {
        SelIO so{};
        so.offsets = off.p;
        so.out = ids.p;
        RT_TRY(launch(PASS_SCATTER, t, queries, Q, so, ctr.p + 1, flags.p, s));
    } else {
        DevBuf<int32_t> leaf(s);
        DevBuf<int2> rng(s);
        RT_TRY(leaf.alloc(h[1], "select leaf hits"));
        RT_TRY(rng.alloc(h[2], "select whole subtrees"));
        SelIO so{};
        so.off_leaf = off_leaf.p;
        so.off_rng = off_rng.p;
        so.leaf_out = leaf.p;
        so.rng_out = rng.p;
        RT_TRY(launch(PASS_DESC, t, queries, Q, so, ctr.p + 1, flags.p, s));
        SortSources src{};
        src.leaf = leaf.p;
        src.off_leaf = off_leaf.p;
        src.rng = rng.p;
        src.off_rng = off_rng.p;
        src.tree_ids = t->ids;
        RT_TRY(segmented_sort_gather(ids.p, off.p, Q, total, src, s));
    }
    RT_CUDA(cudaMemcpyAsync(&hflags, flags.p, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    RT_CUDA(cudaStreamSynchronize(s));
    if (hflags)
        return fail(RTREE_EINTERNAL, "select scatter pass reported device flags 0x%x", hflags);
    res->total = total;
    res->offsets = off.release();
    res->ids = ids.release();
    return RTREE_OK;
}

rtree_status select_pass(const rtree *t, const float4 *queries, int64_t Q, int32_t *counts,
                         const int64_t *offsets, int32_t *out, unsigned long long *ctr,
                         int32_t *flags, cudaStream_t s)
{
    SelIO io{};
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
    SelIO io{};
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
