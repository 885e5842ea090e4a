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
#include "internal.cuh"

namespace rt {
namespace {

constexpr int kWarps = 8;
constexpr int kThreads = kWarps * 32;
enum { PASS_COUNT = 0, PASS_SCATTER = 1 };
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
    k_select(TreeDev t, const float4 *__restrict__ queries, int64_t Q,
             int32_t *__restrict__ counts, const int64_t *__restrict__ offsets,
             int32_t *__restrict__ out, unsigned long long *__restrict__ next_query,
             int32_t *__restrict__ flags, int cap, unsigned long long *__restrict__ stats)
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
        int64_t base = 0, lim = 0;
        if (PASS == PASS_SCATTER) {
            base = __ldg(offsets + qi);
            lim = __ldg(offsets + qi + 1);  // writes never pass the segment end
        }
        int64_t cur = 0;  // ids found so far, warp-uniform
        int top = 0;
        if (t.nodes > 0) {
            if (lane == 0)
                st[0] = 0;
            top = 1;
        }
        __syncwarp();
        bool overflow = false;
        unsigned long long n_visit = 0, n_leaf = 0, n_cont = 0, n_from_ranges = 0;
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
                        out[o] = __ldg(t.ids + m.x + j);
                }
                cur += __popc(me);
                const unsigned mc = __ballot_sync(RT_FULL, cont);
                if (mc) {
                    int lo = 0, hi = 0;
                    if (cont) {
                        const int4 cm = __ldg(t.meta + m.x + j);
                        lo = cm.z;
                        hi = cm.w;
                    }
                    if (stats) {
                        n_cont += __popc(mc);
                        n_from_ranges += __reduce_add_sync(RT_FULL, (unsigned)(hi - lo));
                    }
                    if (PASS == PASS_COUNT) {
                        cur += __reduce_add_sync(RT_FULL, (unsigned)(hi - lo));
                    } else {
                        unsigned mm = mc;
                        while (mm) {
                            const int src = __ffs(mm) - 1;
                            mm &= mm - 1;
                            const int l = __shfl_sync(RT_FULL, lo, src);
                            const int h = __shfl_sync(RT_FULL, hi, src);
                            const int64_t room = lim - (base + cur);
                            const int hh = (int64_t)(h - l) <= room ? h : l + (int)(room > 0 ? room : 0);
                            warp_copy(out + base + cur, t.ids, l, hh, lane);
                            cur += h - l;
                        }
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
            atomicAdd(stats + 3, n_cont);
            atomicAdd(stats + 4, (unsigned long long)cur);
            atomicAdd(stats + 5, n_from_ranges);
        }
        if (lane == 0) {
            if (overflow)
                atomicOr(flags, FLAG_STACK);
            if (PASS == PASS_COUNT)
                counts[qi] = (int32_t)cur;
            else if (cur != __ldg(offsets + qi + 1) - base)
                atomicOr(flags, FLAG_COUNT_MISMATCH);
        }
    }
}

using SelectKernel = void (*)(TreeDev, const float4 *, int64_t, int32_t *, const int64_t *,
                              int32_t *, unsigned long long *, int32_t *, int,
                              unsigned long long *);

template <int F, int LAYOUT>
SelectKernel pick_pass(int pass)
{
    return pass == PASS_COUNT ? k_select<F, LAYOUT, PASS_COUNT> : k_select<F, LAYOUT, PASS_SCATTER>;
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

rtree_status launch(SelectKernel kern, const rtree *t, const float4 *q, int64_t Q, int32_t *counts,
                    const int64_t *offsets, int32_t *out, unsigned long long *ctr, int32_t *flags,
                    cudaStream_t s, unsigned long long *stats = nullptr)
{
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
    KernelTimer kt_(counts ? "select_count" : "select_scatter", s);
    kern<<<(unsigned)grid, kThreads, smem, s>>>(t->view(), q, Q, counts, offsets, out, ctr, flags,
                                                cap, stats);
    RT_LAUNCH();
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
    if (Q == 0 || t->nodes == 0) {
        RT_CUDA(cudaMemsetAsync(off.p, 0, (Q + 1) * sizeof(int64_t), s));
        DevBuf<int32_t> ids(s);
        RT_TRY(ids.alloc(1, "select ids"));
        RT_CUDA(cudaStreamSynchronize(s));
        res->offsets = off.release();
        res->ids = ids.release();
        return RTREE_OK;
    }
    SelectKernel kc = pick(t->fanout, t->layout, PASS_COUNT);
    SelectKernel ks = pick(t->fanout, t->layout, PASS_SCATTER);
    if (!kc || !ks)
        return fail(RTREE_EINVAL, "unsupported fanout %d", t->fanout);

    DevBuf<int32_t> cnt(s), flags(s);
    DevBuf<unsigned long long> ctr(s);
    RT_TRY(cnt.alloc(Q, "select counts"));
    RT_TRY(flags.alloc(1, "select flags"));
    RT_TRY(ctr.alloc(2, "select work counters"));
    RT_CUDA(cudaMemsetAsync(flags.p, 0, sizeof(int32_t), s));
    RT_CUDA(cudaMemsetAsync(ctr.p, 0, 2 * sizeof(unsigned long long), s));

    RT_TRY(launch(kc, t, queries, Q, cnt.p, nullptr, nullptr, ctr.p, flags.p, s));
    RT_TRY(scan_exclusive(cnt.p, off.p, Q, s));
    int64_t total = 0;
    int32_t hflags = 0;
    RT_CUDA(cudaMemcpyAsync(&total, off.p + Q, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    RT_CUDA(cudaMemcpyAsync(&hflags, flags.p, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    RT_CUDA(cudaStreamSynchronize(s));
    if (hflags)
        return fail(RTREE_EINTERNAL, "select count pass reported device flags 0x%x", hflags);

    DevBuf<int32_t> ids(s);
    RT_TRY(ids.alloc(total, "select ids"));
    RT_TRY(launch(ks, t, queries, Q, nullptr, off.p, ids.p, ctr.p + 1, flags.p, s));
    if (sorted)
        RT_TRY(segmented_sort(ids.p, off.p, Q, total, s));
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
    SelectKernel k = pick(t->fanout, t->layout, counts ? PASS_COUNT : PASS_SCATTER);
    if (!k)
        return fail(RTREE_EINVAL, "unsupported fanout %d", t->fanout);
    return launch(k, t, queries, Q, counts, offsets, out, ctr, flags, s);
}

rtree_status select_stats(const rtree *t, const float4 *queries, int64_t Q, cudaStream_t s,
                          int64_t out[8])
{
    for (int i = 0; i < 8; ++i)
        out[i] = 0;
    out[0] = Q;
    if (Q == 0 || t->nodes == 0)
        return RTREE_OK;
    SelectKernel kc = pick(t->fanout, t->layout, PASS_COUNT);
    if (!kc)
        return fail(RTREE_EINVAL, "unsupported fanout %d", t->fanout);
    DevBuf<int32_t> cnt(s), flags(s);
    DevBuf<unsigned long long> ctr(s), st(s);
    RT_TRY(cnt.alloc(Q, "select counts"));
    RT_TRY(flags.alloc(1, "select flags"));
    RT_TRY(ctr.alloc(1, "select work counter"));
    RT_TRY(st.alloc(8, "select statistics"));
    RT_CUDA(cudaMemsetAsync(flags.p, 0, sizeof(int32_t), s));
    RT_CUDA(cudaMemsetAsync(ctr.p, 0, sizeof(unsigned long long), s));
    RT_CUDA(cudaMemsetAsync(st.p, 0, 8 * sizeof(unsigned long long), s));
    RT_TRY(launch(kc, t, queries, Q, cnt.p, nullptr, nullptr, ctr.p, flags.p, s, st.p));
    unsigned long long h[8];
    RT_CUDA(cudaMemcpyAsync(h, st.p, sizeof(h), cudaMemcpyDeviceToHost, s));
    RT_CUDA(cudaStreamSynchronize(s));
    for (int i = 0; i < 6; ++i)
        out[i] = (int64_t)h[i];
    return RTREE_OK;
}

}  // namespace rt
