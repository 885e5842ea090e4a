// segsort.cu -- sort every query's id list ascending.
//
// Results are sets; the traversal emits them in tree order, so each CSR
// segment is sorted afterwards.  Segments are classified by length:
//   2..32      one warp, bitonic network over shuffles;
//   33..4096   one CTA, LSD radix sort in shared memory (8-bit digits);
//   > 4096     one CTA, LSD radix sort through a global scratch area.
// Radix passes whose digit is the same for every key of the segment are
// skipped (found from the AND and OR of the keys).  Stability of each pass
// comes from ranking items in order: each warp owns a contiguous run and
// walks it 32 at a time, ranking equal digits by lane with __match_any_sync.
// Keys are the ids with the sign bit flipped, so unsigned order is signed
// order.
#include <climits>

#include "internal.cuh"

namespace rt {
namespace {

constexpr int kSmallMax = 32;
constexpr int kMidThreads = 256;
constexpr int kMidWarps = kMidThreads / 32;
constexpr int kMidItems = 16;
constexpr int kMidMax = kMidThreads * kMidItems;  // 4096
constexpr int kBins = 256;
constexpr uint32_t kSign = 0x80000000u;

enum { HDR_SMALL = 0, HDR_MID = 1, HDR_LARGE = 2, HDR_SCRATCH = 3 };

__global__ void k_classify(const int64_t *__restrict__ off, int64_t nseg,
                           int32_t *__restrict__ small, int32_t *__restrict__ mid,
                           int32_t *__restrict__ large, int64_t *__restrict__ large_tmp,
                           unsigned long long *__restrict__ hdr)
{
    const int lane = threadIdx.x & 31;
    const unsigned lt = lanemask_lt();
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t b = warp * 32; b < nseg; b += nwarps * 32) {
        const int64_t i = b + lane;
        int64_t len = 0;
        if (i < nseg)
            len = off[i + 1] - off[i];
        const int cls = len <= 1 ? -1 : len <= kSmallMax ? HDR_SMALL : len <= kMidMax ? HDR_MID : HDR_LARGE;
#pragma unroll
        for (int c = HDR_SMALL; c <= HDR_MID; ++c) {
            const unsigned m = __ballot_sync(RT_FULL, cls == c);
            if (m) {
                unsigned long long base = 0;
                const int leader = __ffs(m) - 1;
                if (lane == leader)
                    base = atomicAdd(hdr + c, (unsigned long long)__popc(m));
                base = __shfl_sync(RT_FULL, base, leader);
                if (cls == c)
                    (c == HDR_SMALL ? small : mid)[base + __popc(m & lt)] = (int32_t)i;
            }
        }
        if (cls == HDR_LARGE) {
            const unsigned long long slot = atomicAdd(hdr + HDR_LARGE, 1ull);
            large[slot] = (int32_t)i;
            large_tmp[slot] = (int64_t)atomicAdd(hdr + HDR_SCRATCH, (unsigned long long)len);
        }
    }
}

__global__ void k_sort_small(const int32_t *__restrict__ list, int64_t cnt,
                             const int64_t *__restrict__ off, int32_t *__restrict__ ids)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t w = warp; w < cnt; w += nwarps) {
        const int32_t seg = list[w];
        const int64_t o = off[seg];
        const int n = (int)(off[seg + 1] - o);
        int v = lane < n ? ids[o + lane] : INT_MAX;
#pragma unroll
        for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
            for (int j = k >> 1; j > 0; j >>= 1) {
                const int other = __shfl_xor_sync(RT_FULL, v, j);
                const bool up = (lane & k) == 0;
                const bool lower = (lane & j) == 0;
                v = (lower == up) ? min(v, other) : max(v, other);
            }
        }
        if (lane < n)
            ids[o + lane] = v;
    }
}

// Block-wide AND and OR of one value per thread.
__device__ __forceinline__ void block_and_or(uint32_t &a, uint32_t &o)
{
    __shared__ uint32_t sa[32], so[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        a &= __shfl_xor_sync(RT_FULL, a, d);
        o |= __shfl_xor_sync(RT_FULL, o, d);
    }
    if (lane == 0) {
        sa[w] = a;
        so[w] = o;
    }
    __syncthreads();
    a = 0xffffffffu;
    o = 0;
    for (int x = 0; x < nw; ++x) {
        a &= sa[x];
        o |= so[x];
    }
    __syncthreads();
}

// Ranks one tile of up to 32*ITEMS*WARPS keys held in registers (warp w owns
// keys [w*run, w*run + run) in rounds of 32) and returns, per key, its
// destination inside the tile's digit-sorted order.  dcount[d] receives the
// number of keys with digit d in this tile; dstart[d] their exclusive start.
template <int ITEMS, int WARPS>
__device__ __forceinline__ void rank_tile(const uint32_t (&key)[ITEMS], const bool (&valid)[ITEMS],
                                          int shift, uint32_t (&pos)[ITEMS],
                                          uint32_t (*wcnt)[kBins], uint32_t *dcount,
                                          uint32_t *dstart, uint32_t *wsum)
{
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned lt = lanemask_lt();
    for (int i = threadIdx.x; i < WARPS * kBins; i += WARPS * 32)
        (&wcnt[0][0])[i] = 0;
    __syncthreads();
    int dg[ITEMS];
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        dg[i] = valid[i] ? (int)((key[i] >> shift) & 0xffu) : kBins;
        const unsigned peers = __match_any_sync(RT_FULL, dg[i]);
        const uint32_t prev = dg[i] < kBins ? wcnt[w][dg[i]] : 0u;
        pos[i] = prev + __popc(peers & lt);
        __syncwarp();
        if (dg[i] < kBins && lane == __ffs(peers) - 1)
            wcnt[w][dg[i]] = prev + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    for (int d = threadIdx.x; d < kBins; d += WARPS * 32) {
        uint32_t run = 0;
#pragma unroll
        for (int x = 0; x < WARPS; ++x) {
            const uint32_t c = wcnt[x][d];
            wcnt[x][d] = run;
            run += c;
        }
        dcount[d] = run;
    }
    __syncthreads();
    // exclusive scan of dcount over 256 digits (WARPS*32 >= 256 threads)
    {
        const int d = threadIdx.x;
        const uint32_t v = d < kBins ? dcount[d] : 0u;
        uint32_t inc = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t u = __shfl_up_sync(RT_FULL, inc, o);
            if (lane >= o)
                inc += u;
        }
        if (lane == 31)
            wsum[w] = inc;
        __syncthreads();
        uint32_t add = 0;
        for (int x = 0; x < w; ++x)
            add += wsum[x];
        if (d < kBins)
            dstart[d] = add + inc - v;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < ITEMS; ++i)
        if (dg[i] < kBins)
            pos[i] += dstart[dg[i]] + wcnt[w][dg[i]];
}

__global__ void __launch_bounds__(kMidThreads)
    k_sort_mid(const int32_t *__restrict__ list, int64_t cnt, const int64_t *__restrict__ off,
               int32_t *__restrict__ ids)
{
    __shared__ uint32_t buf[2][kMidMax];
    __shared__ uint32_t wcnt[kMidWarps][kBins];
    __shared__ uint32_t dcount[kBins], dstart[kBins], wsum[kMidWarps];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int64_t b = blockIdx.x; b < cnt; b += gridDim.x) {
        const int32_t seg = list[b];
        const int64_t o = off[seg];
        const int n = (int)(off[seg + 1] - o);
        // warp w owns [w*run, (w+1)*run), run a multiple of 32
        const int run = ((n + kMidWarps * 32 - 1) / (kMidWarps * 32)) * 32;
        uint32_t a_and = 0xffffffffu, a_or = 0;
        uint32_t key[kMidItems];
        bool valid[kMidItems];
#pragma unroll
        for (int i = 0; i < kMidItems; ++i) {
            const int p = w * run + i * 32 + lane;
            valid[i] = (i * 32 < run) && p < n;
            key[i] = valid[i] ? ((uint32_t)ids[o + p] ^ kSign) : 0u;
            if (valid[i]) {
                a_and &= key[i];
                a_or |= key[i];
            }
        }
        block_and_or(a_and, a_or);
        const uint32_t diff = a_and ^ a_or;
        int cur = 0;
        for (int shift = 0; shift < 32; shift += 8) {
            if (((diff >> shift) & 0xffu) == 0)
                continue;
            uint32_t pos[kMidItems];
            rank_tile<kMidItems, kMidWarps>(key, valid, shift, pos, wcnt, dcount, dstart, wsum);
#pragma unroll
            for (int i = 0; i < kMidItems; ++i)
                if (valid[i])
                    buf[cur][pos[i]] = key[i];
            __syncthreads();
            // reload in the same ownership pattern for the next pass
#pragma unroll
            for (int i = 0; i < kMidItems; ++i) {
                const int p = w * run + i * 32 + lane;
                if (valid[i])
                    key[i] = buf[cur][p];
            }
            __syncthreads();
            cur ^= 1;
        }
#pragma unroll
        for (int i = 0; i < kMidItems; ++i) {
            const int p = w * run + i * 32 + lane;
            if (valid[i])
                ids[o + p] = (int32_t)(key[i] ^ kSign);
        }
        __syncthreads();
    }
}

// One CTA per long segment; the segment and an equal scratch area ping-pong.
__global__ void __launch_bounds__(kMidThreads)
    k_sort_large(const int32_t *__restrict__ list, const int64_t *__restrict__ tmp_off,
                 int64_t cnt, const int64_t *__restrict__ off, int32_t *__restrict__ ids,
                 uint32_t *__restrict__ scratch)
{
    __shared__ uint32_t wcnt[kMidWarps][kBins];
    __shared__ uint32_t dcount[kBins], dstart[kBins], wsum[kMidWarps];
    __shared__ uint32_t hist[kBins], running[kBins];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int kTile = kMidMax;
    constexpr int kRun = kTile / kMidWarps;  // 512 per warp per tile
    for (int64_t b = blockIdx.x; b < cnt; b += gridDim.x) {
        const int32_t seg = list[b];
        const int64_t o = off[seg];
        const int64_t n = off[seg + 1] - o;
        uint32_t *a = reinterpret_cast<uint32_t *>(ids + o);
        uint32_t *t = scratch + tmp_off[b];
        uint32_t a_and = 0xffffffffu, a_or = 0;
        for (int64_t p = threadIdx.x; p < n; p += kMidThreads) {
            const uint32_t k = a[p] ^ kSign;
            a[p] = k;
            a_and &= k;
            a_or |= k;
        }
        block_and_or(a_and, a_or);  // includes a barrier: a[] is fully flipped
        const uint32_t diff = a_and ^ a_or;
        uint32_t *src = a, *dst = t;
        for (int shift = 0; shift < 32; shift += 8) {
            if (((diff >> shift) & 0xffu) == 0)
                continue;
            for (int d = threadIdx.x; d < kBins; d += kMidThreads)
                hist[d] = 0;
            __syncthreads();
            for (int64_t p = threadIdx.x; p < n; p += kMidThreads)
                atomicAdd(&hist[(src[p] >> shift) & 0xffu], 1u);
            __syncthreads();
            if (threadIdx.x < 32) {  // exclusive scan of 256 bins by one warp
                uint32_t carry = 0;
                for (int c = 0; c < kBins; c += 32) {
                    const uint32_t v = hist[c + lane];
                    uint32_t inc = v;
#pragma unroll
                    for (int d = 1; d < 32; d <<= 1) {
                        const uint32_t u = __shfl_up_sync(RT_FULL, inc, d);
                        if (lane >= d)
                            inc += u;
                    }
                    running[c + lane] = carry + inc - v;
                    carry += __shfl_sync(RT_FULL, inc, 31);
                }
            }
            __syncthreads();
            for (int64_t t0 = 0; t0 < n; t0 += kTile) {
                uint32_t key[kMidItems], pos[kMidItems];
                bool valid[kMidItems];
#pragma unroll
                for (int i = 0; i < kMidItems; ++i) {
                    const int64_t p = t0 + w * kRun + i * 32 + lane;
                    valid[i] = p < n;
                    key[i] = valid[i] ? src[p] : 0u;
                }
                rank_tile<kMidItems, kMidWarps>(key, valid, shift, pos, wcnt, dcount, dstart, wsum);
#pragma unroll
                for (int i = 0; i < kMidItems; ++i) {
                    if (valid[i]) {
                        const uint32_t d = (key[i] >> shift) & 0xffu;
                        dst[running[d] + (pos[i] - dstart[d])] = key[i];
                    }
                }
                __syncthreads();
                for (int d = threadIdx.x; d < kBins; d += kMidThreads)
                    running[d] += dcount[d];
                __syncthreads();
            }
            uint32_t *x = src;
            src = dst;
            dst = x;
            __syncthreads();
        }
        for (int64_t p = threadIdx.x; p < n; p += kMidThreads)
            a[p] = src[p] ^ kSign;  // src is a or t; either way a ends sorted
        __syncthreads();
    }
}

}  // namespace

rtree_status segmented_sort(int32_t *ids, const int64_t *offsets, int64_t nseg, int64_t total,
                            cudaStream_t s)
{
    if (nseg <= 0 || total <= 1)
        return RTREE_OK;
    if (nseg >= (int64_t)INT32_MAX)
        return fail(RTREE_EOVERFLOW, "too many segments to sort (%lld)", (long long)nseg);
    DevBuf<int32_t> small(s), mid(s), large(s);
    DevBuf<int64_t> large_tmp(s);
    DevBuf<unsigned long long> hdr(s);
    RT_TRY(small.alloc(nseg, "sort lists"));
    RT_TRY(mid.alloc(nseg, "sort lists"));
    RT_TRY(large.alloc(nseg, "sort lists"));
    RT_TRY(large_tmp.alloc(nseg, "sort lists"));
    RT_TRY(hdr.alloc(4, "sort counters"));
    RT_CUDA(cudaMemsetAsync(hdr.p, 0, 4 * sizeof(unsigned long long), s));
    const int sms = sm_count();
    {
        int64_t blocks = (nseg + 255) / 256;
        if (blocks > (int64_t)sms * 16)
            blocks = (int64_t)sms * 16;
        {
            KernelTimer kt_("classify", s);
            k_classify<<<(unsigned)blocks, 256, 0, s>>>(offsets, nseg, small.p, mid.p, large.p,
                                                        large_tmp.p, hdr.p);
            RT_LAUNCH();
        }
    }
    unsigned long long h[4];
    RT_CUDA(cudaMemcpyAsync(h, hdr.p, sizeof(h), cudaMemcpyDeviceToHost, s));
    RT_CUDA(cudaStreamSynchronize(s));
    if (h[HDR_SMALL]) {
        int64_t blocks = ((int64_t)h[HDR_SMALL] + 7) / 8;
        if (blocks > (int64_t)sms * 32)
            blocks = (int64_t)sms * 32;
        {
            KernelTimer kt_("sort_small", s);
            k_sort_small<<<(unsigned)blocks, 256, 0, s>>>(small.p, (int64_t)h[HDR_SMALL], offsets, ids);
            RT_LAUNCH();
        }
    }
    if (h[HDR_MID]) {
        int64_t blocks = (int64_t)h[HDR_MID];
        if (blocks > (int64_t)sms * 8)
            blocks = (int64_t)sms * 8;
        {
            KernelTimer kt_("sort_mid", s);
            k_sort_mid<<<(unsigned)blocks, kMidThreads, 0, s>>>(mid.p, (int64_t)h[HDR_MID], offsets, ids);
            RT_LAUNCH();
        }
    }
    if (h[HDR_LARGE]) {
        DevBuf<uint32_t> scratch(s);
        RT_TRY(scratch.alloc(h[HDR_SCRATCH], "sort scratch"));
        int64_t blocks = (int64_t)h[HDR_LARGE];
        if (blocks > (int64_t)sms * 4)
            blocks = (int64_t)sms * 4;
        {
            KernelTimer kt_("sort_large", s);
            k_sort_large<<<(unsigned)blocks, kMidThreads, 0, s>>>(large.p, large_tmp.p,
                                                                  (int64_t)h[HDR_LARGE], offsets, ids,
                                                                  scratch.p);
            RT_LAUNCH();
        }
    }
    return RTREE_OK;
}

}  // namespace rt
