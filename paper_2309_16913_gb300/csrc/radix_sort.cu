// radix_sort.cu -- stable LSD radix sort of (uint32 key, uint32 value) pairs.
//
// Used by the STR bulk load (sort by centre key, then by slab) and by the
// join (lexicographic sort of result pairs).  Each 8-bit digit pass is three
// launches: per-tile digit histograms, an exclusive scan of the digit-major
// histogram table, and a stable scatter.  Stability inside a tile comes from
// ranking items in input order: each warp owns a contiguous run of the tile
// and walks it 32 items at a time; lanes holding the same digit find each
// other with __match_any_sync and rank by lane order on top of a per-warp
// running count.  The ranked tile is staged in shared memory so each digit's
// run is written out contiguously.
#include "internal.cuh"

namespace rt {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kItems = 16;
constexpr int kTile = kThreads * kItems;  // 4096
constexpr int kBins = 256;
constexpr int kWarpRun = 32 * kItems;     // contiguous items owned by one warp

__global__ void __launch_bounds__(kThreads) k_hist(const uint32_t *__restrict__ keys, int64_t n,
                                                   int shift, uint32_t mask,
                                                   uint32_t *__restrict__ hist, int64_t ntiles)
{
    __shared__ uint32_t h[kWarps][kBins];
    for (int i = threadIdx.x; i < kWarps * kBins; i += kThreads)
        (&h[0][0])[i] = 0;
    __syncthreads();
    const int w = threadIdx.x >> 5;
    const int64_t base = (int64_t)blockIdx.x * kTile;
#pragma unroll 4
    for (int i = 0; i < kItems; ++i) {
        int64_t k = base + i * kThreads + threadIdx.x;
        if (k < n)
            atomicAdd(&h[w][(__ldg(keys + k) >> shift) & mask], 1u);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < kBins; d += kThreads) {
        uint32_t s = 0;
#pragma unroll
        for (int x = 0; x < kWarps; ++x)
            s += h[x][d];
        hist[(int64_t)d * ntiles + blockIdx.x] = s;
    }
}

__global__ void __launch_bounds__(kThreads) k_scatter(const uint32_t *__restrict__ kin,
                                                      const uint32_t *__restrict__ vin,
                                                      uint32_t *__restrict__ kout,
                                                      uint32_t *__restrict__ vout, int64_t n,
                                                      int shift, uint32_t mask,
                                                      const uint32_t *__restrict__ offs,
                                                      int64_t ntiles)
{
    __shared__ uint32_t wcnt[kWarps][kBins];
    __shared__ uint32_t tstart[kBins];
    __shared__ uint32_t gbase[kBins];
    __shared__ uint32_t wsum[kWarps];
    __shared__ uint32_t sk[kTile];
    __shared__ uint32_t sv[kTile];

    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned lt = lanemask_lt();
    for (int i = threadIdx.x; i < kWarps * kBins; i += kThreads)
        (&wcnt[0][0])[i] = 0;
    __syncthreads();

    const int64_t tile0 = (int64_t)blockIdx.x * kTile;
    const int64_t wbase = tile0 + (int64_t)w * kWarpRun;
    uint32_t k[kItems], v[kItems], rank[kItems];
    int dg[kItems];
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        int64_t idx = wbase + i * 32 + lane;
        bool ok = idx < n;
        k[i] = ok ? __ldg(kin + idx) : 0u;
        v[i] = ok ? __ldg(vin + idx) : 0u;
        dg[i] = ok ? (int)((k[i] >> shift) & mask) : kBins;  // kBins: past the end
    }
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        unsigned peers = __match_any_sync(RT_FULL, dg[i]);
        uint32_t prev = dg[i] < kBins ? wcnt[w][dg[i]] : 0u;
        rank[i] = prev + __popc(peers & lt);
        __syncwarp();
        if (dg[i] < kBins && lane == __ffs(peers) - 1)
            wcnt[w][dg[i]] = prev + __popc(peers);
        __syncwarp();
    }
    __syncthreads();

    // Per digit: exclusive prefix over warps (in place) and the tile total.
    const int d = threadIdx.x;  // kThreads == kBins
    uint32_t run = 0;
#pragma unroll
    for (int x = 0; x < kWarps; ++x) {
        uint32_t c = wcnt[x][d];
        wcnt[x][d] = run;
        run += c;
    }
    // Exclusive scan of the digit totals across the block.
    uint32_t inc = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t u = __shfl_up_sync(RT_FULL, inc, o);
        if (lane >= o)
            inc += u;
    }
    if (lane == 31)
        wsum[w] = inc;
    gbase[d] = offs[(int64_t)d * ntiles + blockIdx.x];
    __syncthreads();
    uint32_t add = 0;
    for (int x = 0; x < w; ++x)
        add += wsum[x];
    tstart[d] = add + inc - run;
    __syncthreads();

#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        if (dg[i] < kBins) {
            uint32_t pos = tstart[dg[i]] + wcnt[w][dg[i]] + rank[i];
            sk[pos] = k[i];
            sv[pos] = v[i];
        }
    }
    __syncthreads();
    const int tn = (int)((n - tile0) < kTile ? (n - tile0) : kTile);
    for (int p = threadIdx.x; p < tn; p += kThreads) {
        uint32_t key = sk[p];
        int dd = (int)((key >> shift) & mask);
        uint32_t dst = gbase[dd] + (uint32_t)p - tstart[dd];
        if (dst < (uint64_t)n) {
            kout[dst] = key;
            vout[dst] = sv[p];
        }
    }
}

}  // namespace

rtree_status radix_sort_pairs(const uint32_t *kin, const uint32_t *vin, uint32_t *kout,
                              uint32_t *vout, int64_t n, int bit_lo, int bit_hi, cudaStream_t s)
{
    if (n <= 0)
        return RTREE_OK;
    if (n >= (int64_t)1 << 31)
        return fail(RTREE_EOVERFLOW, "radix sort of %lld items exceeds 2^31", (long long)n);
    if (bit_hi <= bit_lo) {
        RT_CUDA(cudaMemcpyAsync(kout, kin, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
        RT_CUDA(cudaMemcpyAsync(vout, vin, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
        return RTREE_OK;
    }
    const int passes = (bit_hi - bit_lo + 7) / 8;
    const int64_t ntiles = (n + kTile - 1) / kTile;
    DevBuf<uint32_t> tk(s), tv(s), hist(s), offs(s);
    RT_TRY(tk.alloc(n, "radix keys"));
    RT_TRY(tv.alloc(n, "radix values"));
    RT_TRY(hist.alloc((size_t)kBins * ntiles, "radix histogram"));
    RT_TRY(offs.alloc((size_t)kBins * ntiles + 1, "radix offsets"));
    // Ping-pong so that the last pass writes kout/vout.
    uint32_t *bk[2] = {kout, tk.p}, *bv[2] = {vout, tv.p};
    int dst = (passes % 2 == 1) ? 0 : 1;
    const uint32_t *sk = kin, *sv = vin;
    for (int p = 0; p < passes; ++p) {
        const int shift = bit_lo + 8 * p;
        const int bits = min(8, bit_hi - shift);
        const uint32_t mask = (1u << bits) - 1u;
        {
            KernelTimer kt_("hist", s);
            k_hist<<<(unsigned)ntiles, kThreads, 0, s>>>(sk, n, shift, mask, hist.p, ntiles);
            RT_LAUNCH();
        }
        RT_TRY(scan_exclusive(hist.p, offs.p, (int64_t)kBins * ntiles, s));
        {
            KernelTimer kt_("scatter", s);
            k_scatter<<<(unsigned)ntiles, kThreads, 0, s>>>(sk, sv, bk[dst], bv[dst], n, shift, mask,
                                                            offs.p, ntiles);
            RT_LAUNCH();
        }
        sk = bk[dst];
        sv = bv[dst];
        dst ^= 1;
    }
    return RTREE_OK;
}

}  // namespace rt
