// radix_sort.cu -- stable LSD radix sort of (uint32 key, uint32 value) pairs.
//
// Used by the STR bulk load (sort by centre key, then by slab), by the query
// ordering and by the join (lexicographic sort of result pairs).  Each 8-bit
// digit pass is reduce-then-scan over a persistent grid of G CTAs, each
// owning a contiguous run of 4096-item tiles:
//   k_hist     CTA c counts the digits of its run: hist[d * G + c];
//   k_scan     one CTA per digit scans its row: offs[d * G + c] = items of
//              digit d in CTAs before c, and the digit's total;
//   k_scatter  CTA c walks its tiles in order, keeping a running offset per
//              digit: each tile is ranked in shared memory and written out
//              one digit run after another.
// No CTA waits for another.  Stability: items are ranked in input order
// inside a tile (each warp owns a contiguous run of the tile and walks it 32
// items at a time; lanes holding the same digit find each other with one
// ballot per digit bit and rank by lane order on top of a per-warp running
// count), tiles are taken in order inside a CTA, and CTAs own consecutive
// runs.
#include "internal.cuh"

namespace rt {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kItems = 16;
constexpr int kTile = kThreads * kItems;  // 4096
constexpr int kBins = 256;
constexpr int kWarpRun = 32 * kItems;     // contiguous items owned by one warp
static_assert(kThreads == kBins, "one thread per digit");

// Tiles [t0, t1) of CTA c out of G (balanced: they differ by at most one).
__device__ __forceinline__ void run_of(int64_t ntiles, int G, int c, int64_t &t0, int64_t &t1)
{
    t0 = ntiles * c / G;
    t1 = ntiles * (c + 1) / G;
}

// Lanes of the warp whose digit equals this lane's (all lanes valid or not
// take part; the answer is meaningful for valid lanes), from one ballot per
// digit bit.
__device__ __forceinline__ unsigned peers_of(int dg, uint32_t mask, bool ok)
{
    unsigned peers = __ballot_sync(RT_FULL, ok);
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        if (!((mask >> b) & 1u))
            break;
        const unsigned m = __ballot_sync(RT_FULL, (dg >> b) & 1);
        peers &= (dg >> b) & 1 ? m : ~m;
    }
    return peers;
}

// Exclusive scan of one value per thread across the block (wsum: one word
// per warp of shared memory); every thread gets its prefix.
template <int THREADS>
__device__ __forceinline__ uint32_t block_excl(uint32_t v, uint32_t *wsum)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
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
    __syncthreads();
    return add + inc - v;
}

__global__ void __launch_bounds__(kThreads) k_hist(const uint32_t *__restrict__ keys, int64_t n,
                                                   int shift, uint32_t mask, int64_t ntiles, int G,
                                                   uint32_t *__restrict__ hist)
{
    __shared__ uint32_t h[kWarps][kBins];
    for (int i = threadIdx.x; i < kWarps * kBins; i += kThreads)
        (&h[0][0])[i] = 0;
    __syncthreads();
    int64_t t0, t1;
    run_of(ntiles, G, blockIdx.x, t0, t1);
    const int64_t b = t0 * kTile, e = t1 * kTile < n ? t1 * kTile : n;
    const int w = threadIdx.x >> 5;
#pragma unroll 8
    for (int64_t k = b + threadIdx.x; k < e; k += kThreads)
        atomicAdd(&h[w][(__ldg(keys + k) >> shift) & mask], 1u);
    __syncthreads();
    const int d = threadIdx.x;
    uint32_t s = 0;
#pragma unroll
    for (int x = 0; x < kWarps; ++x)
        s += h[x][d];
    hist[(int64_t)d * G + blockIdx.x] = s;
}

// Per digit d (one CTA each): exclusive scan of hist[d*G .. d*G+G) into
// offs (the digit's CTAs in order) and the digit's total into tot[d].
__global__ void __launch_bounds__(kThreads) k_scan(const uint32_t *__restrict__ hist, int G,
                                                   uint32_t *__restrict__ offs, uint32_t *__restrict__ tot)
{
    __shared__ uint32_t wsum[kWarps];
    const int64_t row = (int64_t)blockIdx.x * G;
    const int per = (G + kThreads - 1) / kThreads;
    const int lo = threadIdx.x * per, hi = lo + per < G ? lo + per : G;
    uint32_t s = 0;
    for (int i = lo; i < hi; ++i)
        s += hist[row + i];
    const uint32_t before = block_excl<kThreads>(s, wsum);
    uint32_t run = before;
    for (int i = lo; i < hi; ++i) {
        const uint32_t v = hist[row + i];
        offs[row + i] = run;
        run += v;
    }
    if (threadIdx.x == kThreads - 1)
        tot[blockIdx.x] = run;
}

// Four CTAs per SM (64 registers a thread): the tiles' loads of one CTA
// overlap the ranking of the others.
__global__ void __launch_bounds__(kThreads, 4)
    k_scatter(const uint32_t *__restrict__ kin, const uint32_t *__restrict__ vin,
              uint32_t *__restrict__ kout, uint32_t *__restrict__ vout, int64_t n, int shift,
              uint32_t mask, const uint32_t *__restrict__ offs, const uint32_t *__restrict__ tot,
              int64_t ntiles, int G)
{
    __shared__ uint32_t wcnt[kWarps][kBins];
    __shared__ uint32_t tstart[kBins];
    __shared__ uint32_t base[kBins];  // where this CTA's next item of each digit goes
    __shared__ uint32_t wsum[kWarps];
    __shared__ uint32_t sk[kTile];
    __shared__ uint32_t sv[kTile];

    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, d = threadIdx.x;
    const unsigned lt = lanemask_lt();
    int64_t t0, t1;
    run_of(ntiles, G, blockIdx.x, t0, t1);
    // items of smaller digits come first, then this digit's items of earlier CTAs
    base[d] = block_excl<kThreads>(tot[d], wsum) + offs[(int64_t)d * G + blockIdx.x];
    for (int64_t tile = t0; tile < t1; ++tile) {
        for (int i = threadIdx.x; i < kWarps * kBins; i += kThreads)
            (&wcnt[0][0])[i] = 0;
        __syncthreads();  // also: the previous tile's staging is written out

        const int64_t tile0 = tile * kTile;
        const int64_t wbase = tile0 + (int64_t)w * kWarpRun;
        uint32_t k[kItems], rank[kItems];
#pragma unroll
        for (int i = 0; i < kItems; ++i) {
            const int64_t idx = wbase + i * 32 + lane;
            k[i] = idx < n ? __ldg(kin + idx) : 0u;
        }
#pragma unroll
        for (int i = 0; i < kItems; ++i) {
            const bool ok = wbase + i * 32 + lane < n;
            const int dg = (int)((k[i] >> shift) & mask);
            const unsigned peers = peers_of(dg, mask, ok);
            const uint32_t prev = ok ? wcnt[w][dg] : 0u;
            rank[i] = prev + __popc(peers & lt);
            __syncwarp();
            if (ok && lane == __ffs(peers) - 1)
                wcnt[w][dg] = prev + __popc(peers);
            __syncwarp();
        }
        __syncthreads();

        // per digit: exclusive prefix over warps (in place) and the tile's count
        uint32_t cnt = 0;
#pragma unroll
        for (int x = 0; x < kWarps; ++x) {
            const uint32_t c = wcnt[x][d];
            wcnt[x][d] = cnt;
            cnt += c;
        }
        tstart[d] = block_excl<kThreads>(cnt, wsum);  // the digit runs' starts in the tile
        __syncthreads();

        // stage the tile in digit order: keys, then values (read only now)
#pragma unroll
        for (int i = 0; i < kItems; ++i) {
            if (wbase + i * 32 + lane < n) {
                const int dg = (int)((k[i] >> shift) & mask);
                rank[i] += tstart[dg] + wcnt[w][dg];
                sk[rank[i]] = k[i];
            }
        }
#pragma unroll
        for (int i = 0; i < kItems; ++i) {
            const int64_t idx = wbase + i * 32 + lane;
            if (idx < n)
                sv[rank[i]] = __ldg(vin + idx);
        }
        __syncthreads();
        const int tn = (int)(n - tile0 < kTile ? n - tile0 : kTile);
        for (int p = threadIdx.x; p < tn; p += kThreads) {
            const uint32_t key = sk[p];
            const int dd = (int)((key >> shift) & mask);
            const uint32_t dst = base[dd] + (uint32_t)p - tstart[dd];
            if (dst < (uint64_t)n) {
                kout[dst] = key;
                vout[dst] = sv[p];
            }
        }
        __syncthreads();
        base[d] += cnt;
    }
}

// CTAs of the persistent grid: every SM full (at most one tile each).
int grid_for(int64_t ntiles)
{
    static const int per_sm = [] {  // initialised once, thread-safely
        int v = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_scatter, kThreads, 0) != cudaSuccess || v < 1) {
            cudaGetLastError();
            v = 1;
        }
        return v;
    }();
    const int64_t g = (int64_t)per_sm * sm_count();
    return (int)(ntiles < g ? ntiles : g);
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
    const int G = grid_for(ntiles);
    DevBuf<uint32_t> tk(s), tv(s), hist(s), offs(s), tot(s);
    if (passes > 1) {
        RT_TRY(tk.alloc(n, "radix keys"));
        RT_TRY(tv.alloc(n, "radix values"));
    }
    RT_TRY(hist.alloc((size_t)kBins * G, "radix histogram"));
    RT_TRY(offs.alloc((size_t)kBins * G, "radix offsets"));
    RT_TRY(tot.alloc(kBins, "radix digit totals"));
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
            k_hist<<<(unsigned)G, kThreads, 0, s>>>(sk, n, shift, mask, ntiles, G, hist.p);
            RT_LAUNCH();
        }
        {
            KernelTimer kt_("radix_scan", s);
            k_scan<<<kBins, kThreads, 0, s>>>(hist.p, G, offs.p, tot.p);
            RT_LAUNCH();
        }
        {
            KernelTimer kt_("scatter", s);
            k_scatter<<<(unsigned)G, kThreads, 0, s>>>(sk, sv, bk[dst], bv[dst], n, shift, mask, offs.p,
                                                       tot.p, ntiles, G);
            RT_LAUNCH();
        }
        sk = bk[dst];
        sv = bv[dst];
        dst ^= 1;
    }
    return RTREE_OK;
}

}  // namespace rt
