// scan.cu -- exclusive prefix sums (reduce, scan of tile sums, scan tiles).
//
// Used for CSR offsets (per-query hit counts -> int64 offsets) and for the
// digit-major histograms of the radix sort.  out has n+1 entries; out[n] is
// the total, so one 8-byte read gives the output size.
#include "internal.cuh"

namespace rt {
namespace {

constexpr int kThreads = 256;
constexpr int kItems = 8;
constexpr int kTile = kThreads * kItems;

template <typename T>
__device__ __forceinline__ T warp_incl_scan(T v)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        T u = __shfl_up_sync(RT_FULL, v, d);
        if (lane >= d)
            v += u;
    }
    return v;
}

// Exclusive block scan of one value per thread; also returns the block total.
template <typename T>
__device__ __forceinline__ T block_excl_scan(T v, T &total)
{
    __shared__ T warp_tot[kThreads / 32];
    __shared__ T tot_sh;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    T inc = warp_incl_scan(v);
    if (lane == 31)
        warp_tot[w] = inc;
    __syncthreads();
    if (w == 0) {
        T t = lane < kThreads / 32 ? warp_tot[lane] : T(0);
        T ti = warp_incl_scan(t);
        if (lane < kThreads / 32)
            warp_tot[lane] = ti - t;
        if (lane == kThreads / 32 - 1)
            tot_sh = ti;
    }
    __syncthreads();
    total = tot_sh;
    T r = warp_tot[w] + inc - v;
    __syncthreads();  // the shared words may be reused by a later call
    return r;
}

template <typename Tin, typename Tout>
__global__ void __launch_bounds__(kThreads) k_tile_reduce(const Tin *__restrict__ in, int64_t n,
                                                          Tout *__restrict__ sums)
{
    const int64_t base = (int64_t)blockIdx.x * kTile;
    Tout acc = 0;
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        int64_t k = base + i * kThreads + threadIdx.x;
        if (k < n)
            acc += (Tout)in[k];
    }
    Tout total;
    block_excl_scan<Tout>(acc, total);
    if (threadIdx.x == 0)
        sums[blockIdx.x] = total;
}

// Scans one tile; tile_base (may be null) gives each tile's starting value.
// The last tile writes out[n] = total.
template <typename Tin, typename Tout>
__global__ void __launch_bounds__(kThreads) k_tile_scan(const Tin *__restrict__ in, int64_t n,
                                                        const Tout *__restrict__ tile_base,
                                                        Tout *__restrict__ out)
{
    __shared__ Tout sm[kTile];
    const int64_t base = (int64_t)blockIdx.x * kTile;
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        int p = i * kThreads + threadIdx.x;
        int64_t k = base + p;
        sm[p] = k < n ? (Tout)in[k] : Tout(0);
    }
    __syncthreads();
    Tout v[kItems];
    Tout run = 0;
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        v[i] = sm[threadIdx.x * kItems + i];
        run += v[i];
    }
    Tout total;
    Tout pre = block_excl_scan<Tout>(run, total);
    const Tout tb = tile_base ? tile_base[blockIdx.x] : Tout(0);
    pre += tb;
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        sm[threadIdx.x * kItems + i] = pre;
        pre += v[i];
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        int p = i * kThreads + threadIdx.x;
        int64_t k = base + p;
        if (k < n)
            out[k] = sm[p];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0)
        out[n] = tb + total;
}

template <typename Tin, typename Tout>
rtree_status scan_impl(const Tin *in, Tout *out, int64_t n, cudaStream_t s)
{
    if (n <= 0) {
        RT_CUDA(cudaMemsetAsync(out, 0, sizeof(Tout), s));
        return RTREE_OK;
    }
    const int64_t tiles = (n + kTile - 1) / kTile;
    if (tiles > INT32_MAX)
        return fail(RTREE_EOVERFLOW, "scan of %lld elements exceeds the grid limit", (long long)n);
    if (tiles == 1) {
        {
            KernelTimer kt_("tile_scan", s);
            k_tile_scan<Tin, Tout><<<1, kThreads, 0, s>>>(in, n, nullptr, out);
            RT_LAUNCH();
        }
        return RTREE_OK;
    }
    DevBuf<Tout> sums(s), sums_scan(s);
    RT_TRY(sums.alloc(tiles, "scan tile sums"));
    RT_TRY(sums_scan.alloc(tiles + 1, "scan tile offsets"));
    {
        KernelTimer kt_("tile_reduce", s);
        k_tile_reduce<Tin, Tout><<<(unsigned)tiles, kThreads, 0, s>>>(in, n, sums.p);
        RT_LAUNCH();
    }
    RT_TRY((scan_impl<Tout, Tout>(sums.p, sums_scan.p, tiles, s)));
    {
        KernelTimer kt_("tile_scan", s);
        k_tile_scan<Tin, Tout><<<(unsigned)tiles, kThreads, 0, s>>>(in, n, sums_scan.p, out);
        RT_LAUNCH();
    }
    return RTREE_OK;
}

}  // namespace

rtree_status scan_exclusive(const int32_t *in, int64_t *out, int64_t n, cudaStream_t s)
{
    return scan_impl<int32_t, int64_t>(in, out, n, s);
}
rtree_status scan_exclusive(const uint32_t *in, uint32_t *out, int64_t n, cudaStream_t s)
{
    return scan_impl<uint32_t, uint32_t>(in, out, n, s);
}
rtree_status scan_exclusive(const int64_t *in, int64_t *out, int64_t n, cudaStream_t s)
{
    return scan_impl<int64_t, int64_t>(in, out, n, s);
}

}  // namespace rt
