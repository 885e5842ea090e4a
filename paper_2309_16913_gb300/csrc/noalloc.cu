// noalloc.cu -- range select into caller-owned buffers, allocating nothing.
//
// Some callers cannot allocate device memory once they are running: a host
// application that reserves all of the GPU's memory for its own pool at
// start-up (so the CUDA allocator has nothing left to give), or a request
// loop with a latency budget that must neither block in the allocator nor
// fail with out-of-memory halfway through a request.  For them,
// rtree_range_select_noalloc takes the queries and both output buffers from
// the caller, and keeps the library's own temporary storage (per-query
// counts, two work counters, an error word) in one fixed array in device
// global memory, declared below.  The call makes no cudaMalloc, cudaFree or
// other allocating call.
//
// The array is a file-scope __device__ variable, so every GPU that loads the
// library holds its kNoallocScratchBytes until the process exits.  All calls
// share it: calls whose device work overlaps (different streams, or other
// host threads) race on it and must be serialized by the caller.
#include <cstring>
#include <mutex>

#include "internal.cuh"

namespace rt {
namespace {

constexpr int64_t kNoallocMaxQueries = 65536;
constexpr size_t kCountsBytes = kNoallocMaxQueries * sizeof(int32_t);  // 256 KiB
constexpr size_t kCtrOffset = kCountsBytes;                            // 2 x u64
constexpr size_t kFlagsOffset = kCtrOffset + 2 * sizeof(unsigned long long);
constexpr size_t kNoallocScratchBytes = kCountsBytes + 256;

// The scratch: written and read only by the kernels this file launches.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char *g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch on the current device.  In host code the
// array's name is only a host-side handle, so the address is asked of the
// runtime once per device (with that device current) and cached.
rtree_status scratch_address(int dev, unsigned char **out)
{
    if (dev < 0 || dev >= kMaxDevices)
        return fail(RTREE_EINVAL, "rtree_range_select_noalloc: device %d out of range", dev);
    std::lock_guard<std::mutex> g(g_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return fail(RTREE_ECUDA, "rtree_range_select_noalloc: cudaGetSymbolAddress failed: %s",
                        cudaGetErrorString(e));
        }
        g_scratch_addr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_scratch_addr[dev];
    return RTREE_OK;
}

// True if p is device (or managed) memory that the kernels on `dev` can
// address directly: memory of another GPU is refused, since reaching it
// would need peer access.
bool is_device_memory_on(const void *p, int dev)
{
    cudaPointerAttributes a;
    memset(&a, 0, sizeof(a));
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged)
        return true;
    return a.type == cudaMemoryTypeDevice && a.device == dev;
}

// Exclusive scan of at most kNoallocMaxQueries counts by one block;
// out[n] receives the total.
__global__ void __launch_bounds__(1024) k_noalloc_scan(const int32_t *__restrict__ in, int64_t n,
                                                       int64_t *__restrict__ out)
{
    __shared__ int64_t warp_sum[32];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const int64_t per = (n + 1023) / 1024;
    const int64_t lo = t * per, hi = lo + per < n ? lo + per : n;
    int64_t s = 0;
    for (int64_t i = lo; i < hi; ++i)
        s += in[i];
    int64_t inc = s;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int64_t u = __shfl_up_sync(RT_FULL, inc, d);
        if (lane >= d)
            inc += u;
    }
    if (lane == 31)
        warp_sum[w] = inc;
    __syncthreads();
    int64_t before = 0;
    for (int x = 0; x < w; ++x)
        before += warp_sum[x];
    int64_t run = before + inc - s;
    for (int64_t i = lo; i < hi; ++i) {
        out[i] = run;
        run += in[i];
    }
    if (t == 1023) {
        int64_t total = 0;
        for (int x = 0; x < 32; ++x)
            total += warp_sum[x];
        out[n] = total;
    }
}

struct CurrentDevice {
    int prev = -1;
    explicit CurrentDevice(int dev)
    {
        cudaGetDevice(&prev);
        if (dev != prev)
            cudaSetDevice(dev);
    }
    ~CurrentDevice()
    {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev)
            cudaSetDevice(prev);
    }
};

}  // namespace
}  // namespace rt

using namespace rt;

extern "C" rtree_status rtree_range_select_noalloc(const rtree_t *t, const float *queries, int64_t q,
                                                   int64_t *offsets, int32_t *ids, int64_t capacity,
                                                   int64_t *total, void *stream)
{
    clear_error();
    if (!t || !total)
        return fail(RTREE_EINVAL, "rtree_range_select_noalloc: tree and total must not be NULL");
    *total = 0;
    if (q < 0)
        return fail(RTREE_EINVAL, "rtree_range_select_noalloc: q = %lld is negative", (long long)q);
    if (q > kNoallocMaxQueries)
        return fail(RTREE_EOVERFLOW,
                    "rtree_range_select_noalloc: q = %lld exceeds the fixed maximum of %lld queries "
                    "per call (split the batch)",
                    (long long)q, (long long)kNoallocMaxQueries);
    if (capacity < 0 || !offsets || (capacity > 0 && !ids) || (q > 0 && !queries))
        return fail(RTREE_EINVAL, "rtree_range_select_noalloc: NULL buffer or negative capacity");
    if (!is_device_memory_on(offsets, t->device) || (q > 0 && !is_device_memory_on(queries, t->device)) ||
        (capacity > 0 && !is_device_memory_on(ids, t->device)))
        return fail(RTREE_EINVAL, "rtree_range_select_noalloc: queries, offsets and ids must be "
                                  "device memory on the tree's device (%d)", t->device);
    if ((reinterpret_cast<uintptr_t>(queries) & 15) || (reinterpret_cast<uintptr_t>(offsets) & 7) ||
        (reinterpret_cast<uintptr_t>(ids) & 3))
        return fail(RTREE_EINVAL, "rtree_range_select_noalloc: queries must be 16-byte aligned, "
                                  "offsets 8-byte aligned, ids 4-byte aligned");
    CurrentDevice guard(t->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    RT_TRY(tree_ready_on(t, s));
    unsigned char *scratch = nullptr;
    RT_TRY(scratch_address(t->device, &scratch));
    int32_t *counts = reinterpret_cast<int32_t *>(scratch);
    unsigned long long *ctr = reinterpret_cast<unsigned long long *>(scratch + kCtrOffset);
    int32_t *flags = reinterpret_cast<int32_t *>(scratch + kFlagsOffset);
    const float4 *q4 = reinterpret_cast<const float4 *>(queries);

    // The array keeps the previous call's contents: reset what must start at 0.
    RT_CUDA(cudaMemsetAsync(ctr, 0, 2 * sizeof(unsigned long long), s));
    RT_CUDA(cudaMemsetAsync(flags, 0, sizeof(int32_t), s));
    if (q == 0 || t->nodes == 0) {
        RT_CUDA(cudaMemsetAsync(offsets, 0, (q + 1) * sizeof(int64_t), s));
        RT_CUDA(cudaStreamSynchronize(s));
        return RTREE_OK;
    }
    RT_TRY(select_pass(t, q4, q, counts, nullptr, nullptr, ctr, flags, s));
    {
        KernelTimer kt_("noalloc_scan", s);
        k_noalloc_scan<<<1, 1024, 0, s>>>(counts, q, offsets);
        RT_LAUNCH();
    }
    int64_t h_total = 0;
    int32_t h_flags = 0;
    RT_CUDA(cudaMemcpyAsync(&h_total, offsets + q, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    RT_CUDA(cudaMemcpyAsync(&h_flags, flags, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    RT_CUDA(cudaStreamSynchronize(s));
    if (h_flags)
        return fail(RTREE_EINTERNAL, "rtree_range_select_noalloc: count pass flags 0x%x", h_flags);
    *total = h_total;
    if (h_total > capacity)
        return fail(RTREE_EOVERFLOW,
                    "rtree_range_select_noalloc: result has %lld ids but ids holds %lld; offsets "
                    "and *total are valid, ids was not written",
                    (long long)h_total, (long long)capacity);
    RT_TRY(select_pass(t, q4, q, nullptr, offsets, ids, ctr + 1, flags, s));
    RT_CUDA(cudaMemcpyAsync(&h_flags, flags, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    RT_CUDA(cudaStreamSynchronize(s));
    if (h_flags)
        return fail(RTREE_EINTERNAL, "rtree_range_select_noalloc: scatter pass flags 0x%x", h_flags);
    timing_resolve();
    return RTREE_OK;
}
