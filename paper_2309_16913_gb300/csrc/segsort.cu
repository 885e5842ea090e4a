// segsort.cu -- sort every query's id list ascending.
//
// Results are sets; the traversal emits them in tree order, so each CSR
// segment is sorted afterwards.  The work unit is sized to the segment:
//   2..256 ids    one warp; bitonic network on 1-8 keys per lane held in
//                 registers (shuffles across lanes, swaps inside a lane);
//   257..16384    one CTA of 128-1024 threads, in shared memory with one
//                 read and one write of DRAM: bucket the keys by their top
//                 differing bits (2-4 keys per bucket for spread-out ids),
//                 insertion-sort each bucket; a crowded bucket sends the
//                 segment to an LSD radix sort with 8-bit digits instead;
//   > 16384       one CTA partitions the segment by its top differing bits
//                 into buckets of about 8K ids (MSD step, through a scratch
//                 area), then every bucket is sorted by the CTA radix sort
//                 and written back in place.
// LSD passes whose digit is equal for all keys are skipped (from the AND
// and OR of the keys).  In each LSD pass a key's rank among equal digits
// comes from walking the keys in order: each warp owns a contiguous run and
// takes it 32 at a time, with __match_any_sync grouping equal digits.  Keys
// are ids with the sign bit flipped, so unsigned order is signed order.
#include <climits>

#include "internal.cuh"

namespace rt {
namespace {

constexpr int kBins = 256;
constexpr int kItems = 16;                 // keys per thread in the CTA sort
constexpr int kCtaMax = 1024 * kItems;     // 16384: largest in-shared-memory segment
constexpr uint32_t kSign = 0x80000000u;

// Segment classes (index into the class lists).
enum {
    C_W1 = 0, C_W2, C_W4, C_W8,          // warp sorts, 32*K ids
    C_T128, C_T256, C_T512, C_T1024,     // CTA sorts, 16 ids per thread
    C_LARGE,                             // MSD partition first
    C_COUNT
};
enum { HDR_SCRATCH = C_COUNT, HDR_BUCKETS, HDR_OVERSIZE, HDR_WORDS };

struct SegDesc {
    int64_t src;  // offset of the input keys
    int64_t dst;  // offset of the output ids
    int32_t n;
    int32_t pad;
};

__device__ __forceinline__ int class_of(int64_t n)
{
    if (n <= 1) return -1;
    if (n <= 32) return C_W1;
    if (n <= 64) return C_W2;
    if (n <= 128) return C_W4;
    if (n <= 256) return C_W8;
    if (n <= 2048) return C_T128;
    if (n <= 4096) return C_T256;
    if (n <= 8192) return C_T512;
    if (n <= kCtaMax) return C_T1024;
    return C_LARGE;
}

__global__ void k_classify(const int64_t *__restrict__ off, int64_t nseg, int32_t *__restrict__ lists,
                           int64_t stride, int64_t *__restrict__ large_tmp,
                           unsigned long long *__restrict__ hdr)
{
    const int lane = threadIdx.x & 31;
    const unsigned lt = lanemask_lt();
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t b = warp * 32; b < nseg; b += nwarps * 32) {
        const int64_t i = b + lane;
        const int64_t len = i < nseg ? off[i + 1] - off[i] : 0;
        const int cls = class_of(len);
        for (int c = 0; c < C_COUNT; ++c) {
            const unsigned m = __ballot_sync(RT_FULL, cls == c);
            if (!m)
                continue;
            const int leader = __ffs(m) - 1;
            unsigned long long base = 0;
            if (lane == leader)
                base = atomicAdd(hdr + c, (unsigned long long)__popc(m));
            base = __shfl_sync(RT_FULL, base, leader);
            if (cls == c) {
                const int64_t slot = (int64_t)base + __popc(m & lt);
                lists[c * stride + slot] = (int32_t)i;
                if (c == C_LARGE)
                    large_tmp[slot] = (int64_t)atomicAdd(hdr + HDR_SCRATCH, (unsigned long long)len);
            }
        }
    }
}

// ----------------------------------------------------------- warp sorts
// Bitonic sort of up to 32*K signed ids; element e = k*32 + lane (striped).
template <int K>
__global__ void __launch_bounds__(256) k_sort_warp(const int32_t *__restrict__ list, int64_t cnt,
                                                   const int64_t *__restrict__ off,
                                                   int32_t *__restrict__ ids)
{
    constexpr int N = 32 * K;
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t wi = warp; wi < cnt; wi += nwarps) {
        const int32_t seg = list[wi];
        const int64_t o = off[seg];
        const int n = (int)(off[seg + 1] - o);
        int v[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int e = k * 32 + lane;
            v[k] = e < n ? ids[o + e] : INT_MAX;
        }
#pragma unroll
        for (int size = 2; size <= N; size <<= 1) {
#pragma unroll
            for (int stride = size >> 1; stride > 0; stride >>= 1) {
                if (stride >= 32) {  // partner in the same lane, register k ^ (stride/32)
                    const int ks = stride / 32;
#pragma unroll
                    for (int k = 0; k < K; ++k) {
                        if (k & ks)
                            continue;
                        const int e = k * 32 + lane;
                        const bool up = (e & size) == 0;
                        const int a = v[k], b = v[k | ks];
                        v[k] = up ? min(a, b) : max(a, b);
                        v[k | ks] = up ? max(a, b) : min(a, b);
                    }
                } else {  // partner in lane ^ stride, same register
#pragma unroll
                    for (int k = 0; k < K; ++k) {
                        const int e = k * 32 + lane;
                        const int other = __shfl_xor_sync(RT_FULL, v[k], stride);
                        const bool up = (e & size) == 0;
                        const bool lower = (lane & stride) == 0;
                        v[k] = (lower == up) ? min(v[k], other) : max(v[k], other);
                    }
                }
            }
        }
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int e = k * 32 + lane;
            if (e < n)
                ids[o + e] = v[k];
        }
    }
}

// ------------------------------------------------------------ CTA sort
constexpr int kBucketBitsMax = 12;  // at most 4096 buckets
constexpr int kBucketCrowded = 32;  // a bucket longer than this sends the segment to LSD

template <int THREADS>
struct CtaSmem {
    static constexpr int W = THREADS / 32;
    uint32_t buf[THREADS * kItems];
    union {
        uint32_t cnt[1 << kBucketBitsMax];  // bucket sort: per-bucket counts, then ends
        struct {
            uint32_t wcnt[W][kBins];
            uint32_t dcount[kBins];
            uint32_t dstart[kBins];
        };
    };
    uint32_t wsum[W];
    uint32_t red_and[W], red_or[W];
    uint32_t crowded;
};

// Ranks the keys held in registers for one LSD pass; on return pos[i] is the
// position of key[i] in the pass's output order (valid where i < rounds and
// the key exists).  Warp w owns keys [w*run, (w+1)*run), taken 32 at a time.
template <int THREADS>
__device__ __forceinline__ void rank_pass(CtaSmem<THREADS> &sm, const uint32_t (&key)[kItems],
                                          int rounds, int run, int n, int shift,
                                          uint32_t (&pos)[kItems])
{
    constexpr int W = THREADS / 32;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned lt = lanemask_lt();
    for (int i = threadIdx.x; i < W * kBins; i += THREADS)
        (&sm.wcnt[0][0])[i] = 0;
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        if (i < rounds) {
            const bool ok = w * run + i * 32 + lane < n;
            const int dg = ok ? (int)((key[i] >> shift) & 0xffu) : kBins;
            const unsigned peers = __match_any_sync(RT_FULL, dg);
            const uint32_t prev = ok ? sm.wcnt[w][dg] : 0u;
            pos[i] = prev + __popc(peers & lt);
            __syncwarp();
            if (ok && lane == __ffs(peers) - 1)
                sm.wcnt[w][dg] = prev + __popc(peers);
            __syncwarp();
        }
    }
    __syncthreads();
    for (int d = threadIdx.x; d < kBins; d += THREADS) {
        uint32_t r = 0;
#pragma unroll 8
        for (int x = 0; x < W; ++x) {
            const uint32_t c = sm.wcnt[x][d];
            sm.wcnt[x][d] = r;
            r += c;
        }
        sm.dcount[d] = r;
    }
    __syncthreads();
    if (threadIdx.x < 32) {  // exclusive scan of the 256 digit totals by one warp
        uint32_t carry = 0;
#pragma unroll
        for (int c = 0; c < kBins; c += 32) {
            const uint32_t v = sm.dcount[c + lane];
            uint32_t inc = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t u = __shfl_up_sync(RT_FULL, inc, o);
                if (lane >= o)
                    inc += u;
            }
            sm.dstart[c + lane] = carry + inc - v;
            carry += __shfl_sync(RT_FULL, inc, 31);
        }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        if (i < rounds && w * run + i * 32 + lane < n) {
            const int dg = (int)((key[i] >> shift) & 0xffu);
            pos[i] += sm.dstart[dg] + sm.wcnt[w][dg];
        }
    }
}

// Sorts one segment of n <= THREADS*kItems keys: src keys (xor flip_in)
// -> dst ids (xor flip_out).
template <int THREADS>
__device__ __forceinline__ void cta_sort_one(CtaSmem<THREADS> &sm, const uint32_t *__restrict__ src,
                                             uint32_t *__restrict__ dst, int n, uint32_t flip_in,
                                             uint32_t flip_out)
{
    constexpr int W = THREADS / 32;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int run = ((n + W * 32 - 1) / (W * 32)) * 32;
    const int rounds = run / 32;
    uint32_t key[kItems], pos[kItems];
    uint32_t a_and = 0xffffffffu, a_or = 0;
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        key[i] = 0;
        const int p = w * run + i * 32 + lane;
        if (i < rounds && p < n) {
            key[i] = src[p] ^ flip_in;
            a_and &= key[i];
            a_or |= key[i];
        }
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        a_and &= __shfl_xor_sync(RT_FULL, a_and, d);
        a_or |= __shfl_xor_sync(RT_FULL, a_or, d);
    }
    if (lane == 0) {
        sm.red_and[w] = a_and;
        sm.red_or[w] = a_or;
    }
    __syncthreads();
    a_and = 0xffffffffu;
    a_or = 0;
    for (int x = 0; x < W; ++x) {
        a_and &= sm.red_and[x];
        a_or |= sm.red_or[x];
    }
    const uint32_t diff = a_and ^ a_or;
    int last = -1;
    for (int shift = 0; shift < 32; shift += 8)
        if ((diff >> shift) & 0xffu)
            last = shift;
    if (last < 0) {  // all keys equal: already sorted
#pragma unroll
        for (int i = 0; i < kItems; ++i) {
            const int p = w * run + i * 32 + lane;
            if (i < rounds && p < n)
                dst[p] = key[i] ^ flip_out;
        }
        __syncthreads();
        return;
    }
    for (int shift = 0; shift <= last; shift += 8) {
        if (((diff >> shift) & 0xffu) == 0)
            continue;
        rank_pass<THREADS>(sm, key, rounds, run, n, shift, pos);
#pragma unroll
        for (int i = 0; i < kItems; ++i)
            if (i < rounds && w * run + i * 32 + lane < n)
                sm.buf[pos[i]] = key[i];
        __syncthreads();
        if (shift == last) {
            for (int p = threadIdx.x; p < n; p += THREADS)
                dst[p] = sm.buf[p] ^ flip_out;
        } else {
#pragma unroll
            for (int i = 0; i < kItems; ++i) {
                const int p = w * run + i * 32 + lane;
                if (i < rounds && p < n)
                    key[i] = sm.buf[p];
            }
        }
        __syncthreads();
    }
}

// Block-wide AND and OR of the keys' bits; every thread gets the result.
template <int THREADS>
__device__ __forceinline__ uint32_t block_diff(CtaSmem<THREADS> &sm, uint32_t a_and, uint32_t a_or)
{
    constexpr int W = THREADS / 32;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        a_and &= __shfl_xor_sync(RT_FULL, a_and, d);
        a_or |= __shfl_xor_sync(RT_FULL, a_or, d);
    }
    if (lane == 0) {
        sm.red_and[w] = a_and;
        sm.red_or[w] = a_or;
    }
    __syncthreads();
    a_and = 0xffffffffu;
    a_or = 0;
    for (int x = 0; x < W; ++x) {
        a_and &= sm.red_and[x];
        a_or |= sm.red_or[x];
    }
    __syncthreads();
    return a_and ^ a_or;
}

// Sorts one segment of n <= THREADS*kItems keys by bucketing on the top B
// bits that differ between its keys (B about log2(n) - 1, at most 12, so a
// bucket holds 2-4 keys on average for spread-out ids), then sorting each
// bucket by insertion.  Buckets are filled with shared-memory atomics (the
// order inside a bucket does not matter: the bucket is sorted next).  If any
// bucket holds more than kBucketCrowded keys the segment is re-sorted by the
// stable LSD radix path instead, so skewed id sets stay correct and cheap.
// Returns false (writing nothing) if a bucket is crowded.
template <int THREADS>
__device__ __forceinline__ bool cta_bucket_sort(CtaSmem<THREADS> &sm, const uint32_t *__restrict__ src,
                                                uint32_t *__restrict__ dst, int n, uint32_t flip_in,
                                                uint32_t flip_out)
{
    uint32_t key[kItems];
    uint32_t a_and = 0xffffffffu, a_or = 0;
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        const int p = i * THREADS + threadIdx.x;
        if (i * THREADS >= n)
            break;
        key[i] = 0;
        if (p < n) {
            key[i] = src[p] ^ flip_in;
            a_and &= key[i];
            a_or |= key[i];
        }
    }
    const uint32_t diff = block_diff<THREADS>(sm, a_and, a_or);
    if (diff == 0) {  // all keys equal
#pragma unroll
        for (int i = 0; i < kItems; ++i) {
            const int p = i * THREADS + threadIdx.x;
            if (i * THREADS >= n)
                break;
            if (p < n)
                dst[p] = key[i] ^ flip_out;
        }
        __syncthreads();
        return true;
    }
    const int hb = 31 - __clz(diff);
    int bits = 32 - __clz((unsigned)(n - 1));  // ceil(log2(n)) for n >= 2
    bits = bits - 1;
    bits = bits < 1 ? 1 : (bits > kBucketBitsMax ? kBucketBitsMax : bits);
    if (bits > hb + 1)
        bits = hb + 1;
    const int shift = hb + 1 - bits;
    const int nb = 1 << bits;
    const uint32_t mask = (uint32_t)nb - 1u;
    for (int b = threadIdx.x; b < nb; b += THREADS)
        sm.cnt[b] = 0;
    if (threadIdx.x == 0)
        sm.crowded = 0;
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        if (i * THREADS >= n)
            break;
        if (i * THREADS + threadIdx.x < n)
            atomicAdd(&sm.cnt[(key[i] >> shift) & mask], 1u);
    }
    __syncthreads();
    {  // exclusive scan of the nb counts: each thread owns a run of them
        constexpr int W = THREADS / 32;
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
        const int per = (nb + THREADS - 1) / THREADS;
        const int lo = threadIdx.x * per;
        uint32_t sum = 0;
        for (int b = lo; b < lo + per && b < nb; ++b)
            sum += sm.cnt[b];
        uint32_t inc = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t u = __shfl_up_sync(RT_FULL, inc, o);
            if (lane >= o)
                inc += u;
        }
        if (lane == 31)
            sm.wsum[w] = inc;
        __syncthreads();
        uint32_t run = inc - sum;
        for (int x = 0; x < w; ++x)
            run += sm.wsum[x];
        for (int b = lo; b < lo + per && b < nb; ++b) {
            const uint32_t c = sm.cnt[b];
            if (c > (uint32_t)kBucketCrowded)
                sm.crowded = 1;
            sm.cnt[b] = run;
            run += c;
        }
        (void)W;
    }
    __syncthreads();
    if (sm.crowded) {
        __syncthreads();
        return false;
    }
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        if (i * THREADS >= n)
            break;
        if (i * THREADS + threadIdx.x < n) {
            const uint32_t pos = atomicAdd(&sm.cnt[(key[i] >> shift) & mask], 1u);
            sm.buf[pos] = key[i];
        }
    }
    __syncthreads();
    // cnt[b] is now the end of bucket b; sort each bucket by insertion
    for (int b = threadIdx.x; b < nb; b += THREADS) {
        const int e = (int)sm.cnt[b];
        const int s0 = b ? (int)sm.cnt[b - 1] : 0;
        for (int i = s0 + 1; i < e; ++i) {
            const uint32_t x = sm.buf[i];
            int j = i - 1;
            while (j >= s0 && sm.buf[j] > x) {
                sm.buf[j + 1] = sm.buf[j];
                --j;
            }
            sm.buf[j + 1] = x;
        }
    }
    __syncthreads();
    for (int p = threadIdx.x; p < n; p += THREADS)
        dst[p] = sm.buf[p] ^ flip_out;
    __syncthreads();
    return true;
}

// One CTA per listed segment (BUCKETS: list of SegDesc; else segment ids).
// Segments with a crowded bucket are appended to `crowded` for k_sort_lsd.
template <int THREADS, bool BUCKETS>
__global__ void __launch_bounds__(THREADS, 1024 / THREADS)
    k_sort_cta(const void *__restrict__ list, int64_t cnt, const int64_t *__restrict__ off,
               const uint32_t *__restrict__ src_base, uint32_t *__restrict__ dst_base,
               uint32_t flip_in, uint32_t flip_out, SegDesc *__restrict__ crowded,
               unsigned long long *__restrict__ n_crowded, int64_t crowded_cap)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    CtaSmem<THREADS> &sm = *reinterpret_cast<CtaSmem<THREADS> *>(smem_raw);
    for (int64_t b = blockIdx.x; b < cnt; b += gridDim.x) {
        int64_t so, dof;
        int n;
        if (BUCKETS) {
            const SegDesc d = static_cast<const SegDesc *>(list)[b];
            so = d.src;
            dof = d.dst;
            n = d.n;
        } else {
            const int32_t seg = static_cast<const int32_t *>(list)[b];
            so = dof = off[seg];
            n = (int)(off[seg + 1] - so);
        }
        if (n > THREADS * kItems)
            continue;  // never listed here; guarded anyway
        if (!cta_bucket_sort<THREADS>(sm, src_base + so, dst_base + dof, n, flip_in, flip_out) &&
            threadIdx.x == 0) {
            const unsigned long long slot = atomicAdd(n_crowded, 1ull);
            if ((int64_t)slot < crowded_cap)
                crowded[slot] = SegDesc{so, dof, n, 0};
        }
    }
}

// Stable LSD radix sort (in shared memory) of the segments whose buckets
// were crowded.  Persistent: the list length is read on the device.
__global__ void __launch_bounds__(1024, 1)
    k_sort_lsd(const SegDesc *__restrict__ list, const unsigned long long *__restrict__ count,
               int64_t cap, const uint32_t *__restrict__ src_base, uint32_t *__restrict__ dst_base,
               uint32_t flip_in, uint32_t flip_out)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    CtaSmem<1024> &sm = *reinterpret_cast<CtaSmem<1024> *>(smem_raw);
    int64_t cnt = (int64_t)*count;
    if (cnt > cap)
        cnt = cap;
    for (int64_t b = blockIdx.x; b < cnt; b += gridDim.x) {
        const SegDesc d = list[b];
        if (d.n > 1024 * kItems)
            continue;
        cta_sort_one<1024>(sm, src_base + d.src, dst_base + d.dst, d.n, flip_in, flip_out);
    }
}

// ------------------------------------------------------------ MSD step
// One CTA per segment longer than kCtaMax: partitions its keys by their top
// b differing bits (2^b buckets of about kCtaMax/2) into the scratch area and
// lists every bucket for the CTA sort (or, if a bucket is still too long,
// for the global LSD fallback).
__global__ void __launch_bounds__(1024)
    k_msd_partition(const int32_t *__restrict__ list, const int64_t *__restrict__ tmp_off,
                    int64_t cnt, const int64_t *__restrict__ off, const uint32_t *__restrict__ ids,
                    uint32_t *__restrict__ scratch, SegDesc *__restrict__ buckets,
                    SegDesc *__restrict__ oversize, int64_t desc_cap,
                    unsigned long long *__restrict__ hdr)
{
    __shared__ uint32_t hist[kBins], cursor[kBins];
    __shared__ uint32_t red_and[32], red_or[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int64_t b = blockIdx.x; b < cnt; b += gridDim.x) {
        const int32_t seg = list[b];
        const int64_t o = off[seg];
        const int64_t n = off[seg + 1] - o;
        const int64_t t = tmp_off[b];
        uint32_t a_and = 0xffffffffu, a_or = 0;
        for (int64_t p = threadIdx.x; p < n; p += 1024) {
            const uint32_t k = ids[o + p] ^ kSign;
            a_and &= k;
            a_or |= k;
        }
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) {
            a_and &= __shfl_xor_sync(RT_FULL, a_and, d);
            a_or |= __shfl_xor_sync(RT_FULL, a_or, d);
        }
        if (lane == 0) {
            red_and[w] = a_and;
            red_or[w] = a_or;
        }
        if (threadIdx.x < kBins)
            hist[threadIdx.x] = 0;
        __syncthreads();
        a_and = 0xffffffffu;
        a_or = 0;
        for (int x = 0; x < 32; ++x) {
            a_and &= red_and[x];
            a_or |= red_or[x];
        }
        const uint32_t diff = a_and ^ a_or;
        if (diff == 0) {  // all equal: nothing to do
            __syncthreads();
            continue;
        }
        const int hb = 31 - __clz(diff);
        int nb_bits = 1;
        while (nb_bits < 8 && (n >> nb_bits) > kCtaMax / 2)
            ++nb_bits;
        if (nb_bits > hb + 1)
            nb_bits = hb + 1;
        const int shift = hb + 1 - nb_bits;
        const uint32_t mask = (1u << nb_bits) - 1u;
        for (int64_t p = threadIdx.x; p < n; p += 1024)
            atomicAdd(&hist[((ids[o + p] ^ kSign) >> shift) & mask], 1u);
        __syncthreads();
        if (threadIdx.x < 32) {
            uint32_t carry = 0;
            for (int c = 0; c < kBins; c += 32) {
                const uint32_t v = hist[c + lane];
                uint32_t inc = v;
#pragma unroll
                for (int q = 1; q < 32; q <<= 1) {
                    const uint32_t u = __shfl_up_sync(RT_FULL, inc, q);
                    if (lane >= q)
                        inc += u;
                }
                cursor[c + lane] = carry + inc - v;
                carry += __shfl_sync(RT_FULL, inc, 31);
            }
        }
        __syncthreads();
        if (threadIdx.x < kBins && hist[threadIdx.x] > 0) {
            const uint32_t d = threadIdx.x;
            SegDesc s;
            s.src = t + cursor[d];
            s.dst = o + cursor[d];
            s.n = (int32_t)hist[d];
            s.pad = 0;
            if (hist[d] <= (uint32_t)kCtaMax) {
                const unsigned long long slot = atomicAdd(hdr + HDR_BUCKETS, 1ull);
                if ((int64_t)slot < desc_cap)
                    buckets[slot] = s;
            } else {
                const unsigned long long slot = atomicAdd(hdr + HDR_OVERSIZE, 1ull);
                if ((int64_t)slot < desc_cap)
                    oversize[slot] = s;
            }
        }
        __syncthreads();
        for (int64_t p = threadIdx.x; p < n; p += 1024) {
            const uint32_t k = ids[o + p] ^ kSign;
            const uint32_t pos = atomicAdd(&cursor[(k >> shift) & mask], 1u);
            scratch[t + pos] = k;
        }
        __syncthreads();
    }
}

// Fallback for buckets longer than kCtaMax (heavily skewed ids): copy the
// bucket to its destination, then LSD radix sort it there through global
// memory, using the bucket's scratch range as the second buffer.
__global__ void __launch_bounds__(256)
    k_sort_global(const SegDesc *__restrict__ list, int64_t cnt, uint32_t *__restrict__ scratch,
                  int32_t *__restrict__ ids)
{
    __shared__ uint32_t hist[kBins], run[kBins];
    __shared__ uint32_t red_and[8], red_or[8];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int64_t b = blockIdx.x; b < cnt; b += gridDim.x) {
        const SegDesc d = list[b];
        uint32_t *x = scratch + d.src;                              // keys (flipped)
        uint32_t *y = reinterpret_cast<uint32_t *>(ids) + d.dst;    // output area
        const int64_t n = d.n;
        uint32_t a_and = 0xffffffffu, a_or = 0;
        for (int64_t p = threadIdx.x; p < n; p += 256) {
            a_and &= x[p];
            a_or |= x[p];
        }
#pragma unroll
        for (int q = 16; q > 0; q >>= 1) {
            a_and &= __shfl_xor_sync(RT_FULL, a_and, q);
            a_or |= __shfl_xor_sync(RT_FULL, a_or, q);
        }
        if (lane == 0) {
            red_and[w] = a_and;
            red_or[w] = a_or;
        }
        __syncthreads();
        a_and = 0xffffffffu;
        a_or = 0;
        for (int q = 0; q < 8; ++q) {
            a_and &= red_and[q];
            a_or |= red_or[q];
        }
        const uint32_t diff = a_and ^ a_or;
        uint32_t *src = x, *dst = y;
        for (int shift = 0; shift < 32; shift += 8) {
            if (((diff >> shift) & 0xffu) == 0)
                continue;
            hist[threadIdx.x] = 0;
            __syncthreads();
            for (int64_t p = threadIdx.x; p < n; p += 256)
                atomicAdd(&hist[(src[p] >> shift) & 0xffu], 1u);
            __syncthreads();
            if (threadIdx.x < 32) {
                uint32_t carry = 0;
                for (int c = 0; c < kBins; c += 32) {
                    const uint32_t v = hist[c + lane];
                    uint32_t inc = v;
#pragma unroll
                    for (int q = 1; q < 32; q <<= 1) {
                        const uint32_t u = __shfl_up_sync(RT_FULL, inc, q);
                        if (lane >= q)
                            inc += u;
                    }
                    run[c + lane] = carry + inc - v;
                    carry += __shfl_sync(RT_FULL, inc, 31);
                }
            }
            __syncthreads();
            // stable scatter: one warp walks the keys in order, 32 at a time
            if (w == 0) {
                const unsigned lt = lanemask_lt();
                for (int64_t p0 = 0; p0 < n; p0 += 32) {
                    const int64_t p = p0 + lane;
                    const bool ok = p < n;
                    const uint32_t k = ok ? src[p] : 0u;
                    const int dg = ok ? (int)((k >> shift) & 0xffu) : kBins;
                    const unsigned peers = __match_any_sync(RT_FULL, dg);
                    const uint32_t base = ok ? run[dg] : 0u;
                    if (ok)
                        dst[base + __popc(peers & lt)] = k;
                    __syncwarp();
                    if (ok && lane == __ffs(peers) - 1)
                        run[dg] = base + __popc(peers);
                    __syncwarp();
                }
            }
            __syncthreads();
            uint32_t *tmp = src;
            src = dst;
            dst = tmp;
        }
        for (int64_t p = threadIdx.x; p < n; p += 256)
            y[p] = src[p] ^ kSign;
        __syncthreads();
    }
}

template <typename K>
rtree_status set_smem(K kern, size_t bytes)
{
    if (bytes > 48 * 1024)
        RT_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    return RTREE_OK;
}

struct Crowded {
    SegDesc *list;
    unsigned long long *count;
    int64_t cap;
};

template <int THREADS, bool BUCKETS>
rtree_status launch_cta(const void *list, int64_t cnt, const int64_t *off, const uint32_t *src,
                        uint32_t *dst, uint32_t flip_in, uint32_t flip_out, const Crowded &cr,
                        cudaStream_t s, const char *name)
{
    if (cnt <= 0)
        return RTREE_OK;
    auto kern = k_sort_cta<THREADS, BUCKETS>;
    const size_t bytes = sizeof(CtaSmem<THREADS>);
    RT_TRY(set_smem(kern, bytes));
    int per_sm = 0;
    RT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, THREADS, bytes));
    int64_t grid = (int64_t)(per_sm > 0 ? per_sm : 1) * sm_count();
    if (grid > cnt)
        grid = cnt;
    KernelTimer kt_(name, s);
    kern<<<(unsigned)grid, THREADS, bytes, s>>>(list, cnt, off, src, dst, flip_in, flip_out,
                                                cr.list, cr.count, cr.cap);
    RT_LAUNCH();
    return RTREE_OK;
}

rtree_status launch_lsd(const Crowded &cr, const uint32_t *src, uint32_t *dst, uint32_t flip_in,
                        uint32_t flip_out, cudaStream_t s)
{
    const size_t bytes = sizeof(CtaSmem<1024>);
    RT_TRY(set_smem(k_sort_lsd, bytes));
    KernelTimer kt_("sort_lsd", s);
    k_sort_lsd<<<(unsigned)sm_count(), 1024, bytes, s>>>(cr.list, cr.count, cr.cap, src, dst, flip_in,
                                                         flip_out);
    RT_LAUNCH();
    return RTREE_OK;
}

template <int K>
rtree_status launch_warp(const int32_t *list, int64_t cnt, const int64_t *off, int32_t *ids,
                         cudaStream_t s)
{
    if (cnt <= 0)
        return RTREE_OK;
    int64_t blocks = (cnt + 7) / 8;
    const int64_t cap = (int64_t)sm_count() * 16;
    if (blocks > cap)
        blocks = cap;
    KernelTimer kt_("sort_warp", s);
    k_sort_warp<K><<<(unsigned)blocks, 256, 0, s>>>(list, cnt, off, ids);
    RT_LAUNCH();
    return RTREE_OK;
}

}  // namespace

rtree_status segmented_sort(int32_t *ids, const int64_t *offsets, int64_t nseg, int64_t total,
                            cudaStream_t s)
{
    if (nseg <= 0 || total <= 1)
        return RTREE_OK;
    if (nseg >= (int64_t)INT32_MAX)
        return fail(RTREE_EOVERFLOW, "too many segments to sort (%lld)", (long long)nseg);
    DevBuf<int32_t> lists(s);
    DevBuf<int64_t> large_tmp(s);
    DevBuf<unsigned long long> hdr(s);
    RT_TRY(lists.alloc((size_t)C_COUNT * nseg, "sort lists"));
    RT_TRY(large_tmp.alloc(nseg, "sort lists"));
    RT_TRY(hdr.alloc(HDR_WORDS, "sort counters"));
    RT_CUDA(cudaMemsetAsync(hdr.p, 0, HDR_WORDS * sizeof(unsigned long long), s));
    const int sms = sm_count();
    {
        int64_t blocks = (nseg + 255) / 256;
        if (blocks > (int64_t)sms * 16)
            blocks = (int64_t)sms * 16;
        KernelTimer kt_("sort_classify", s);
        k_classify<<<(unsigned)blocks, 256, 0, s>>>(offsets, nseg, lists.p, nseg, large_tmp.p, hdr.p);
        RT_LAUNCH();
    }
    unsigned long long h[HDR_WORDS];
    RT_CUDA(cudaMemcpyAsync(h, hdr.p, sizeof(h), cudaMemcpyDeviceToHost, s));
    RT_CUDA(cudaStreamSynchronize(s));
    auto L = [&](int c) { return lists.p + (int64_t)c * nseg; };
    uint32_t *u = reinterpret_cast<uint32_t *>(ids);
    RT_TRY(launch_warp<1>(L(C_W1), (int64_t)h[C_W1], offsets, ids, s));
    RT_TRY(launch_warp<2>(L(C_W2), (int64_t)h[C_W2], offsets, ids, s));
    RT_TRY(launch_warp<4>(L(C_W4), (int64_t)h[C_W4], offsets, ids, s));
    RT_TRY(launch_warp<8>(L(C_W8), (int64_t)h[C_W8], offsets, ids, s));
    const int64_t n_cta = (int64_t)(h[C_T128] + h[C_T256] + h[C_T512] + h[C_T1024]);
    DevBuf<SegDesc> crowded(s);
    DevBuf<unsigned long long> n_crowded(s);
    RT_TRY(crowded.alloc(n_cta > 0 ? n_cta : 1, "sort crowded list"));
    RT_TRY(n_crowded.alloc(2, "sort crowded count"));
    RT_CUDA(cudaMemsetAsync(n_crowded.p, 0, 2 * sizeof(unsigned long long), s));
    const Crowded cr1{crowded.p, n_crowded.p, n_cta};
    RT_TRY((launch_cta<128, false>(L(C_T128), (int64_t)h[C_T128], offsets, u, u, kSign, kSign, cr1, s, "sort_cta")));
    RT_TRY((launch_cta<256, false>(L(C_T256), (int64_t)h[C_T256], offsets, u, u, kSign, kSign, cr1, s, "sort_cta")));
    RT_TRY((launch_cta<512, false>(L(C_T512), (int64_t)h[C_T512], offsets, u, u, kSign, kSign, cr1, s, "sort_cta")));
    RT_TRY((launch_cta<1024, false>(L(C_T1024), (int64_t)h[C_T1024], offsets, u, u, kSign, kSign, cr1, s, "sort_cta")));
    if (n_cta > 0)
        RT_TRY(launch_lsd(cr1, u, u, kSign, kSign, s));
    const int64_t n_large = (int64_t)h[C_LARGE];
    if (n_large == 0)
        return RTREE_OK;

    // Long segments: MSD partition into the scratch area, then sort buckets back.
    const int64_t scratch_n = (int64_t)h[HDR_SCRATCH];
    const int64_t desc_cap = n_large * 2 + 4 * (scratch_n / kCtaMax) + 256;
    DevBuf<uint32_t> scratch(s);
    DevBuf<SegDesc> buckets(s), oversize(s);
    RT_TRY(scratch.alloc(scratch_n, "sort scratch"));
    RT_TRY(buckets.alloc(desc_cap, "sort buckets"));
    RT_TRY(oversize.alloc(desc_cap, "sort buckets"));
    {
        int64_t grid = n_large < (int64_t)sms * 2 ? n_large : (int64_t)sms * 2;
        KernelTimer kt_("sort_msd", s);
        k_msd_partition<<<(unsigned)grid, 1024, 0, s>>>(L(C_LARGE), large_tmp.p, n_large, offsets, u,
                                                        scratch.p, buckets.p, oversize.p, desc_cap,
                                                        hdr.p);
        RT_LAUNCH();
    }
    RT_CUDA(cudaMemcpyAsync(h, hdr.p, sizeof(h), cudaMemcpyDeviceToHost, s));
    RT_CUDA(cudaStreamSynchronize(s));
    const int64_t nb = (int64_t)h[HDR_BUCKETS], no = (int64_t)h[HDR_OVERSIZE];
    if (nb > desc_cap || no > desc_cap)
        return fail(RTREE_EINTERNAL, "sort bucket list overflow (%lld, %lld > %lld)", (long long)nb,
                    (long long)no, (long long)desc_cap);
    DevBuf<SegDesc> crowded2(s);
    RT_TRY(crowded2.alloc(nb > 0 ? nb : 1, "sort crowded list"));
    const Crowded cr2{crowded2.p, n_crowded.p + 1, nb};
    RT_TRY((launch_cta<1024, true>(buckets.p, nb, nullptr, scratch.p, u, 0u, kSign, cr2, s, "sort_bucket")));
    if (nb > 0)
        RT_TRY(launch_lsd(cr2, scratch.p, u, 0u, kSign, s));
    if (no > 0) {
        int64_t grid = no < (int64_t)sms * 4 ? no : (int64_t)sms * 4;
        KernelTimer kt_("sort_global", s);
        k_sort_global<<<(unsigned)grid, 256, 0, s>>>(oversize.p, no, scratch.p, ids);
        RT_LAUNCH();
    }
    return RTREE_OK;
}

}  // namespace rt
