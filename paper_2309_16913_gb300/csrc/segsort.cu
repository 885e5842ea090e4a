// segsort.cu -- build every query's id list, sorted ascending.
//
// The select's traversal emits a query's ids in tree order, partly as single
// leaf hits and partly as whole subtrees (contiguous runs of the tree's id
// array).  This file gathers each query's ids from those sources and sorts
// them, with the work unit sized to the segment:
//   2..256 ids    one warp: gather into shared memory, then a bitonic network
//                 on 1-8 keys per lane in registers (shuffles across lanes,
//                 swaps inside a lane);
//   257..16384    one CTA of 64-512 threads (32 keys each), entirely in
//                 shared memory:
//                 bucket the keys by value within their range (at most 8192
//                 buckets: a few keys each for spread-out ids) with shared
//                 atomics, then each thread sorts whole buckets in registers
//                 with a bitonic network; a crowded bucket sends the segment
//                 to a stable LSD radix sort (8-bit digits);
//   16385..40960  the same with one CTA of 1024 threads, 40 keys each (160 KB
//                 of shared memory; a crowded one goes on to the next path);
//   > 40960       gathered into place, partitioned by its top differing bits
//                 into buckets of about 8K ids (MSD step through a scratch
//                 area), each bucket then sorted like a mid-size segment.
// Each class runs as a persistent grid whose CTAs claim segments from an
// atomic counter, so CTAs that drew long segments do not hold up the rest.
// LSD passes whose digit is equal for all keys are skipped (from the AND and
// OR of the keys).  In each LSD pass a key's rank among equal digits comes
// from walking the keys in order: each warp owns a contiguous run and takes it
// 32 at a time, with __match_any_sync grouping equal digits.  Keys are ids
// with the sign bit flipped, so unsigned order is signed order.
#include <climits>

#include "internal.cuh"

namespace rt {
namespace {

constexpr int kBins = 256;
constexpr int kItems = 16;              // keys per thread of the LSD fallback (1024 threads)
constexpr int kCtaMax = 1024 * kItems;  // 16384: longest segment the LSD fallback takes
constexpr int kItemsMid = 32;           // keys per thread of the CTA sorts up to kCtaMax
constexpr int kItemsBig = 40;           // keys per thread of the CTA sort above kCtaMax
constexpr int kCtaBigMax = 1024 * kItemsBig;
constexpr uint32_t kSign = 0x80000000u;
constexpr int kBucketBitsMax = 13;      // at most 8192 buckets
constexpr int kBucketDensity = 1;       // 2^(ceil(log2 n) - 1) buckets of the key range
constexpr int kBucketCrowded = 32;      // a longer bucket sends the segment to LSD

// Segment classes (index into the class lists).
enum {
    C_W1 = 0, C_W2, C_W4, C_W8,       // warp sorts, 32*K ids
    C_CTA2K, C_CTA4K, C_CTA8K, C_CTA16K,  // CTA sorts of 64..512 threads, kItemsMid ids each
    C_CTA40K,                             // CTA sort of 1024 threads, kItemsBig ids each
    C_LARGE,                          // MSD partition first
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
    if (n <= 2048) return C_CTA2K;
    if (n <= 4096) return C_CTA4K;
    if (n <= 8192) return C_CTA8K;
    if (n <= kCtaMax) return C_CTA16K;
    if (n <= kCtaBigMax) return C_CTA40K;
    return C_LARGE;
}

// End of segment i's leaf hits in S.leaf.
__device__ __forceinline__ int64_t leaf_end(const SortSources &S, int64_t i)
{
    return S.leaf_len ? S.off_leaf[i] + S.leaf_len[i] : S.off_leaf[i + 1];
}

// Segments of length 1 are written directly (class -1 otherwise).
__global__ void k_classify(const int64_t *__restrict__ off, int64_t nseg, int32_t *__restrict__ lists,
                           int64_t stride, int64_t *__restrict__ large_tmp,
                           unsigned long long *__restrict__ hdr, SortSources S,
                           int32_t *__restrict__ out, int64_t out_cap)
{
    const int lane = threadIdx.x & 31;
    const unsigned lt = lanemask_lt();
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t b = warp * 32; b < nseg; b += nwarps * 32) {
        const int64_t i = b + lane;
        int64_t len = i < nseg ? off[i + 1] - off[i] : 0;
        // a segment whose output or sources reach past a buffer's capacity is
        // skipped (the caller sees the totals exceed the capacities)
        if (len > 0 && (off[i + 1] > out_cap ||
                        (S.leaf_cap && leaf_end(S, i) > S.leaf_cap) ||
                        (S.rng && S.rng_cap && S.off_rng[i + 1] > S.rng_cap)))
            len = 0;
        const int cls = class_of(len);
        if (len == 1) {  // a single id: copy it from its source
            int32_t v;
            if (leaf_end(S, i) > S.off_leaf[i])
                v = S.leaf[S.off_leaf[i]];
            else
                v = S.tree_ids[S.rng[S.off_rng[i]].x];
            out[off[i]] = v;
        }
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

// ------------------------------------------------------------- gathering
// One warp copies segment i's ids into sm[0 .. n) (in source order).
__device__ __forceinline__ void warp_gather(int32_t *__restrict__ sm, const SortSources &S,
                                            int64_t i, int lane)
{
    const int64_t l0 = S.off_leaf[i], l1 = leaf_end(S, i);
    for (int64_t e = l0 + lane; e < l1; e += 32)
        sm[e - l0] = S.leaf[e];
    int pos = (int)(l1 - l0);
    if (S.rng) {
        const int64_t r0 = S.off_rng[i], r1 = S.off_rng[i + 1];
        for (int64_t rb = r0; rb < r1; rb += 32) {
            // lanes hold up to 32 ranges; an inclusive scan of their lengths
            // gives each range's place, then the warp copies them in turn
            const int64_t r = rb + lane;
            int2 rg = make_int2(0, 0);
            if (r < r1)
                rg = S.rng[r];
            const int len = rg.y - rg.x;
            int inc = len;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int u = __shfl_up_sync(RT_FULL, inc, o);
                if (lane >= o)
                    inc += u;
            }
            const int start = pos + inc - len;
            const int cnt = (int)(r1 - rb < 32 ? r1 - rb : 32);
            for (int k = 0; k < cnt; ++k) {
                const int lo = __shfl_sync(RT_FULL, rg.x, k);
                const int ln = __shfl_sync(RT_FULL, len, k);
                const int st = __shfl_sync(RT_FULL, start, k);
                for (int e = lane; e < ln; e += 32)
                    sm[st + e] = __ldg(S.tree_ids + lo + e);
            }
            pos += __shfl_sync(RT_FULL, inc, 31);
        }
    }
    __syncwarp();
}

// ----------------------------------------------------------- warp sorts
// Device-resident list lengths: kernels launched without a host round trip
// read how many entries to process.
__device__ __forceinline__ int64_t list_len(const unsigned long long *count, int64_t cap)
{
    const int64_t c = (int64_t)*count;
    return c < cap ? c : cap;
}

// Bitonic sort of up to 32*K signed ids; element e = k*32 + lane (striped).
template <int K>
__global__ void __launch_bounds__(256) k_sort_warp(const int32_t *__restrict__ list,
                                                   const unsigned long long *__restrict__ count,
                                                   int64_t cap, const int64_t *__restrict__ off,
                                                   SortSources S, int32_t *__restrict__ out)
{
    constexpr int N = 32 * K;
    const int64_t cnt = list_len(count, cap);
    __shared__ int32_t stage[8][N];
    const int lane = threadIdx.x & 31;
    int32_t *sm = stage[threadIdx.x >> 5];
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t wi = warp; wi < cnt; wi += nwarps) {
        const int32_t seg = list[wi];
        const int64_t o = off[seg];
        const int n = (int)(off[seg + 1] - o);
        warp_gather(sm, S, seg, lane);
        int v[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int e = k * 32 + lane;
            v[k] = e < n ? sm[e] : INT_MAX;
        }
        __syncwarp();
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
                out[o + e] = v[k];
        }
    }
}

// ------------------------------------------------------------ CTA sort
constexpr int log2_floor(int v) { return v > 1 ? 1 + log2_floor(v / 2) : 0; }

template <int THREADS, int ITEMS = kItems>
struct CtaSmem {
    static constexpr int W = THREADS / 32;
    // at most 2^(ceil(log2 n) - 1) <= n/2 buckets are used (and at most 2^13)
    static constexpr int kCntBits = log2_floor(THREADS * ITEMS / 2) < kBucketBitsMax
                                        ? log2_floor(THREADS * ITEMS / 2) : kBucketBitsMax;
    uint32_t buf[THREADS * ITEMS];
    union {
        uint32_t cnt[1 << kCntBits];  // bucket sort: per-bucket counts, then ends
        struct {                            // LSD ranks
            uint32_t wcnt[W][kBins];
            uint32_t dcount[kBins];
            uint32_t dstart[kBins];
        };
        struct {                            // gathering: one chunk of ranges
            int32_t rlo[THREADS];
            int32_t rstart[THREADS];
            int32_t rlen[THREADS];
        };
    };
    uint32_t wsum[W];
    uint32_t red0[W], red1[W];  // per-warp partial reductions
    uint32_t crowded;
    long long claim;  // the list entry this CTA takes next
};

// Exclusive block scan of one int per thread (uses sm.wsum); returns the
// prefix and writes the block total to *total.
template <int THREADS, int ITEMS>
__device__ __forceinline__ int block_scan_int(CtaSmem<THREADS, ITEMS> &sm, int v, int *total)
{
    constexpr int W = THREADS / 32;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(RT_FULL, inc, o);
        if (lane >= o)
            inc += u;
    }
    if (lane == 31)
        sm.wsum[w] = (uint32_t)inc;
    __syncthreads();
    int before = 0, all = 0;
    for (int x = 0; x < W; ++x) {
        const int s = (int)sm.wsum[x];
        if (x < w)
            before += s;
        all += s;
    }
    *total = all;
    __syncthreads();
    return before + inc - v;
}

// The CTA copies segment i's ids into sm.buf[0 .. n), flipped to keys.  The
// first chunk of range descriptors is requested before the leaf hits are
// copied, so both loads are in flight together.
template <int THREADS, int ITEMS>
__device__ __forceinline__ void cta_gather(CtaSmem<THREADS, ITEMS> &sm, const SortSources &S, int64_t i)
{
    constexpr int W = THREADS / 32;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t l0 = S.off_leaf[i], l1 = leaf_end(S, i);
    int64_t r0 = 0, r1 = 0;
    if (S.rng) {
        r0 = S.off_rng[i];
        r1 = S.off_rng[i + 1];
    }
    int2 rg = make_int2(0, 0);
    if (r0 + threadIdx.x < r1)
        rg = S.rng[r0 + threadIdx.x];
    const int nl = (int)(l1 - l0);
#pragma unroll 4
    for (int e = threadIdx.x; e < nl; e += THREADS)
        sm.buf[e] = (uint32_t)S.leaf[l0 + e] ^ kSign;
    int pos = nl;
    for (int64_t rb = r0; rb < r1; rb += THREADS) {
        if (rb != r0) {
            rg = make_int2(0, 0);
            if (rb + threadIdx.x < r1)
                rg = S.rng[rb + threadIdx.x];
        }
        const int len = rg.y - rg.x;
        int total;
        const int start = block_scan_int<THREADS>(sm, len, &total);
        sm.rlo[threadIdx.x] = rg.x;
        sm.rlen[threadIdx.x] = len;
        sm.rstart[threadIdx.x] = pos + start;
        __syncthreads();
        const int cnt = (int)(r1 - rb < THREADS ? r1 - rb : THREADS);
        for (int k = w; k < cnt; k += W) {  // warp w copies ranges w, w+W, ...
            const int lo = sm.rlo[k], ln = sm.rlen[k], st = sm.rstart[k];
            for (int e = lane; e < ln; e += 32)
                sm.buf[st + e] = (uint32_t)__ldg(S.tree_ids + lo + e) ^ kSign;
        }
        pos += total;
        __syncthreads();
    }
    __syncthreads();
}

// The CTA copies keys src[0 .. n) (xor flip) into sm.buf.
template <int THREADS, int ITEMS>
__device__ __forceinline__ void cta_load(CtaSmem<THREADS, ITEMS> &sm, const uint32_t *__restrict__ src,
                                         int n, uint32_t flip)
{
    for (int p = threadIdx.x; p < n; p += THREADS)
        sm.buf[p] = src[p] ^ flip;
    __syncthreads();
}

// Block-wide AND and OR of the keys' bits; every thread gets AND ^ OR.
template <int THREADS, int ITEMS>
__device__ __forceinline__ uint32_t block_diff(CtaSmem<THREADS, ITEMS> &sm, uint32_t a_and, uint32_t a_or)
{
    constexpr int W = THREADS / 32;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        a_and &= __shfl_xor_sync(RT_FULL, a_and, d);
        a_or |= __shfl_xor_sync(RT_FULL, a_or, d);
    }
    if (lane == 0) {
        sm.red0[w] = a_and;
        sm.red1[w] = a_or;
    }
    __syncthreads();
    a_and = 0xffffffffu;
    a_or = 0;
    for (int x = 0; x < W; ++x) {
        a_and &= sm.red0[x];
        a_or |= sm.red1[x];
    }
    __syncthreads();
    return a_and ^ a_or;
}

// Block-wide minimum and maximum of the keys; every thread gets both.
template <int THREADS, int ITEMS>
__device__ __forceinline__ void block_minmax(CtaSmem<THREADS, ITEMS> &sm, uint32_t &kmin, uint32_t &kmax)
{
    constexpr int W = THREADS / 32;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    kmin = __reduce_min_sync(RT_FULL, kmin);
    kmax = __reduce_max_sync(RT_FULL, kmax);
    if (lane == 0) {
        sm.red0[w] = kmin;
        sm.red1[w] = kmax;
    }
    __syncthreads();
    kmin = 0xffffffffu;
    kmax = 0;
    for (int x = 0; x < W; ++x) {
        kmin = min(kmin, sm.red0[x]);
        kmax = max(kmax, sm.red1[x]);
    }
    __syncthreads();
}

// Sorts buf[s0 .. s0+c), c <= N, in registers: a bitonic network over N
// values padded with the largest key (the first c outputs are then exactly
// the sorted bucket, whatever equal keys it holds).
template <int N>
__device__ __forceinline__ void bucket_network(uint32_t *buf, int s0, int c)
{
    uint32_t v[N];
#pragma unroll
    for (int k = 0; k < N; ++k)
        v[k] = k < c ? buf[s0 + k] : 0xffffffffu;
#pragma unroll
    for (int size = 2; size <= N; size <<= 1) {
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
#pragma unroll
            for (int k = 0; k < N; ++k) {
                const int m = k ^ stride;
                if (m > k) {
                    const bool up = (k & size) == 0;
                    const uint32_t a = v[k], b = v[m];
                    v[k] = up ? min(a, b) : max(a, b);
                    v[m] = up ? max(a, b) : min(a, b);
                }
            }
        }
    }
#pragma unroll
    for (int k = 0; k < N; ++k)
        if (k < c)
            buf[s0 + k] = v[k];
}

// Sorts the n <= THREADS*kItems keys in sm.buf and writes them to dst (xor
// kSign back to ids).  Keys are bucketed by value, (key - min) >> shift with
// B = ceil(log2 n) - 1 bits (at most 13) of the key range, using shared
// atomics, so a bucket of spread-out keys holds one to a few keys (about
// five on average for the 40960-id class); each
// bucket is then sorted in registers.  Measuring from the minimum keeps a
// range that straddles a power of two (e.g. ids around 2^k, or of both
// signs) from crowding into a few buckets.
// Returns false, having written the unsorted ids to dst, if a bucket holds
// more than kBucketCrowded keys (the caller then sorts dst with LSD).
template <int THREADS, int ITEMS>
__device__ __forceinline__ bool cta_bucket_sort(CtaSmem<THREADS, ITEMS> &sm, int32_t *__restrict__ dst,
                                                int n)
{
    uint32_t key[ITEMS];
    uint32_t kmin = 0xffffffffu, kmax = 0;
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        if (i * THREADS >= n)
            break;
        const int p = i * THREADS + threadIdx.x;
        key[i] = 0;
        if (p < n) {
            key[i] = sm.buf[p];
            kmin = min(kmin, key[i]);
            kmax = max(kmax, key[i]);
        }
    }
    block_minmax<THREADS>(sm, kmin, kmax);
    if (kmin == kmax) {  // all keys equal
        for (int p = threadIdx.x; p < n; p += THREADS)
            dst[p] = (int32_t)(sm.buf[p] ^ kSign);
        __syncthreads();
        return true;
    }
    // bucket = (key - kmin) >> shift: B = ceil(log2 n) - 1 bits (at most 13)
    // of the key range, so only buckets inside [kmin, kmax] exist
    const uint32_t span = kmax - kmin;
    const int width = 32 - __clz(span);
    int bits = (32 - __clz((unsigned)(n - 1))) - kBucketDensity;
    constexpr int kMaxBits = CtaSmem<THREADS, ITEMS>::kCntBits;
    bits = bits < 1 ? 1 : (bits > kMaxBits ? kMaxBits : bits);
    if (bits > width)
        bits = width;
    const int shift = width - bits;
    const int nb = (int)(span >> shift) + 1;
    for (int b = threadIdx.x; b < nb; b += THREADS)
        sm.cnt[b] = 0;
    if (threadIdx.x == 0)
        sm.crowded = 0;
    __syncthreads();
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        if (i * THREADS >= n)
            break;
        if (i * THREADS + threadIdx.x < n)
            atomicAdd(&sm.cnt[(key[i] - kmin) >> shift], 1u);
    }
    __syncthreads();
    {  // exclusive scan of the nb counts: each thread owns a run of them
        const int per = (nb + THREADS - 1) / THREADS;
        const int lo = threadIdx.x * per;
        int sum = 0;
        for (int b = lo; b < lo + per && b < nb; ++b)
            sum += (int)sm.cnt[b];
        int total;
        int run = block_scan_int<THREADS>(sm, sum, &total);
        for (int b = lo; b < lo + per && b < nb; ++b) {
            const int c = (int)sm.cnt[b];
            if (c > kBucketCrowded)
                sm.crowded = 1;
            sm.cnt[b] = (uint32_t)run;
            run += c;
        }
    }
    __syncthreads();
    if (sm.crowded) {
        for (int p = threadIdx.x; p < n; p += THREADS)
            dst[p] = (int32_t)(sm.buf[p] ^ kSign);
        __syncthreads();
        return false;
    }
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        if (i * THREADS >= n)
            break;
        if (i * THREADS + threadIdx.x < n) {
            const uint32_t pos = atomicAdd(&sm.cnt[(key[i] - kmin) >> shift], 1u);
            sm.buf[pos] = key[i];
        }
    }
    __syncthreads();
    // cnt[b] is now the end of bucket b.  Each thread sorts whole buckets in
    // registers with a sorting network sized to the warp's largest bucket.
    for (int b0 = threadIdx.x - (threadIdx.x & 31); b0 < nb; b0 += THREADS) {
        const int b = b0 + (threadIdx.x & 31);
        int s0 = 0, c = 0;
        if (b < nb) {
            s0 = b ? (int)sm.cnt[b - 1] : 0;
            c = (int)sm.cnt[b] - s0;
        }
        const int cmax = __reduce_max_sync(RT_FULL, c);
        if (cmax <= 1)
            continue;
        if (cmax <= 4)
            bucket_network<4>(sm.buf, s0, c);
        else if (cmax <= 8)
            bucket_network<8>(sm.buf, s0, c);
        else if (cmax <= 16)
            bucket_network<16>(sm.buf, s0, c);
        else
            bucket_network<32>(sm.buf, s0, c);
    }
    __syncthreads();
    for (int p = threadIdx.x; p < n; p += THREADS)
        dst[p] = (int32_t)(sm.buf[p] ^ kSign);
    __syncthreads();
    return true;
}

__device__ __forceinline__ void push_crowded(SegDesc *list, unsigned long long *count, int64_t cap,
                                             int64_t dst, int n)
{
    const unsigned long long slot = atomicAdd(count, 1ull);
    if ((int64_t)slot < cap)
        list[slot] = SegDesc{dst, dst, n, 0};
}

// The MSD path's segment list, its scratch offsets and the header counters.
struct LongList {
    int32_t *list;
    int64_t *tmp;
    unsigned long long *hdr;
};

// Lists segment seg (n ids) for the MSD path, with a scratch range of its own.
__device__ __forceinline__ void push_large(const LongList &lg, int32_t seg, int64_t n)
{
    const unsigned long long slot = atomicAdd(lg.hdr + C_LARGE, 1ull);
    lg.list[slot] = seg;
    lg.tmp[slot] = (int64_t)atomicAdd(lg.hdr + HDR_SCRATCH, (unsigned long long)n);
}

// One CTA per listed segment.  BUCKETS: the list holds SegDesc entries whose
// keys sit in `scratch`; otherwise segment ids whose ids are gathered from S.
// ITEMS keys per thread; a segment of more than 16384 ids whose buckets are
// crowded goes to the MSD path.  CTAs claim list entries from the counter
// *next (zero at launch), so a CTA that drew short segments takes more.
template <int THREADS, bool BUCKETS, int ITEMS = kItems>
__global__ void __launch_bounds__(THREADS, 1024 / THREADS)
    k_sort_cta(const void *__restrict__ list, const unsigned long long *__restrict__ count,
               int64_t list_cap, const int64_t *__restrict__ off, SortSources S,
               const uint32_t *__restrict__ scratch, int32_t *__restrict__ out,
               SegDesc *__restrict__ crowded, unsigned long long *__restrict__ n_crowded,
               int64_t crowded_cap, LongList lg, unsigned long long *__restrict__ next)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    CtaSmem<THREADS, ITEMS> &sm = *reinterpret_cast<CtaSmem<THREADS, ITEMS> *>(smem_raw);
    const int64_t cnt = list_len(count, list_cap);
    for (;;) {
        if (threadIdx.x == 0)
            sm.claim = (long long)atomicAdd(next, 1ull);
        __syncthreads();
        const int64_t b = sm.claim;
        __syncthreads();  // every thread has read the claim before the next one is written
        if (b >= cnt)
            break;
        int64_t dof;
        int n;
        if (BUCKETS) {
            const SegDesc d = static_cast<const SegDesc *>(list)[b];
            dof = d.dst;
            n = d.n;
            if (n > THREADS * ITEMS)
                continue;
            cta_load<THREADS>(sm, scratch + d.src, n, 0u);
        } else {
            const int32_t seg = static_cast<const int32_t *>(list)[b];
            dof = off[seg];
            n = (int)(off[seg + 1] - dof);
            if (n > THREADS * ITEMS)
                continue;
            cta_gather<THREADS>(sm, S, seg);
        }
        if (!cta_bucket_sort<THREADS>(sm, out + dof, n) && threadIdx.x == 0) {
            if (!BUCKETS && n > kCtaMax)  // longer than the LSD fallback takes: MSD path
                push_large(lg, static_cast<const int32_t *>(list)[b], n);
            else
                push_crowded(crowded, n_crowded, crowded_cap, dof, n);
        }
    }
}

// Ranks the keys held in registers for one LSD pass; on return pos[i] is the
// position of key[i] in the pass's output order.  Warp w owns keys
// [w*run, (w+1)*run), taken 32 at a time.
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
        if (i >= rounds)
            break;
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
        if (i >= rounds)
            break;
        if (w * run + i * 32 + lane < n) {
            const int dg = (int)((key[i] >> shift) & 0xffu);
            pos[i] += sm.dstart[dg] + sm.wcnt[w][dg];
        }
    }
}

// Stable LSD radix sort of n <= 16384 ids in place at ids[0 .. n).
__device__ __forceinline__ void cta_lsd_sort(CtaSmem<1024> &sm, int32_t *__restrict__ ids, int n)
{
    constexpr int THREADS = 1024, W = 32;
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
            key[i] = (uint32_t)ids[p] ^ kSign;
            a_and &= key[i];
            a_or |= key[i];
        }
    }
    const uint32_t diff = block_diff<THREADS>(sm, a_and, a_or);
    int last = -1;
    for (int shift = 0; shift < 32; shift += 8)
        if ((diff >> shift) & 0xffu)
            last = shift;
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
                ids[p] = (int32_t)(sm.buf[p] ^ kSign);
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

// Segments whose buckets were crowded, sorted in place by LSD radix.
// Persistent: the list length is read on the device.
__global__ void __launch_bounds__(1024, 1)
    k_sort_lsd(const SegDesc *__restrict__ list, const unsigned long long *__restrict__ count,
               int64_t cap, int32_t *__restrict__ out)
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
        cta_lsd_sort(sm, out + d.dst, d.n);
    }
}

// ------------------------------------------------------------ MSD step
// Gathers each long segment into its place in `out` (unsorted).
__global__ void __launch_bounds__(1024)
    k_gather_large(const int32_t *__restrict__ list, const unsigned long long *__restrict__ count,
                   int64_t list_cap, const int64_t *__restrict__ tmp_off, int64_t scratch_cap,
                   const int64_t *__restrict__ off, SortSources S, int32_t *__restrict__ out,
                   unsigned long long *__restrict__ next)
{
    const int64_t cnt = list_len(count, list_cap);
    __shared__ int32_t rstart[1024];
    __shared__ int32_t wsum[32];
    __shared__ long long claim;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (;;) {
        if (threadIdx.x == 0)
            claim = (long long)atomicAdd(next, 1ull);
        __syncthreads();
        const int64_t b = claim;
        __syncthreads();
        if (b >= cnt)
            break;
        const int32_t i = list[b];
        int32_t *dst = out + off[i];
        if (tmp_off[b] + (off[i + 1] - off[i]) > scratch_cap)
            continue;  // over the scratch capacity: reported by k_msd_partition
        const int64_t l0 = S.off_leaf[i], l1 = leaf_end(S, i);
        if (S.leaf + l0 != dst)
            for (int64_t e = l0 + threadIdx.x; e < l1; e += 1024)
                dst[e - l0] = S.leaf[e];
        int64_t pos = l1 - l0;
        if (!S.rng)
            continue;
        const int64_t r0 = S.off_rng[i], r1 = S.off_rng[i + 1];
        for (int64_t rb = r0; rb < r1; rb += 1024) {
            const int64_t r = rb + threadIdx.x;
            int2 rg = make_int2(0, 0);
            if (r < r1)
                rg = S.rng[r];
            const int len = rg.y - rg.x;
            int inc = len;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int u = __shfl_up_sync(RT_FULL, inc, o);
                if (lane >= o)
                    inc += u;
            }
            if (lane == 31)
                wsum[w] = inc;
            __syncthreads();
            int before = 0, all = 0;
            for (int x = 0; x < 32; ++x) {
                if (x < w)
                    before += wsum[x];
                all += wsum[x];
            }
            rstart[threadIdx.x] = before + inc - len;
            __syncthreads();
            const int cntr = (int)(r1 - rb < 1024 ? r1 - rb : 1024);
            for (int k = w; k < cntr; k += 32) {
                const int2 g = S.rng[rb + k];
                const int64_t st = pos + rstart[k];
                for (int e = lane; e < g.y - g.x; e += 32)
                    dst[st + e] = __ldg(S.tree_ids + g.x + e);
            }
            pos += all;
            __syncthreads();
        }
    }
}

// One CTA per listed long segment (over 40960 ids, or over 16384 with crowded
// buckets): partitions its keys by their top b differing bits (2^b buckets
// of about kCtaMax/2) into the scratch area and lists every bucket for the
// CTA sort (or, if a bucket is still too long, for the global LSD fallback).
__global__ void __launch_bounds__(1024)
    k_msd_partition(const int32_t *__restrict__ list, const int64_t *__restrict__ tmp_off,
                    const unsigned long long *__restrict__ count, int64_t list_cap,
                    int64_t scratch_cap, const int64_t *__restrict__ off,
                    const uint32_t *__restrict__ ids, uint32_t *__restrict__ scratch,
                    SegDesc *__restrict__ buckets, SegDesc *__restrict__ oversize, int64_t desc_cap,
                    unsigned long long *__restrict__ hdr, int32_t *__restrict__ flags,
                    unsigned long long *__restrict__ next)
{
    const int64_t cnt = list_len(count, list_cap);
    __shared__ uint32_t hist[kBins], cursor[kBins];
    __shared__ uint32_t red_and[32], red_or[32];
    __shared__ long long claim;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (;;) {
        if (threadIdx.x == 0)
            claim = (long long)atomicAdd(next, 1ull);
        __syncthreads();
        const int64_t b = claim;
        __syncthreads();
        if (b >= cnt)
            break;
        const int32_t seg = list[b];
        const int64_t o = off[seg];
        const int64_t n = off[seg + 1] - o;
        const int64_t t = tmp_off[b];
        if (t + n > scratch_cap) {  // cannot happen when the scratch holds all ids
            if (threadIdx.x == 0)
                atomicOr(flags, 1);
            continue;
        }
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
                else
                    atomicOr(flags, 2);
            } else {
                const unsigned long long slot = atomicAdd(hdr + HDR_OVERSIZE, 1ull);
                if ((int64_t)slot < desc_cap)
                    oversize[slot] = s;
                else
                    atomicOr(flags, 2);
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

// Fallback for buckets longer than kCtaMax (heavily skewed ids): LSD radix
// sort through global memory from the bucket's scratch range (keys) to its
// place in the output, ping-ponging between the two.
__global__ void __launch_bounds__(256)
    k_sort_global(const SegDesc *__restrict__ list, const unsigned long long *__restrict__ count,
                  int64_t list_cap, uint32_t *__restrict__ scratch, int32_t *__restrict__ ids)
{
    const int64_t cnt = list_len(count, list_cap);
    __shared__ uint32_t hist[kBins], run[kBins];
    __shared__ uint32_t red_and[8], red_or[8];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int64_t b = blockIdx.x; b < cnt; b += gridDim.x) {
        const SegDesc d = list[b];
        uint32_t *x = scratch + d.src;                            // keys (flipped)
        uint32_t *y = reinterpret_cast<uint32_t *>(ids) + d.dst;  // output area
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

// --------------------------------------------------------------- launches
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

template <int THREADS, bool BUCKETS, int ITEMS = kItems>
rtree_status launch_cta(const void *list, const unsigned long long *count, int64_t list_cap,
                        const int64_t *off, const SortSources &S, const uint32_t *scratch,
                        int32_t *out, const Crowded &cr, unsigned long long *next, cudaStream_t s,
                        const char *name, const LongList &lg = LongList{})
{
    if (list_cap <= 0)
        return RTREE_OK;
    auto kern = k_sort_cta<THREADS, BUCKETS, ITEMS>;
    const size_t bytes = sizeof(CtaSmem<THREADS, ITEMS>);
    RT_TRY(set_smem(kern, bytes));
    int per_sm = 0;
    RT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, THREADS, bytes));
    int64_t grid = (int64_t)(per_sm > 0 ? per_sm : 1) * sm_count();
    if (grid > list_cap)
        grid = list_cap;
    KernelTimer kt_(name, s);
    kern<<<(unsigned)grid, THREADS, bytes, s>>>(list, count, list_cap, off, S, scratch, out, cr.list,
                                                cr.count, cr.cap, lg, next);
    RT_LAUNCH();
    return RTREE_OK;
}

rtree_status launch_lsd(const Crowded &cr, int32_t *out, cudaStream_t s)
{
    if (cr.cap <= 0)
        return RTREE_OK;
    const size_t bytes = sizeof(CtaSmem<1024>);
    RT_TRY(set_smem(k_sort_lsd, bytes));
    KernelTimer kt_("sort_lsd", s);
    k_sort_lsd<<<(unsigned)sm_count(), 1024, bytes, s>>>(cr.list, cr.count, cr.cap, out);
    RT_LAUNCH();
    return RTREE_OK;
}

template <int K>
rtree_status launch_warp(const int32_t *list, const unsigned long long *count, int64_t list_cap,
                         const int64_t *off, const SortSources &S, int32_t *out, cudaStream_t s)
{
    if (list_cap <= 0)
        return RTREE_OK;
    int64_t blocks = (list_cap + 7) / 8;
    const int64_t cap = (int64_t)sm_count() * 16;
    if (blocks > cap)
        blocks = cap;
    KernelTimer kt_("sort_warp", s);
    k_sort_warp<K><<<(unsigned)blocks, 256, 0, s>>>(list, count, list_cap, off, S, out);
    RT_LAUNCH();
    return RTREE_OK;
}

// Helper streams of this host thread on the current device, created on first
// use and kept for the thread's life: the sort's independent class kernels
// run on them beside the call's stream, so that one kernel's tail (its last
// CTAs finishing while the rest of the GPU idles) overlaps the next.
constexpr int kSide = 3;
struct SideStreams {
    int device = -1;
    cudaStream_t st[kSide] = {};
    cudaEvent_t ev[kSide + 1] = {};
};

rtree_status side_streams(SideStreams **out)
{
    constexpr int kMaxDev = 64;
    static thread_local SideStreams t_side[kMaxDev];
    int dev = 0;
    RT_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDev)
        return fail(RTREE_ECUDA, "device %d out of range", dev);
    SideStreams &sd = t_side[dev];
    if (sd.device != dev) {
        for (int i = 0; i < kSide; ++i)
            RT_CUDA(cudaStreamCreateWithFlags(&sd.st[i], cudaStreamNonBlocking));
        for (int i = 0; i <= kSide; ++i)
            RT_CUDA(cudaEventCreateWithFlags(&sd.ev[i], cudaEventDisableTiming));
        sd.device = dev;
    }
    *out = &sd;
    return RTREE_OK;
}

// Work enqueued on the side streams after begin() runs after everything
// enqueued on the main stream before it; the main stream waits for all of it
// when the Fork is joined or destroyed (also on an early error return, so
// that buffers freed in the main stream's order outlive their users).
// Declare it after every buffer the side work uses.
struct Fork {
    SideStreams *sd = nullptr;
    cudaStream_t s = nullptr;
    bool open = false;
    rtree_status begin(cudaStream_t main)
    {
        s = main;
        RT_TRY(side_streams(&sd));
        RT_CUDA(cudaEventRecord(sd->ev[kSide], s));
        for (int i = 0; i < kSide; ++i)
            RT_CUDA(cudaStreamWaitEvent(sd->st[i], sd->ev[kSide], 0));
        open = true;
        return RTREE_OK;
    }
    cudaStream_t side(int i) const { return sd->st[i]; }
    // The main stream waits for side stream i's work enqueued so far.
    rtree_status wait(int i)
    {
        RT_CUDA(cudaEventRecord(sd->ev[i], sd->st[i]));
        RT_CUDA(cudaStreamWaitEvent(s, sd->ev[i], 0));
        return RTREE_OK;
    }
    rtree_status join()
    {
        if (!open)
            return RTREE_OK;
        open = false;
        for (int i = 0; i < kSide; ++i)
            RT_TRY(wait(i));
        return RTREE_OK;
    }
    ~Fork()
    {
        if (open && join() != RTREE_OK)
            cudaGetLastError();
    }
};

}  // namespace

rtree_status segmented_sort_gather(int32_t *out, const int64_t *offsets, int64_t nseg, int64_t total,
                                   const SortSources &S, cudaStream_t s, int32_t *flags, int64_t out_cap)
{
    if (nseg <= 0 || total <= 0)
        return RTREE_OK;
    if (out_cap < 0)
        out_cap = total;
    if (nseg >= (int64_t)INT32_MAX)
        return fail(RTREE_EOVERFLOW, "too many segments to sort (%lld)", (long long)nseg);
    // the whole sort, all classes, as one span (its kernels overlap)
    PhaseTimer span_("sort_all", s);
    // Every list length stays on the device; the launches below are sized
    // by upper bounds and read the actual lengths themselves, so the whole
    // sort is enqueued without a host round trip.
    const int64_t max_large = total / (kCtaMax + 1) + 1 < nseg ? total / (kCtaMax + 1) + 1 : nseg;
    const int64_t scratch_cap = total;
    const int64_t desc_cap = 2 * max_large + 4 * (scratch_cap / kCtaMax) + 256;
    DevBuf<int32_t> lists(s);
    DevBuf<int64_t> large_tmp(s);
    DevBuf<unsigned long long> hdr(s);
    RT_TRY(lists.alloc((size_t)C_COUNT * nseg, "sort lists"));
    RT_TRY(large_tmp.alloc(nseg, "sort lists"));
    // the header, two crowded-list counters, and one claim counter per CTA-sort launch
    constexpr int kClaims = 8;
    RT_TRY(hdr.alloc(HDR_WORDS + 2 + kClaims, "sort counters"));
    RT_CUDA(cudaMemsetAsync(hdr.p, 0, (HDR_WORDS + 2 + kClaims) * sizeof(unsigned long long), s));
    auto claim = [&](int k) { return hdr.p + HDR_WORDS + 2 + k; };
    const int sms = sm_count();
    {
        int64_t blocks = (nseg + 255) / 256;
        if (blocks > (int64_t)sms * 16)
            blocks = (int64_t)sms * 16;
        KernelTimer kt_("sort_classify", s);
        k_classify<<<(unsigned)blocks, 256, 0, s>>>(offsets, nseg, lists.p, nseg, large_tmp.p, hdr.p,
                                                    S, out, out_cap);
        RT_LAUNCH();
    }
    auto L = [&](int c) { return lists.p + (int64_t)c * nseg; };
    auto H = [&](int c) { return hdr.p + c; };
    // a class can hold at most total / (its smallest length) segments
    auto cap_of = [&](int64_t min_len) { return total / min_len < nseg ? total / min_len : nseg; };
    const int64_t cta_cap = cap_of(257);
    DevBuf<SegDesc> crowded(s);
    RT_TRY(crowded.alloc(cta_cap > 0 ? cta_cap : 1, "sort crowded list"));
    unsigned long long *n_crowded = hdr.p + HDR_WORDS;  // two counters after the header
    const Crowded cr1{crowded.p, n_crowded, cta_cap};
    const bool long_path = total > kCtaMax;  // else no segment can be long
    // the long path's buffers (segments over 40960 ids, or crowded over 16384)
    DevBuf<uint32_t> scratch(s);
    DevBuf<SegDesc> buckets(s), oversize(s), crowded2(s);
    if (long_path) {
        RT_TRY(scratch.alloc(scratch_cap, "sort scratch"));
        RT_TRY(buckets.alloc(desc_cap, "sort buckets"));
        RT_TRY(oversize.alloc(desc_cap, "sort buckets"));
        RT_TRY(crowded2.alloc(desc_cap, "sort crowded list"));
    }
    // Three side streams and the call's stream run the classes side by side:
    //   side 2: the 40960-id CTA sort, then the long path (which it feeds);
    //   side 1: the CTA sorts up to 8192 ids;
    //   side 0: the warp sorts;
    //   stream: the CTA sort up to 16384 ids, then (after side 1) the LSD
    //           fallback for crowded segments of all CTA classes up to 16384.
    // The largest kernels are enqueued first so that smaller ones fill the
    // SMs their last CTAs leave idle.
    Fork fk;
    RT_TRY(fk.begin(s));
    constexpr int M = kItemsMid;
    if (long_path) {
        const cudaStream_t s2 = fk.side(2);
        const LongList lg{L(C_LARGE), large_tmp.p, hdr.p};
        RT_TRY((launch_cta<1024, false, kItemsBig>(L(C_CTA40K), H(C_CTA40K), cap_of(kCtaMax + 1), offsets, S,
                                                   nullptr, out, cr1, claim(0), s2, "sort_cta", lg)));
        // Long segments: gather into place, MSD-partition into the scratch
        // area, then sort the buckets back into place.
        const int64_t grid = max_large < (int64_t)sms * 2 ? max_large : (int64_t)sms * 2;
        {
            KernelTimer kt_("sort_gather", s2);
            k_gather_large<<<(unsigned)grid, 1024, 0, s2>>>(L(C_LARGE), H(C_LARGE), max_large, large_tmp.p,
                                                            scratch_cap, offsets, S, out, claim(6));
            RT_LAUNCH();
        }
        {
            KernelTimer kt_("sort_msd", s2);
            k_msd_partition<<<(unsigned)grid, 1024, 0, s2>>>(
                L(C_LARGE), large_tmp.p, H(C_LARGE), max_large, scratch_cap, offsets,
                reinterpret_cast<const uint32_t *>(out), scratch.p, buckets.p, oversize.p, desc_cap,
                hdr.p, flags, claim(7));
            RT_LAUNCH();
        }
        const Crowded cr2{crowded2.p, n_crowded + 1, desc_cap};
        RT_TRY((launch_cta<512, true, kItemsMid>(buckets.p, H(HDR_BUCKETS), desc_cap, nullptr, S, scratch.p, out, cr2, claim(1), s2, "sort_bucket")));
        RT_TRY(launch_lsd(cr2, out, s2));
        {
            int64_t g2 = desc_cap < (int64_t)sms * 4 ? desc_cap : (int64_t)sms * 4;
            KernelTimer kt_("sort_global", s2);
            k_sort_global<<<(unsigned)g2, 256, 0, s2>>>(oversize.p, H(HDR_OVERSIZE), desc_cap, scratch.p,
                                                        out);
            RT_LAUNCH();
        }
    }
    RT_TRY((launch_cta<512, false, M>(L(C_CTA16K), H(C_CTA16K), cap_of(8193), offsets, S, nullptr, out, cr1, claim(2), s, "sort_cta")));
    const cudaStream_t s1 = fk.side(1), s0 = fk.side(0);
    RT_TRY((launch_cta<256, false, M>(L(C_CTA8K), H(C_CTA8K), cap_of(4097), offsets, S, nullptr, out, cr1, claim(3), s1, "sort_cta")));
    RT_TRY((launch_cta<128, false, M>(L(C_CTA4K), H(C_CTA4K), cap_of(2049), offsets, S, nullptr, out, cr1, claim(4), s1, "sort_cta")));
    RT_TRY((launch_cta<64, false, M>(L(C_CTA2K), H(C_CTA2K), cap_of(257), offsets, S, nullptr, out, cr1, claim(5), s1, "sort_cta")));
    RT_TRY(launch_warp<8>(L(C_W8), H(C_W8), cap_of(129), offsets, S, out, s0));
    RT_TRY(launch_warp<4>(L(C_W4), H(C_W4), cap_of(65), offsets, S, out, s0));
    RT_TRY(launch_warp<2>(L(C_W2), H(C_W2), cap_of(33), offsets, S, out, s0));
    RT_TRY(launch_warp<1>(L(C_W1), H(C_W1), cap_of(2), offsets, S, out, s0));
    RT_TRY(fk.wait(1));
    RT_TRY(launch_lsd(cr1, out, s));
    return fk.join();
}

rtree_status segmented_sort(int32_t *ids, const int64_t *offsets, int64_t nseg, int64_t total,
                            cudaStream_t s)
{
    SortSources S{};
    S.leaf = ids;
    S.off_leaf = offsets;
    DevBuf<int32_t> flags(s);
    RT_TRY(flags.alloc(1, "sort flags"));
    RT_CUDA(cudaMemsetAsync(flags.p, 0, sizeof(int32_t), s));
    return segmented_sort_gather(ids, offsets, nseg, total, S, s, flags.p);
}

}  // namespace rt
