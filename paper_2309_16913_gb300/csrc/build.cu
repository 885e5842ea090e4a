// build.cu -- Sort-Tile-Recursive bulk load of the R-tree on the device.
//
// The paper fixes the node (up to F entries (MBR, ptr) plus count and depth,
// Section 2.3) but not how the tree is built.  This file packs it bottom-up
// with STR, every sort a stable device radix sort:
//   level items: the data rectangles, then the nodes of the level below;
//   P = ceil(m/F) nodes, S = ceil(sqrt(P)) slabs of S*F items;
//   order A = sort by centre key xmin+xmax (float32; ties keep item order);
//   slab(item) = rank in A / (S*F);
//   order B = sort by (slab, ymin+ymax, item index)  -- LSD: sort by the y key
//             first, then stably by slab;
//   node k = items B[kF .. kF+F), only the last node of a level may be partial.
// A centre key of NaN (-inf + inf) counts as 0 and -0 as +0.
//
// With sort_children, the items of each packed node are then reordered by
// ascending lx (ties keep their packing position), the node order Section
// 4.2 assumes for its join prunings.  Which items share a node is unchanged.
//
// The nodes are then laid out level by level from the root; a level's nodes
// appear in the order their parents list them, so every node's children are
// contiguous and every subtree owns a contiguous run of leaf entries.  Only
// the last-packed node of a level is partial, so the first child of the node
// stored at position s is s*F (minus the shortfall once the partial node has
// been passed) and no prefix sum is needed.
#include <vector>

#include "internal.cuh"

namespace rt {
namespace {

constexpr int kThreads = 256;

inline unsigned blocks_for(int64_t n, int per_block = kThreads)
{
    int64_t b = (n + per_block - 1) / per_block;
    return (unsigned)(b < 1 ? 1 : (b > 1048576 ? 1048576 : b));
}

// float32 centre key as an order-preserving unsigned integer.
__device__ __forceinline__ uint32_t centre_key(float lo, float hi)
{
    const float k = __fadd_rn(lo, hi);
    uint32_t u = __float_as_uint(k);
    if (k != k || (u << 1) == 0u)
        u = 0u;  // NaN -> +0, -0 -> +0
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__global__ void k_validate(const float4 *__restrict__ r, int64_t n, unsigned long long *bad)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float4 b = r[i];
        const bool nan = b.x != b.x || b.y != b.y || b.z != b.z || b.w != b.w;
        if (nan || b.x > b.z || b.y > b.w)
            atomicMin(bad, (unsigned long long)i);
    }
}

__global__ void k_keys(const float4 *__restrict__ boxes, int64_t m, int axis,
                       uint32_t *__restrict__ keys, uint32_t *__restrict__ vals)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float4 b = boxes[i];
        keys[i] = axis == 0 ? centre_key(b.x, b.z) : centre_key(b.y, b.w);
        vals[i] = (uint32_t)i;
    }
}

__global__ void k_slab_of(const uint32_t *__restrict__ order_x, int64_t m, int64_t cap,
                          uint32_t *__restrict__ slab)
{
    const uint32_t cap32 = (uint32_t)cap;  // m < 2^31, so ranks and cap fit 32 bits
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < m;
         r += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t i = order_x[r];
        if (i < m)
            slab[i] = (uint32_t)r / cap32;
    }
}

__global__ void k_gather_slab(const uint32_t *__restrict__ order_y,
                              const uint32_t *__restrict__ slab, int64_t m,
                              uint32_t *__restrict__ keys)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < m;
         p += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t i = order_y[p];
        keys[p] = i < m ? slab[i] : 0u;
    }
}

// Bounding box of each packed node (exact min/max).  A group of G = min(F,
// 32) lanes takes one node: each lane reduces every G-th item, then the
// group reduces by shuffles (min/max are exact in any order).
__global__ void k_node_boxes(const float4 *__restrict__ items, const uint32_t *__restrict__ pack,
                             int64_t m, int F, int64_t P, float4 *__restrict__ out)
{
    const int G = F < 32 ? F : 32;
    const int lane = threadIdx.x & 31, sub = lane % G;
    const int64_t group = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / G;
    const int64_t groups = ((int64_t)gridDim.x * blockDim.x) / G;
    const int64_t rounds = (P + groups - 1) / groups;  // the same count for every lane
    for (int64_t t = 0; t < rounds; ++t) {
        const int64_t k = group + t * groups;
        float4 acc = empty_box();
        if (k < P) {
            const int64_t lo = k * F, hi = min(m, lo + F);
            for (int64_t r = lo + sub; r < hi; r += G) {
                const uint32_t it = pack[r];
                if (it >= m)
                    continue;
                const float4 b = items[it];
                acc.x = fminf(acc.x, b.x);
                acc.y = fminf(acc.y, b.y);
                acc.z = fmaxf(acc.z, b.z);
                acc.w = fmaxf(acc.w, b.w);
            }
        }
        for (int d = G >> 1; d > 0; d >>= 1) {
            acc.x = fminf(acc.x, __shfl_xor_sync(RT_FULL, acc.x, d));
            acc.y = fminf(acc.y, __shfl_xor_sync(RT_FULL, acc.y, d));
            acc.z = fmaxf(acc.z, __shfl_xor_sync(RT_FULL, acc.z, d));
            acc.w = fmaxf(acc.w, __shfl_xor_sync(RT_FULL, acc.w, d));
        }
        if (k < P && sub == 0)
            out[k] = acc;
    }
}

// One warp per packed node: ranks each item by (lx, packing position) among
// the node's items and rewrites the node's run of pack[] in that order.
__global__ void k_sort_children(const float4 *__restrict__ items, uint32_t *__restrict__ pack,
                                int64_t m, int F, int64_t P)
{
    constexpr int kMaxPer = 4;  // F <= 128
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int per = (F + 31) / 32;
    for (int64_t k = warp; k < P; k += nwarps) {
        const int64_t lo = k * F;
        const int cnt = (int)(m - lo < F ? m - lo : F);
        uint32_t it[kMaxPer];
        float lx[kMaxPer];
#pragma unroll
        for (int t = 0; t < kMaxPer; ++t) {
            const int j = t * 32 + lane;
            it[t] = 0xffffffffu;
            lx[t] = __int_as_float(0x7f800000);  // +inf: never ranks below a real item
            if (t < per && j < cnt) {
                it[t] = pack[lo + j];
                if (it[t] < (uint64_t)m)
                    lx[t] = items[it[t]].x;
            }
        }
        int rank[kMaxPer] = {0, 0, 0, 0};
        for (int t2 = 0; t2 < per; ++t2) {
            for (int src = 0; src < 32; ++src) {
                const float v = __shfl_sync(RT_FULL, lx[t2], src);
                const int jv = t2 * 32 + src;
                if (jv >= cnt)
                    break;  // uniform: jv depends only on the loop counters
#pragma unroll
                for (int t = 0; t < kMaxPer; ++t) {
                    const int j = t * 32 + lane;
                    rank[t] += (v < lx[t]) || (v == lx[t] && jv < j);
                }
            }
        }
        __syncwarp();
#pragma unroll
        for (int t = 0; t < kMaxPer; ++t) {
            const int j = t * 32 + lane;
            if (t < per && j < cnt && rank[t] < cnt)
                pack[lo + rank[t]] = it[t];
        }
        __syncwarp();
    }
}

// ---- small levels: one CTA builds every level of at most kSmallLevel items
// (the upper levels of a big tree, or all of a small one), instead of a
// dozen launches per level.  Each level is sorted twice in shared memory by
// a bitonic network over 64-bit composite keys that end in the item index,
// which gives exactly the stable orders of the radix path:
//   (x centre key, item)  -> slab = rank / (S*F),
//   (slab, y centre key, item) -> the packing order.
constexpr int kSmallLevel = 4096;  // item indices fit 12 bits

struct SmallLevels {
    int count;                      // levels to build, bottom up
    int sort_children;
    int64_t m[RT_MAX_LEVELS];       // items of each level
    uint32_t *pack[RT_MAX_LEVELS];  // packing order of each level
    float4 *box[RT_MAX_LEVELS];     // node boxes of each level (items of the next)
};

__device__ __forceinline__ void block_bitonic_u64(unsigned long long *key, int M)
{
    for (int size = 2; size <= M; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = threadIdx.x; i < (M >> 1); i += blockDim.x) {
                const int lo = 2 * stride * (i / stride) + (i % stride), hi = lo + stride;
                const bool up = (lo & size) == 0;
                const unsigned long long a = key[lo], b = key[hi];
                if ((a > b) == up) {
                    key[lo] = b;
                    key[hi] = a;
                }
            }
            __syncthreads();
        }
    }
}

__global__ void __launch_bounds__(1024) k_build_small(const float4 *__restrict__ items0, int F,
                                                       SmallLevels L)
{
    __shared__ unsigned long long key[kSmallLevel];
    __shared__ uint32_t aux[kSmallLevel];  // slab of each item; then a node's reordered items
    for (int l = 0; l < L.count; ++l) {
        const float4 *it = l == 0 ? items0 : L.box[l - 1];
        const int m = (int)L.m[l];
        const int P = (m + F - 1) / F;
        int S = (int)sqrtf((float)P);
        while (S * S < P)
            ++S;
        while (S > 1 && (S - 1) * (S - 1) >= P)
            --S;
        const int cap = S * F;
        int M = 1;
        while (M < m)
            M <<= 1;
        for (int i = threadIdx.x; i < M; i += blockDim.x)
            key[i] = i < m ? ((unsigned long long)centre_key(it[i].x, it[i].z) << 32) | (unsigned)i : ~0ull;
        __syncthreads();
        block_bitonic_u64(key, M);
        for (int r = threadIdx.x; r < m; r += blockDim.x)
            aux[key[r] & 0xfffu] = (uint32_t)(r / cap);
        __syncthreads();
        for (int i = threadIdx.x; i < M; i += blockDim.x)
            key[i] = i < m ? ((unsigned long long)aux[i] << 44) |
                                 ((unsigned long long)centre_key(it[i].y, it[i].w) << 12) | (unsigned)i
                           : ~0ull;
        __syncthreads();
        block_bitonic_u64(key, M);
        uint32_t *pack = L.pack[l];
        if (L.sort_children) {  // each node's items by ascending lx, ties in packing order
            for (int r = threadIdx.x; r < m; r += blockDim.x) {
                const int lo = r / F * F, hi = min(m, lo + F);
                const uint32_t item = (uint32_t)(key[r] & 0xfffu);
                const float x = it[item].x;
                int rank = 0;
                for (int j = lo; j < hi; ++j) {
                    const float v = it[key[j] & 0xfffu].x;
                    rank += (v < x) || (v == x && j < r);
                }
                aux[lo + rank] = item;
            }
        } else {
            for (int r = threadIdx.x; r < m; r += blockDim.x)
                aux[r] = (uint32_t)(key[r] & 0xfffu);
        }
        __syncthreads();
        for (int r = threadIdx.x; r < m; r += blockDim.x)
            pack[r] = aux[r];
        for (int k = threadIdx.x; k < P; k += blockDim.x) {
            float4 acc = empty_box();
            for (int r = k * F; r < min(m, k * F + F); ++r) {
                const float4 b = it[aux[r]];
                acc.x = fminf(acc.x, b.x);
                acc.y = fminf(acc.y, b.y);
                acc.z = fmaxf(acc.z, b.z);
                acc.w = fmaxf(acc.w, b.w);
            }
            L.box[l][k] = acc;
        }
        __syncthreads();  // the next level reads these boxes
    }
}

__global__ void k_find_partial(const uint32_t *__restrict__ order, int64_t P,
                               int64_t *__restrict__ pos)
{
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < P;
         s += (int64_t)gridDim.x * blockDim.x)
        if (order[s] == (uint32_t)(P - 1))
            *pos = s;
}

// Writes the P nodes of one level (thread per slot).  order[s] is the packed
// node stored at position s; pack maps packing positions to items.
__global__ void k_layout(int F, int layout, int64_t P, int64_t m,
                         const uint32_t *__restrict__ order, const uint32_t *__restrict__ pack,
                         const int64_t *__restrict__ partial_pos,
                         const float4 *__restrict__ item_boxes,
                         const float4 *__restrict__ node_boxes, int64_t g_base,
                         int64_t child_base, float *__restrict__ mbr, int4 *__restrict__ meta,
                         float4 *__restrict__ nbox, uint32_t *__restrict__ order_below,
                         const int32_t *__restrict__ ids_in, int32_t *__restrict__ ids_out)
{
    const int64_t last_cnt = m - (P - 1) * F;
    const int64_t pp = *partial_pos;
    const int logF = __ffs(F) - 1;  // F is a power of two
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < P * F;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = idx >> logF;
        const int j = (int)(idx & (F - 1));
        const int64_t o = order[s];
        const int64_t cnt = (o == P - 1) ? last_cnt : F;
        const int64_t first = s * F - (s > pp ? (F - last_cnt) : 0);
        const int64_t g = g_base + s;
        float4 b;
        const uint32_t item = (o < P && j < cnt) ? pack[o * F + j] : 0xffffffffu;
        if (item < (uint64_t)m && first + j < m) {
            b = item_boxes[item];
            if (child_base >= 0)
                order_below[first + j] = item;
            else
                ids_out[first + j] = ids_in ? ids_in[item] : (int32_t)item;
        } else {
            b = empty_box();
        }
        if (layout == RTREE_LAYOUT_AOS) {
            reinterpret_cast<float4 *>(mbr)[g * F + j] = b;
        } else if (layout == RTREE_LAYOUT_LOHI) {
            float2 *p = reinterpret_cast<float2 *>(mbr + g * 4 * F);
            p[j] = make_float2(b.x, b.y);
            p[F + j] = make_float2(b.z, b.w);
        } else {
            float *p = mbr + g * 4 * F + j;
            p[0] = b.x;
            p[F] = b.y;
            p[2 * F] = b.z;
            p[3 * F] = b.w;
        }
        if (j == 0) {
            meta[g] = make_int4((int)(child_base >= 0 ? child_base + first : first), (int)cnt, 0, 0);
            nbox[g] = o < P ? node_boxes[o] : empty_box();
        }
    }
}

// part = {position of a short leaf (-1: none), its count, short leaves}:
// every leaf whose count is not F records itself (part starts {-1, 0, 0}).
__global__ void k_leaf_part(const int4 *__restrict__ leaf_meta, int64_t P, int F,
                            unsigned long long *__restrict__ part)
{
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < P;
         s += (int64_t)gridDim.x * blockDim.x) {
        const int c = leaf_meta[s].y;
        if (c != F) {
            part[0] = (unsigned long long)s;
            part[1] = (unsigned long long)c;
            atomicAdd(part + 2, 1ull);
        }
    }
}

__global__ void k_ranges_leaf(int4 *__restrict__ meta, int64_t g_base, int64_t P)
{
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < P;
         s += (int64_t)gridDim.x * blockDim.x) {
        int4 m = meta[g_base + s];
        m.z = m.x;
        m.w = m.x + m.y;
        meta[g_base + s] = m;
    }
}

__global__ void k_ranges_up(int4 *__restrict__ meta, int64_t g_base, int64_t P)
{
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < P;
         s += (int64_t)gridDim.x * blockDim.x) {
        int4 m = meta[g_base + s];
        m.z = meta[m.x].z;
        m.w = meta[m.x + m.y - 1].w;
        meta[g_base + s] = m;
    }
}

int64_t ceil_sqrt(int64_t p)
{
    int64_t s = 1;
    while (s * s < p)
        ++s;
    return s;
}

int bits_for(uint64_t v)  // bits needed to hold values 0..v
{
    int b = 0;
    while (v) {
        ++b;
        v >>= 1;
    }
    return b;
}

// Allocates the leaf record (TreeDev::leaf_part) and fills it from the leaf
// level's metadata, on stream s.
rtree_status leaf_part_into(const int4 *leaf_meta, int64_t P, int F, DevBuf<int64_t> &part, cudaStream_t s)
{
    RT_TRY(part.alloc(3, "leaf record"));
    RT_CUDA(cudaMemsetAsync(part.p, 0xff, sizeof(int64_t), s));
    RT_CUDA(cudaMemsetAsync(part.p + 1, 0, 2 * sizeof(int64_t), s));
    KernelTimer kt_("leaf_part", s);
    k_leaf_part<<<blocks_for(P), kThreads, 0, s>>>(leaf_meta, P, F,
                                                   reinterpret_cast<unsigned long long *>(part.p));
    RT_LAUNCH();
    return RTREE_OK;
}

}  // namespace

rtree_status build_tree(const float4 *rects, const int32_t *ids, int64_t n, int F, int layout,
                        bool sort_children, cudaStream_t s, rtree *t)
{
    t->fanout = F;
    t->layout = layout;
    t->sorted = sort_children ? 1 : 0;
    t->n = n;
    t->levels = 0;
    t->nodes = 0;
    t->bytes = 0;
    const float inf = __builtin_huge_valf();
    t->root_mbr[0] = inf;
    t->root_mbr[1] = inf;
    t->root_mbr[2] = -inf;
    t->root_mbr[3] = -inf;
    if (n == 0)
        return RTREE_OK;

    // NaN and inverted rectangles are looked for first, and the outcome is
    // read at once through a mailbox (no copy-engine queue to wait behind):
    // it is the one host read of the build, so that the rest of the packing
    // runs in the order of `s` after the call has returned.
    {
        DevBuf<unsigned long long> bad(s);
        RT_TRY(bad.alloc(1, "validation flag"));
        RT_CUDA(cudaMemsetAsync(bad.p, 0xff, sizeof(unsigned long long), s));
        {
            KernelTimer kt_("validate", s);
            k_validate<<<blocks_for(n), kThreads, 0, s>>>(rects, n, bad.p);
            RT_LAUNCH();
        }
        MailboxRef mb;
        RT_TRY(mailbox_get(&mb.m));
        PostList pl{};
        pl.src[0] = bad.p;
        pl.words[0] = 2;
        pl.at[0] = 0;
        pl.n = 1;
        RT_TRY(mailbox_post(mb.m, pl, s));
        RT_TRY(mailbox_wait(mb.m));
        const volatile uint32_t *w = mb.m.h;
        const unsigned long long h = (unsigned long long)w[0] | ((unsigned long long)w[1] << 32);
        if (h != ~0ull)
            return fail(RTREE_EINVAL,
                        "rectangle %llu has a NaN coordinate or xmin > xmax or ymin > ymax", h);
    }

    // ---- bottom-up packing
    std::vector<int64_t> m_of;  // items per build level
    std::vector<int64_t> p_of;  // nodes per build level
    std::vector<DevBuf<uint32_t> *> packs;
    std::vector<DevBuf<float4> *> boxes;  // node boxes per build level
    struct Cleanup {
        std::vector<DevBuf<uint32_t> *> &a;
        std::vector<DevBuf<float4> *> &b;
        ~Cleanup()
        {
            for (auto *x : a)
                delete x;
            for (auto *x : b)
                delete x;
        }
    } cleanup{packs, boxes};

    {
        DevBuf<uint32_t> k0(s), v0(s), k1(s), v1(s), slab(s);
        RT_TRY(k0.alloc(n, "build keys"));
        RT_TRY(v0.alloc(n, "build values"));
        RT_TRY(k1.alloc(n, "build keys"));
        RT_TRY(v1.alloc(n, "build values"));
        RT_TRY(slab.alloc(n, "build slabs"));
        const float4 *cur = rects;
        int64_t m = n;
        for (;;) {
            if ((int)m_of.size() >= RT_MAX_LEVELS)
                return fail(RTREE_EOVERFLOW, "tree would exceed %d levels", RT_MAX_LEVELS);
            if (m <= kSmallLevel) {  // this level and all above it in one CTA
                SmallLevels L{};
                L.sort_children = sort_children ? 1 : 0;
                for (int64_t mm = m;;) {
                    if ((int)m_of.size() >= RT_MAX_LEVELS)
                        return fail(RTREE_EOVERFLOW, "tree would exceed %d levels", RT_MAX_LEVELS);
                    const int64_t P = (mm + F - 1) / F;
                    auto *pk = new DevBuf<uint32_t>(s);
                    packs.push_back(pk);
                    RT_TRY(pk->alloc(mm, "build packing order"));
                    auto *bx = new DevBuf<float4>(s);
                    boxes.push_back(bx);
                    RT_TRY(bx->alloc(P, "node boxes"));
                    L.m[L.count] = mm;
                    L.pack[L.count] = pk->p;
                    L.box[L.count] = bx->p;
                    ++L.count;
                    m_of.push_back(mm);
                    p_of.push_back(P);
                    if (P == 1)
                        break;
                    mm = P;
                }
                KernelTimer kt_("build_small", s);
                k_build_small<<<1, 1024, 0, s>>>(cur, F, L);
                RT_LAUNCH();
                break;
            }
            const int64_t P = (m + F - 1) / F;
            const int64_t S = ceil_sqrt(P);
            const int64_t cap = S * F;
            const int64_t nslab = (m + cap - 1) / cap;
            auto *pack = new DevBuf<uint32_t>(s);
            packs.push_back(pack);
            RT_TRY(pack->alloc(m, "build packing order"));
            if (nslab > 1) {
                {
                    KernelTimer kt_("keys", s);
                    k_keys<<<blocks_for(m), kThreads, 0, s>>>(cur, m, 0, k0.p, v0.p);
                    RT_LAUNCH();
                }
                RT_TRY(radix_sort_pairs(k0.p, v0.p, k1.p, v1.p, m, 0, 32, s));
                {
                    KernelTimer kt_("slab_of", s);
                    k_slab_of<<<blocks_for(m), kThreads, 0, s>>>(v1.p, m, cap, slab.p);
                    RT_LAUNCH();
                }
                {
                    KernelTimer kt_("keys", s);
                    k_keys<<<blocks_for(m), kThreads, 0, s>>>(cur, m, 1, k0.p, v0.p);
                    RT_LAUNCH();
                }
                RT_TRY(radix_sort_pairs(k0.p, v0.p, k1.p, v1.p, m, 0, 32, s));
                {
                    KernelTimer kt_("gather_slab", s);
                    k_gather_slab<<<blocks_for(m), kThreads, 0, s>>>(v1.p, slab.p, m, k0.p);
                    RT_LAUNCH();
                }
                RT_TRY(radix_sort_pairs(k0.p, v1.p, k1.p, pack->p, m, 0,
                                        bits_for((uint64_t)(nslab - 1)), s));
            } else {
                {
                    KernelTimer kt_("keys", s);
                    k_keys<<<blocks_for(m), kThreads, 0, s>>>(cur, m, 1, k0.p, v0.p);
                    RT_LAUNCH();
                }
                RT_TRY(radix_sort_pairs(k0.p, v0.p, k1.p, pack->p, m, 0, 32, s));
            }
            if (sort_children && F > 1) {
                KernelTimer kt_("sort_children", s);
                k_sort_children<<<blocks_for(P * 32), kThreads, 0, s>>>(cur, pack->p, m, F, P);
                RT_LAUNCH();
            }
            auto *nb = new DevBuf<float4>(s);
            boxes.push_back(nb);
            RT_TRY(nb->alloc(P, "node boxes"));
            {
                KernelTimer kt_("node_boxes", s);
                k_node_boxes<<<blocks_for(P * (F < 32 ? F : 32)), kThreads, 0, s>>>(cur, pack->p, m, F, P, nb->p);
                RT_LAUNCH();
            }
            m_of.push_back(m);
            p_of.push_back(P);
            cur = nb->p;
            m = P;
            if (P == 1)
                break;
        }
    }

    // ---- level sizes, root level first
    const int H = (int)p_of.size();
    t->levels = H;
    int64_t nodes = 0;
    for (int e = 0; e < H; ++e) {
        t->level_nodes[e] = p_of[H - 1 - e];
        t->level_base[e] = nodes;
        nodes += t->level_nodes[e];
    }
    t->nodes = nodes;
    if (nodes >= (int64_t)INT32_MAX)
        return fail(RTREE_EOVERFLOW, "tree has %lld nodes; at most 2^31-1 supported", (long long)nodes);

    DevBuf<float> mbr(s);
    DevBuf<int4> meta(s);
    DevBuf<float4> nbox(s);
    DevBuf<int32_t> ids_out(s);
    DevBuf<int64_t> part(s);  // the leaf record (TreeDev::leaf_part)
    RT_TRY(mbr.alloc((size_t)nodes * F * 4, "node entries"));
    RT_TRY(meta.alloc(nodes, "node metadata"));
    RT_TRY(nbox.alloc(nodes, "node boxes"));
    RT_TRY(ids_out.alloc(n, "entry ids"));

    // ---- top-down layout
    {
        DevBuf<uint32_t> order(s), below(s);
        DevBuf<int64_t> pos(s);
        RT_TRY(order.alloc(1, "layout order"));
        RT_TRY(pos.alloc(1, "layout partial position"));
        RT_CUDA(cudaMemsetAsync(order.p, 0, sizeof(uint32_t), s));
        for (int L = H - 1; L >= 0; --L) {
            const int e = H - 1 - L;
            const int64_t P = p_of[L], m = m_of[L];
            {
                KernelTimer kt_("find_partial", s);
                RT_CUDA(cudaMemcpyAsync(pos.p, &P, sizeof(int64_t), cudaMemcpyHostToDevice, s));
                k_find_partial<<<blocks_for(P), kThreads, 0, s>>>(order.p, P, pos.p);
                RT_LAUNCH();
            }
            if (L > 0)
                RT_TRY(below.alloc(m, "layout order"));
            const float4 *item_boxes = L > 0 ? boxes[L - 1]->p : rects;
            const int64_t child_base = L > 0 ? t->level_base[e + 1] : -1;
            {
                KernelTimer kt_("layout", s);
                k_layout<<<blocks_for(P * F), kThreads, 0, s>>>(
                    F, layout, P, m, order.p, packs[L]->p, pos.p, item_boxes, boxes[L]->p,
                    t->level_base[e], child_base, mbr.p, meta.p, nbox.p, L > 0 ? below.p : nullptr,
                    ids, ids_out.p);
                RT_LAUNCH();
            }
            if (L > 0) {
                std::swap(order.p, below.p);
                below.reset();
            }
        }
        for (int e = H - 1; e >= 0; --e) {
            const int64_t P = t->level_nodes[e];
            KernelTimer kt_("ranges", s);
            if (e == H - 1)
                k_ranges_leaf<<<blocks_for(P), kThreads, 0, s>>>(meta.p, t->level_base[e], P);
            else
                k_ranges_up<<<blocks_for(P), kThreads, 0, s>>>(meta.p, t->level_base[e], P);
            RT_LAUNCH();
        }
        // the leaf record is filled before the root box is posted: the post's
        // event is what calls on other streams wait for
        RT_TRY(leaf_part_into(meta.p + t->level_base[H - 1], t->level_nodes[H - 1], F, part, s));
        // the root box goes to a mailbox of the tree, read when first asked
        // for (tree_root_box): the call does not wait for the packing
        Mailbox *mb = new Mailbox();
        rtree_status st = mailbox_get(mb);
        if (st != RTREE_OK) {
            delete mb;
            return st;
        }
        PostList pl{};
        pl.src[0] = boxes[H - 1]->p;
        pl.words[0] = 4;
        pl.at[0] = 0;
        pl.n = 1;
        st = mailbox_post(*mb, pl, s);
        if (st != RTREE_OK) {
            cudaEventSynchronize(mb->ev);
            mailbox_put(mb);
            delete mb;
            return st;
        }
        t->root_mb = mb;
        t->root_ready = false;
    }
    t->mbr = mbr.release();
    t->meta = meta.release();
    t->nbox = nbox.release();
    t->ids = ids_out.release();
    t->leaf_part = part.release();
    t->bytes = (int64_t)nodes * F * 16 + nodes * 32 + n * 4;
    return RTREE_OK;
}

rtree_status compute_leaf_part(rtree *t, cudaStream_t s)
{
    if (t->levels == 0)
        return RTREE_OK;
    DevBuf<int64_t> part(s);
    RT_TRY(leaf_part_into(t->meta + t->level_base[t->levels - 1], t->level_nodes[t->levels - 1], t->fanout,
                          part, s));
    t->leaf_part = part.release();
    return RTREE_OK;
}

}  // namespace rt
