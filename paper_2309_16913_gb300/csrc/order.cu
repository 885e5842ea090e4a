// order.cu -- query ordering for locality (an addition; the paper has none).
//
// A batch of queries in arbitrary order sends neighbouring warps to
// unrelated parts of the tree.  Taking the queries in the order of their
// centres along a Hilbert curve makes warps that run at the same time (and
// consecutive work items of one warp) visit nearby nodes, so upper and
// middle levels are re-read from L2 rather than HBM.  This extends the
// latency-hiding aim of the paper's prefetching (O2, Section 3) to the
// memory hierarchy of the GPU.  Only the traversal order changes: every
// query's results are still written at its own place, so the output is
// identical.
//
// Key: the query centre, scaled into the tree's bounding box and quantized
// to a 2^16 x 2^16 grid, mapped to its distance along the Hilbert curve of
// that grid (the iterative quadrant-rotation construction: at each scale
// the quadrant contributes s*s*((3*rx)^ry), then the coordinates are
// reflected/swapped into the quadrant's frame).  The order is the stable
// radix sort of (key, query index).
#include "internal.cuh"

namespace rt {
namespace {

constexpr int kGridBits = 16;

__device__ __forceinline__ uint32_t hilbert_distance(uint32_t x, uint32_t y)
{
    const uint32_t n = 1u << kGridBits;
    uint32_t d = 0;
    for (uint32_t s = n >> 1; s > 0; s >>= 1) {
        const uint32_t rx = (x & s) ? 1u : 0u;
        const uint32_t ry = (y & s) ? 1u : 0u;
        d += s * s * ((3u * rx) ^ ry);
        if (ry == 0) {  // rotate into the quadrant's frame
            if (rx == 1) {
                x = n - 1 - x;
                y = n - 1 - y;
            }
            const uint32_t t = x;
            x = y;
            y = t;
        }
    }
    return d;
}

// Grid cell of coordinate c in [lo, lo + w): 0 for NaN or a degenerate box.
__device__ __forceinline__ uint32_t cell_of(float c, float lo, float w)
{
    const float u = (c - lo) / w;
    if (!(u > 0.f))  // NaN, negative or zero
        return 0u;
    if (!(u < 1.f))
        return (1u << kGridBits) - 1u;
    const uint32_t v = (uint32_t)(u * (float)(1u << kGridBits));
    return v < (1u << kGridBits) ? v : (1u << kGridBits) - 1u;
}

__global__ void k_hilbert_keys(const float4 *__restrict__ q, int64_t Q, const float4 *__restrict__ root,
                               uint32_t *__restrict__ keys, uint32_t *__restrict__ idx)
{
    const float4 box = *root;
    const float wx = box.z - box.x, wy = box.w - box.y;
    const bool okx = wx > 0.f && wx < __int_as_float(0x7f800000);
    const bool oky = wy > 0.f && wy < __int_as_float(0x7f800000);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < Q;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float4 b = q[i];
        const float cx = 0.5f * b.x + 0.5f * b.z, cy = 0.5f * b.y + 0.5f * b.w;
        const uint32_t x = okx ? cell_of(cx, box.x, wx) : 0u;
        const uint32_t y = oky ? cell_of(cy, box.y, wy) : 0u;
        keys[i] = hilbert_distance(x, y);
        idx[i] = (uint32_t)i;
    }
}

}  // namespace

rtree_status hilbert_order(const rtree *t, const float4 *queries, int64_t Q, uint32_t *order,
                           cudaStream_t s)
{
    if (Q <= 0)
        return RTREE_OK;
    DevBuf<uint32_t> k0(s), v0(s), k1(s);
    RT_TRY(k0.alloc(Q, "query order keys"));
    RT_TRY(v0.alloc(Q, "query order"));
    RT_TRY(k1.alloc(Q, "query order keys"));
    {  // the tree's bounding box is read on the device: the root's node box
        KernelTimer kt_("hilbert_keys", s);
        int64_t b = (Q + 255) / 256;
        k_hilbert_keys<<<(unsigned)(b > 65536 ? 65536 : b), 256, 0, s>>>(queries, Q, t->nbox, k0.p, v0.p);
        RT_LAUNCH();
    }
    return radix_sort_pairs(k0.p, v0.p, k1.p, order, Q, 0, 32, s);
}

}  // namespace rt
