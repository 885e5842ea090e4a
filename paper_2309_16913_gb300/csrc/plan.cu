// plan.cu -- batched range select captured in CUDA graphs.
//
// A plan owns every buffer a sorted select needs, sized by capacities given
// up front (queries per batch, ids per batch), and records the whole device
// pipeline -- count pass, three scans, descriptor pass, segmented sort and
// the copy of the totals to pinned host memory -- as one CUDA graph.  No
// step needs the host in between, so one graph launch runs a batch.  Graphs
// are kept per batch-size bucket (powers of two from 256 up to the plan's
// maximum); a batch is padded to its bucket with NaN queries, which match
// nothing.  If a batch's totals exceed the capacities the outputs are
// incomplete and the run reports RTREE_EOVERFLOW with the sizes it needed.
#include <cstring>
#include <new>
#include <vector>

#include "internal.cuh"

namespace rt {
namespace {

__global__ void k_fill_nan(float4 *__restrict__ q, int64_t from, int64_t to)
{
    const float nan = __int_as_float(0x7fc00000);
    for (int64_t i = from + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < to;
         i += (int64_t)gridDim.x * blockDim.x)
        q[i] = make_float4(nan, nan, nan, nan);
}

struct Graph {
    int64_t q;
    cudaGraphExec_t exec;
    long long launches;
};

}  // namespace
}  // namespace rt

struct rtree_plan {
    const rtree *tree = nullptr;
    int device = 0;
    int mapping = RTREE_MAP_WARP_PER_QUERY;
    int64_t max_q = 0, ids_cap = 0;
    int64_t leaf_cap = 0;  // leaf-hit slots: the bound pass reserves F per intersecting leaf
    float4 *queries = nullptr;
    rt::SelectBuffers b{};
    void *block = nullptr;            // one device allocation holding the buffers
    int64_t *host = nullptr;          // mapped page-locked: totals [3] + flags (2 x int32)
    int64_t *host_dev = nullptr;      // its device view, written by the graph's last kernel
    cudaStream_t cap_stream = nullptr;
    std::vector<rt::Graph> graphs;
    int64_t last_q = 0;
};

namespace rt {
namespace {

int64_t bucket_of(int64_t q, int64_t max_q)
{
    int64_t b = 256;
    while (b < q)
        b <<= 1;
    return b < max_q ? b : max_q;
}

void free_plan(rtree_plan *p)
{
    for (Graph &g : p->graphs)
        cudaGraphExecDestroy(g.exec);
    p->graphs.clear();
    if (p->block) {
        const rtree_allocator_t *a = p->tree ? p->tree->allocator() : nullptr;
        if (a) {
            cudaDeviceSynchronize();
            a->free(p->block, nullptr, a->ctx);
        } else {
            cudaFree(p->block);
        }
    }
    if (p->host)
        cudaFreeHost(p->host);
    if (p->cap_stream)
        cudaStreamDestroy(p->cap_stream);
    cudaGetLastError();
}

// Carves the plan's buffers out of one allocation (256-byte aligned pieces).
rtree_status allocate(rtree_plan *p)
{
    const int64_t Q = p->max_q, C = p->ids_cap;
    // slots exceed hits: about 2x on large queries, up to F per hit on tiny ones
    const int64_t LC = 2 * C + 4 * (int64_t)p->tree->fanout * Q;
    p->leaf_cap = LC;
    const long long wq_cap = Q + (Q > (1 << 20) ? Q : (1 << 20));
    struct Piece {
        void **dst;
        size_t bytes;
    };
    SelectBuffers &b = p->b;
    Piece pieces[] = {
        {reinterpret_cast<void **>(&p->queries), (size_t)Q * sizeof(float4)},
        {reinterpret_cast<void **>(&b.cnt), (size_t)Q * 4},
        {reinterpret_cast<void **>(&b.cnt_leaf), (size_t)Q * 4},
        {reinterpret_cast<void **>(&b.cnt_rng), (size_t)Q * 4},
        {reinterpret_cast<void **>(&b.off), (size_t)(Q + 1) * 8},
        {reinterpret_cast<void **>(&b.off_leaf), (size_t)(Q + 1) * 8},
        {reinterpret_cast<void **>(&b.off_rng), (size_t)(Q + 1) * 8},
        {reinterpret_cast<void **>(&b.leaf), (size_t)LC * 4},
        {reinterpret_cast<void **>(&b.rng), (size_t)C * 8},
        {reinterpret_cast<void **>(&b.ids), (size_t)C * 4},
        {reinterpret_cast<void **>(&b.cursors), (size_t)Q * 8},
        {reinterpret_cast<void **>(&b.flags), 8},
        {reinterpret_cast<void **>(&b.ctr), 16},
        {reinterpret_cast<void **>(&b.wq_ctl), 24},
        {reinterpret_cast<void **>(&b.wq_items), (size_t)wq_cap * 8},
    };
    size_t total = 0;
    for (const Piece &pc : pieces)
        total += (pc.bytes + 255) & ~(size_t)255;
    if (const rtree_allocator_t *a = p->tree->allocator()) {  // the tree's device-memory hook
        p->block = a->alloc(total, nullptr, a->ctx);
        if (!p->block)
            return fail(RTREE_ENOMEM, "rtree_plan_create: the tree's allocator returned no memory (%zu bytes)",
                        total);
        RT_CUDA(cudaDeviceSynchronize());  // usable by the plan's own streams
    }
    cudaError_t e = p->block ? cudaSuccess : cudaMalloc(&p->block, total);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return fail(RTREE_ENOMEM, "rtree_plan_create: %zu bytes of device memory not available", total);
    }
    if (e != cudaSuccess)
        return fail(RTREE_ECUDA, "rtree_plan_create: cudaMalloc: %s", cudaGetErrorString(e));
    char *at = static_cast<char *>(p->block);
    for (const Piece &pc : pieces) {
        *pc.dst = at;
        at += (pc.bytes + 255) & ~(size_t)255;
    }
    b.rng_cap = b.ids_cap = C;
    b.leaf_cap = LC;
    b.wq_cap = wq_cap;
    RT_CUDA(cudaHostAlloc(reinterpret_cast<void **>(&p->host), 64, cudaHostAllocMapped | cudaHostAllocPortable));
    memset(p->host, 0, 64);
    RT_CUDA(cudaHostGetDevicePointer(reinterpret_cast<void **>(&p->host_dev), p->host, 0));
    return RTREE_OK;
}

// Records the pipeline for a batch of qb queries on the plan's stream.
rtree_status capture(rtree_plan *p, int64_t qb, Graph *out)
{
    cudaStream_t s = p->cap_stream;
    // scratch allocated while capturing becomes graph memory (cudaMallocAsync
    // inside a capture), owned by the graph: never the tree's allocator, whose
    // blocks would be handed out again while the graph still uses them
    AllocScope scope(nullptr);
    RT_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    timing_capture_begin();
    rtree_status st = select_enqueue(p->tree, p->queries, qb, p->mapping, p->b, s);
    if (st == RTREE_OK) {
        // the totals and flags are stored into mapped host memory by a kernel:
        // a small copy would wait behind other plans' result copies
        PostList pl{};
        const void *src[4] = {p->b.off + qb, p->b.off_leaf + qb, p->b.off_rng + qb, p->b.flags};
        for (int i = 0; i < 4; ++i) {
            pl.src[i] = src[i];
            pl.words[i] = 2;
            pl.at[i] = 2 * i;
        }
        pl.n = 4;
        st = post_words(pl, reinterpret_cast<uint32_t *>(p->host_dev), s);
    }
    const long long launches = timing_capture_end();
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(s, &graph);
    if (st != RTREE_OK) {
        if (graph)
            cudaGraphDestroy(graph);
        cudaGetLastError();
        return st;
    }
    if (e != cudaSuccess)
        return fail(RTREE_ECUDA, "rtree_plan_run: stream capture failed: %s", cudaGetErrorString(e));
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess)
        return fail(RTREE_ECUDA, "rtree_plan_run: cudaGraphInstantiate: %s", cudaGetErrorString(e));
    *out = Graph{qb, exec, launches};
    return RTREE_OK;
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

bool on_device(const void *p)
{
    cudaPointerAttributes a;
    memset(&a, 0, sizeof(a));
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace
}  // namespace rt

using namespace rt;

extern "C" {

rtree_status rtree_plan_create(const rtree_t *tree, int64_t max_queries, int64_t max_ids,
                               const rtree_select_opts_t *opts, rtree_plan_t **out)
{
    clear_error();
    if (!out)
        return fail(RTREE_EINVAL, "rtree_plan_create: out is NULL");
    *out = nullptr;
    if (!tree || max_queries < 1 || max_queries >= (int64_t)INT32_MAX || max_ids < 1)
        return fail(RTREE_EINVAL, "rtree_plan_create: need a tree, 1 <= max_queries < 2^31, max_ids >= 1");
    if (opts && opts->unsorted)
        return fail(RTREE_EINVAL, "rtree_plan_create: plans produce sorted results only");
    if (opts && opts->order != RTREE_ORDER_INPUT)
        return fail(RTREE_EINVAL, "rtree_plan_create: plans take queries in input order");
    const int mapping = opts ? opts->mapping : RTREE_MAP_AUTO;
    if (mapping < RTREE_MAP_AUTO || mapping > RTREE_MAP_WORK_QUEUE)
        return fail(RTREE_EINVAL, "rtree_plan_create: unknown mapping %d", mapping);
    try {
        CurrentDevice guard(tree->device);
        rtree_plan *p = new rtree_plan();
        p->tree = tree;
        p->device = tree->device;
        p->mapping = mapping == RTREE_MAP_AUTO ? RTREE_MAP_WARP_PER_QUERY : mapping;
        p->max_q = max_queries;
        p->ids_cap = max_ids;
        rtree_status st = allocate(p);
        if (st == RTREE_OK && cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
            st = fail(RTREE_ECUDA, "rtree_plan_create: cudaStreamCreate failed");
        if (st != RTREE_OK) {
            free_plan(p);
            delete p;
            return st;
        }
        *out = p;
        return RTREE_OK;
    } catch (...) {
        return fail(RTREE_ENOMEM, "rtree_plan_create: host allocation failed");
    }
}

rtree_status rtree_plan_run(rtree_plan_t *p, const float *queries, int64_t q, void *stream,
                            int64_t *total)
{
    clear_error();
    if (!p || !total)
        return fail(RTREE_EINVAL, "rtree_plan_run: NULL plan or total");
    *total = 0;
    if (q < 0 || q > p->max_q)
        return fail(RTREE_EOVERFLOW, "rtree_plan_run: %lld queries; the plan holds at most %lld",
                    (long long)q, (long long)p->max_q);
    if (q > 0 && !queries)
        return fail(RTREE_EINVAL, "rtree_plan_run: queries is NULL");
    try {
        CurrentDevice guard(p->device);
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        RT_TRY(tree_ready_on(p->tree, s));
        const int64_t qb = bucket_of(q > 0 ? q : 1, p->max_q);
        if (q > 0)
            RT_CUDA(cudaMemcpyAsync(p->queries, queries, q * sizeof(float4),
                                    on_device(queries) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
        if (qb > q) {
            KernelTimer kt_("plan_pad", s);
            k_fill_nan<<<(unsigned)((qb - q + 255) / 256), 256, 0, s>>>(p->queries, q, qb);
            RT_LAUNCH();
        }
        Graph *g = nullptr;
        for (Graph &x : p->graphs)
            if (x.q == qb)
                g = &x;
        if (!g) {
            Graph ng{};
            RT_TRY(capture(p, qb, &ng));
            p->graphs.push_back(ng);
            g = &p->graphs.back();
        }
        RT_CUDA(cudaGraphLaunch(g->exec, s));
        RT_CUDA(cudaStreamSynchronize(s));
        timing_add_replay("plan_graph", g->launches);
        p->last_q = q;
        const int64_t tot = p->host[0], tleaf = p->host[1], trng = p->host[2];
        int32_t fl[2];
        memcpy(fl, p->host + 3, sizeof(fl));
        *total = tot;
        if (fl[0] & 4)
            return fail(RTREE_ETIMEOUT, "rtree_plan_run: a work-queue wait exceeded its limit");
        if (tot > p->ids_cap || tleaf > p->leaf_cap || trng > p->ids_cap)
            return fail(RTREE_EOVERFLOW,
                        "rtree_plan_run: the batch needs %lld ids (%lld leaf-hit slots, %lld ranges) but "
                        "the plan holds %lld ids and %lld slots; results are incomplete",
                        (long long)tot, (long long)tleaf, (long long)trng, (long long)p->ids_cap,
                        (long long)p->leaf_cap);
        if (fl[0] || fl[1])
            return fail(RTREE_EINTERNAL, "rtree_plan_run: device flags 0x%x / 0x%x", fl[0], fl[1]);
        return RTREE_OK;
    } catch (...) {
        return fail(RTREE_ENOMEM, "rtree_plan_run: host allocation failed");
    }
}

const int64_t *rtree_plan_offsets(const rtree_plan_t *p) { return p ? p->b.off : nullptr; }
const int32_t *rtree_plan_ids(const rtree_plan_t *p) { return p ? p->b.ids : nullptr; }

void rtree_plan_free(rtree_plan_t *p)
{
    if (!p)
        return;
    CurrentDevice guard(p->device);
    free_plan(p);
    delete p;
}

}  // extern "C"
