// capi.cu -- the extern "C" entry points declared in include/rtree.h.
//
// Argument checks, host/device staging of inputs, error reporting and
// object lifetimes live here; the computation is in build.cu, select.cu,
// segsort.cu, join.cu, radix_sort.cu and scan.cu.
#include <atomic>
#include <cstdarg>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <string>

#include "internal.cuh"

namespace rt {

static thread_local std::string g_err;
static std::atomic<long long> g_alloc_countdown{-1};  // < 0: no injected failure
thread_local const rtree_allocator_t *t_alloc = nullptr;

// Test hook (rtree_debug_wq_wait): the next work-queue pass waits at most
// this many cycles and, with hold, counts one item that is never published.
static std::atomic<long long> g_dbg_wait_cycles{0};
static std::atomic<int> g_dbg_hold{0};

void debug_wq_take(long long *cycles, int *hold)
{
    *cycles = g_dbg_wait_cycles.exchange(0);
    *hold = g_dbg_hold.exchange(0);
}

rtree_status fail(rtree_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

void clear_error() { g_err.clear(); }

void setup_device_pool(int dev)
{
    static std::mutex mu;
    static bool done[64] = {};
    std::lock_guard<std::mutex> g(mu);
    if (dev < 0 || dev >= 64 || done[dev])
        return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t keep = UINT64_MAX;  // keep freed blocks in the pool between calls
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    cudaGetLastError();
    done[dev] = true;
}

rtree_status dmalloc(void **p, size_t bytes, cudaStream_t s, const char *what)
{
    *p = nullptr;
    long long c = g_alloc_countdown.load();
    while (c >= 0) {
        if (g_alloc_countdown.compare_exchange_weak(c, c - 1)) {
            if (c == 0)
                return fail(RTREE_ENOMEM, "injected allocation failure (%s, %zu bytes)", what, bytes);
            break;
        }
    }
    if (t_alloc) {
        *p = t_alloc->alloc(bytes, s, t_alloc->ctx);
        if (!*p)
            return fail(RTREE_ENOMEM, "the tree's allocator returned no memory: %zu bytes for %s", bytes, what);
        return RTREE_OK;
    }
    cudaError_t e = cudaMallocAsync(p, bytes, s);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        *p = nullptr;
        return fail(RTREE_ENOMEM, "out of device memory: %zu bytes for %s", bytes, what);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(RTREE_ECUDA, "cudaMallocAsync(%zu) for %s: %s", bytes, what, cudaGetErrorString(e));
    }
    return RTREE_OK;
}

void dfree(void *p, cudaStream_t s)
{
    if (!p)
        return;
    if (t_alloc)
        t_alloc->free(p, s, t_alloc->ctx);
    else
        cudaFreeAsync(p, s);
}

namespace {
// Gives p back to allocator a (null: the default pool): in the order of
// stream s if `ordered`, else once the whole device has finished.
void release(void *p, const rtree_allocator_t *a, cudaStream_t s, bool ordered)
{
    if (!p)
        return;
    if (!ordered)
        cudaDeviceSynchronize();
    if (a)
        a->free(p, ordered ? s : nullptr, a->ctx);
    else if (ordered)
        cudaFreeAsync(p, s);
    else
        cudaFree(p);
}
}  // namespace

int sm_count()
{
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

namespace {

// Where a pointer lives: 1 = device memory usable by kernels, 0 = host.
int pointer_kind(const void *p, int *device)
{
    cudaPointerAttributes a;
    memset(&a, 0, sizeof(a));
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) {
        if (device)
            *device = a.device;
        return 1;
    }
    return 0;
}

// Returns a 16-byte aligned device copy (or the pointer itself) of n rows.
template <typename T>
rtree_status stage(const void *p, size_t bytes, size_t align, cudaStream_t s, DevBuf<T> &tmp,
                   const T **out)
{
    if (bytes == 0) {
        RT_TRY(tmp.alloc(1, "input staging"));
        *out = tmp.p;
        return RTREE_OK;
    }
    const bool dev = pointer_kind(p, nullptr) == 1;
    if (dev && (reinterpret_cast<uintptr_t>(p) % align) == 0) {
        *out = static_cast<const T *>(p);
        return RTREE_OK;
    }
    RT_TRY(tmp.alloc(bytes / sizeof(T) + 1, "input staging"));
    RT_CUDA(cudaMemcpyAsync(tmp.p, p, bytes, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    *out = tmp.p;
    return RTREE_OK;
}

}  // namespace

void free_tree_arrays(rtree *t, cudaStream_t s, bool ordered)
{
    const rtree_allocator_t *a = t->allocator();
    release(t->mbr, a, s, ordered);
    release(t->meta, a, s, ordered);
    release(t->nbox, a, s, ordered);
    release(t->ids, a, s, ordered);
    release(t->leaf_part, a, s, ordered);
    t->mbr = nullptr;
    t->meta = nullptr;
    t->nbox = nullptr;
    t->ids = nullptr;
    t->leaf_part = nullptr;
    if (t->root_mb) {  // a kernel may still write it: reused only after its event
        mailbox_put_deferred(t->root_mb);
        delete t->root_mb;
        t->root_mb = nullptr;
    }
}

void free_result_arrays(rtree_result *r, cudaStream_t s, bool ordered)
{
    const rtree_allocator_t *a = r->custom_alloc ? &r->alloc : nullptr;
    release(r->offsets, a, s, ordered);
    release(r->ids, a, s, ordered);
    r->offsets = nullptr;
    r->ids = nullptr;
    if (r->status) {
        mailbox_put_deferred(r->status);
        delete r->status;
        r->status = nullptr;
    }
}

bool fanout_ok(int f) { return f == 4 || f == 8 || f == 16 || f == 32 || f == 64 || f == 128; }

namespace {
std::mutex g_root_mu;  // guards rtree::root_mb / root_ready of every tree
}

rtree_status tree_ready_on(const rtree *t, cudaStream_t s)
{
    if (!t)
        return RTREE_OK;
    std::lock_guard<std::mutex> g(g_root_mu);
    if (t->root_mb)  // the build's last kernel records this event
        RT_CUDA(cudaStreamWaitEvent(s, t->root_mb->ev, 0));
    return RTREE_OK;
}

rtree_status tree_root_box(const rtree *t, float box[4])
{
    std::lock_guard<std::mutex> g(g_root_mu);
    rtree *m = const_cast<rtree *>(t);
    if (!m->root_ready && m->root_mb) {
        RT_TRY(mailbox_wait(*m->root_mb));  // the build's packing has finished
        const volatile uint32_t *w = m->root_mb->h;
        for (int c = 0; c < 4; ++c) {
            const uint32_t v = w[c];
            memcpy(&m->root_mbr[c], &v, 4);
        }
        mailbox_put(m->root_mb);
        delete m->root_mb;
        m->root_mb = nullptr;
        m->root_ready = true;
    }
    memcpy(box, m->root_mbr, 4 * sizeof(float));
    return RTREE_OK;
}

}  // namespace rt

using namespace rt;

extern "C" {

const char *rtree_last_error(void) { return g_err.c_str(); }

const char *rtree_version(void) { return "rtree-gb300 0.1 (sm_103a)"; }

// Test hook: make the k-th following device allocation fail (k = -1 disables).
void rtree_debug_fail_alloc_after(long long k) { g_alloc_countdown.store(k); }

void rtree_debug_wq_wait(long long cycles, int hold)
{
    g_dbg_wait_cycles.store(cycles > 0 ? cycles : 0);
    g_dbg_hold.store(hold != 0);
}

rtree_status rtree_build(const float *rects, const int32_t *ids, int64_t n,
                         const rtree_config_t *cfg, const rtree_allocator_t *alloc, void *stream,
                         rtree_t **out)
{
    clear_error();
    if (!out)
        return fail(RTREE_EINVAL, "rtree_build: out is NULL");
    *out = nullptr;
    if (n < 0 || n >= (int64_t)INT32_MAX)
        return fail(RTREE_EINVAL, "rtree_build: n = %lld out of range [0, 2^31-1)", (long long)n);
    if (n > 0 && !rects)
        return fail(RTREE_EINVAL, "rtree_build: rects is NULL");
    const int F = (cfg && cfg->fanout) ? cfg->fanout : 16;
    const int layout = cfg ? cfg->layout : RTREE_LAYOUT_SOA;
    const bool sort_children = cfg && cfg->sort_children;
    if (cfg && cfg->sort_children != 0 && cfg->sort_children != 1)
        return fail(RTREE_EINVAL, "rtree_build: sort_children must be 0 or 1");
    if (!fanout_ok(F))
        return fail(RTREE_EINVAL, "rtree_build: fanout %d not in {4,8,16,32,64,128}", F);
    if (layout != RTREE_LAYOUT_SOA && layout != RTREE_LAYOUT_AOS && layout != RTREE_LAYOUT_LOHI)
        return fail(RTREE_EINVAL, "rtree_build: unknown layout %d", layout);
    if (alloc && (!alloc->alloc || !alloc->free))
        return fail(RTREE_EINVAL, "rtree_build: allocator with a NULL alloc or free function");
    try {
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        int dev = 0;
        RT_CUDA(cudaGetDevice(&dev));
        if (n > 0)
            pointer_kind(rects, &dev);
        DeviceGuard guard(dev);
        setup_device_pool(dev);
        rtree *t = new rtree();
        t->device = dev;
        if (alloc) {
            t->alloc = *alloc;
            t->custom_alloc = true;
        }
        AllocScope scope(t->allocator());
        rtree_status st;
        {
            DevBuf<float4> rtmp(s);
            DevBuf<int32_t> itmp(s);
            const float4 *drects = nullptr;
            const int32_t *dids = nullptr;
            st = stage<float4>(rects, (size_t)n * 16, 16, s, rtmp, &drects);
            if (st == RTREE_OK && ids)
                st = stage<int32_t>(ids, (size_t)n * 4, 4, s, itmp, &dids);
            if (st == RTREE_OK)
                st = build_tree(drects, dids, n, F, layout, sort_children, s, t);
            if (st == RTREE_OK) {  // launch errors only: the packing runs on in the order of s
                cudaError_t e = cudaGetLastError();
                if (e != cudaSuccess)
                    st = fail(RTREE_ECUDA, "rtree_build: %s", cudaGetErrorString(e));
            }
        }
        if (st != RTREE_OK) {
            free_tree_arrays(t);
            delete t;
            return st;
        }
        timing_resolve();
        *out = t;
        return RTREE_OK;
    } catch (const std::bad_alloc &) {
        return fail(RTREE_ENOMEM, "rtree_build: host allocation failed");
    } catch (...) {
        return fail(RTREE_EINTERNAL, "rtree_build: unexpected exception");
    }
}

void rtree_free(rtree_t *t)
{
    if (!t)
        return;
    DeviceGuard guard(t->device);
    free_tree_arrays(t);
    delete t;
}

void rtree_free_async(rtree_t *t, void *stream)
{
    if (!t)
        return;
    DeviceGuard guard(t->device);
    if (tree_ready_on(t, static_cast<cudaStream_t>(stream)) != RTREE_OK)
        cudaDeviceSynchronize();  // could not order the release after the build: wait for it
    free_tree_arrays(t, static_cast<cudaStream_t>(stream), true);
    delete t;
}

rtree_status rtree_get_info(const rtree_t *t, rtree_info_t *info)
{
    clear_error();
    if (!t || !info)
        return fail(RTREE_EINVAL, "rtree_get_info: NULL argument");
    info->n = t->n;
    info->nodes = t->nodes;
    info->levels = t->levels;
    info->fanout = t->fanout;
    info->layout = t->layout;
    info->device = t->device;
    info->device_bytes = t->bytes;
    {
        DeviceGuard guard(t->device);
        RT_TRY(tree_root_box(t, info->root_mbr));
    }
    info->sort_children = t->sorted;
    memset(info->reserved, 0, sizeof(info->reserved));
    return RTREE_OK;
}

rtree_status rtree_export(const rtree_t *t, int64_t *level_nodes, int32_t *counts, float *mbrs,
                          int32_t *leaf_ids, void *stream)
{
    clear_error();
    if (!t)
        return fail(RTREE_EINVAL, "rtree_export: tree is NULL");
    if (t->levels == 0)
        return RTREE_OK;
    if (!level_nodes || !counts || !mbrs || !leaf_ids)
        return fail(RTREE_EINVAL, "rtree_export: NULL output");
    try {
        DeviceGuard guard(t->device);
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        RT_TRY(tree_ready_on(t, s));
        const int F = t->fanout;
        const int64_t M = t->nodes;
        for (int e = 0; e < t->levels; ++e)
            level_nodes[e] = t->level_nodes[e];
        int4 *meta = static_cast<int4 *>(malloc(M * sizeof(int4)));
        float *raw = static_cast<float *>(malloc(M * F * 4 * sizeof(float)));
        if (!meta || !raw) {
            free(meta);
            free(raw);
            return fail(RTREE_ENOMEM, "rtree_export: host allocation failed");
        }
        cudaError_t e1 = cudaMemcpyAsync(meta, t->meta, M * sizeof(int4), cudaMemcpyDeviceToHost, s);
        cudaError_t e2 = cudaMemcpyAsync(raw, t->mbr, M * F * 4 * sizeof(float), cudaMemcpyDeviceToHost, s);
        cudaError_t e3 = cudaMemcpyAsync(leaf_ids, t->ids, t->n * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
        cudaError_t e4 = cudaStreamSynchronize(s);
        if (e1 || e2 || e3 || e4) {
            free(meta);
            free(raw);
            return fail(RTREE_ECUDA, "rtree_export: copy failed: %s",
                        cudaGetErrorString(e1 ? e1 : e2 ? e2 : e3 ? e3 : e4));
        }
        for (int64_t g = 0; g < M; ++g) {
            counts[g] = meta[g].y;
            for (int j = 0; j < F; ++j) {
                float *o = mbrs + (g * F + j) * 4;
                if (t->layout == RTREE_LAYOUT_AOS) {
                    memcpy(o, raw + (g * F + j) * 4, 16);
                } else if (t->layout == RTREE_LAYOUT_LOHI) {
                    const float *b = raw + g * 4 * F;
                    o[0] = b[2 * j];
                    o[1] = b[2 * j + 1];
                    o[2] = b[2 * F + 2 * j];
                    o[3] = b[2 * F + 2 * j + 1];
                } else {
                    const float *b = raw + g * 4 * F + j;
                    o[0] = b[0];
                    o[1] = b[F];
                    o[2] = b[2 * F];
                    o[3] = b[3 * F];
                }
            }
        }
        free(meta);
        free(raw);
        return RTREE_OK;
    } catch (...) {
        return fail(RTREE_ENOMEM, "rtree_export: host allocation failed");
    }
}

rtree_status rtree_range_select(const rtree_t *t, const float *queries, int64_t q,
                                const rtree_select_opts_t *opts, void *stream,
                                rtree_result_t **out)
{
    clear_error();
    if (!out)
        return fail(RTREE_EINVAL, "rtree_range_select: out is NULL");
    *out = nullptr;
    if (!t)
        return fail(RTREE_EINVAL, "rtree_range_select: tree is NULL");
    if (q < 0 || q >= (int64_t)INT32_MAX)
        return fail(RTREE_EINVAL, "rtree_range_select: q = %lld out of range", (long long)q);
    if (q > 0 && !queries)
        return fail(RTREE_EINVAL, "rtree_range_select: queries is NULL");
    const bool sorted = !(opts && opts->unsorted);
    const int mapping = opts ? opts->mapping : RTREE_MAP_AUTO;
    if (mapping < RTREE_MAP_AUTO || mapping > RTREE_MAP_WORK_QUEUE)
        return fail(RTREE_EINVAL, "rtree_range_select: unknown mapping %d", mapping);
    const int order = opts ? opts->order : RTREE_ORDER_INPUT;
    if (order != RTREE_ORDER_INPUT && order != RTREE_ORDER_HILBERT)
        return fail(RTREE_EINVAL, "rtree_range_select: unknown order %d", order);
    try {
        DeviceGuard guard(t->device);
        AllocScope scope(t->allocator());
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        rtree_result *res = new rtree_result();
        res->device = t->device;
        res->alloc = t->alloc;
        res->custom_alloc = t->custom_alloc;
        res->stream = stream;
        rtree_status st = tree_ready_on(t, s);
        if (st == RTREE_OK) {
            DevBuf<float4> qtmp(s);
            const float4 *dq = nullptr;
            st = stage<float4>(queries, (size_t)q * 16, 16, s, qtmp, &dq);
            if (st == RTREE_OK)
                st = range_select(t, dq, q, sorted, mapping, order, s, res);
            if (st == RTREE_OK) {  // launch errors; the rest is reported by rtree_result_wait
                cudaError_t e = cudaGetLastError();
                if (e != cudaSuccess)
                    st = fail(RTREE_ECUDA, "rtree_range_select: %s", cudaGetErrorString(e));
            }
        }
        if (st != RTREE_OK) {
            free_result_arrays(res);
            delete res;
            return st;
        }
        timing_resolve();
        *out = res;
        return RTREE_OK;
    } catch (...) {
        return fail(RTREE_ENOMEM, "rtree_range_select: host allocation failed");
    }
}

rtree_status rtree_result_wait(const rtree_result_t *r)
{
    clear_error();
    if (!r)
        return fail(RTREE_EINVAL, "rtree_result_wait: result is NULL");
    if (!r->status)
        return RTREE_OK;
    DeviceGuard guard(r->device);
    RT_TRY(mailbox_wait(*r->status));
    const volatile uint32_t *w = r->status->h;
    const uint32_t sel = w[0], sort = w[1];
    if (sel & 4u)
        return fail(RTREE_ETIMEOUT, "range select: a work-queue wait exceeded its limit");
    if (sel)
        return fail(RTREE_EINTERNAL, "range select pass reported device flags 0x%x", sel);
    if (sort)
        return fail(RTREE_EINTERNAL, "segmented sort reported device flags 0x%x", sort);
    return RTREE_OK;
}

namespace {

rtree_status select_host_call(const char *name, const rtree_t *t, const float *queries, int64_t q,
                              const rtree_select_opts_t *opts, void *stream, int64_t *offsets,
                              int32_t *ids, int64_t capacity, int64_t *total, rtree_pending_t **pending)
{
    if (!t || !offsets || !total || capacity < 0 || (capacity > 0 && !ids))
        return fail(RTREE_EINVAL, "%s: bad argument", name);
    *total = 0;
    if (q < 0 || q >= (int64_t)INT32_MAX)
        return fail(RTREE_EINVAL, "%s: q = %lld out of range", name, (long long)q);
    if (q > 0 && !queries)
        return fail(RTREE_EINVAL, "%s: queries is NULL", name);
    const bool sorted = !(opts && opts->unsorted);
    const int mapping = opts ? opts->mapping : RTREE_MAP_AUTO;
    if (mapping < RTREE_MAP_AUTO || mapping > RTREE_MAP_WORK_QUEUE)
        return fail(RTREE_EINVAL, "%s: unknown mapping %d", name, mapping);
    const int order = opts ? opts->order : RTREE_ORDER_INPUT;
    if (order != RTREE_ORDER_INPUT && order != RTREE_ORDER_HILBERT)
        return fail(RTREE_EINVAL, "%s: unknown order %d", name, order);
    try {
        DeviceGuard guard(t->device);
        AllocScope scope(t->allocator());
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        RT_TRY(tree_ready_on(t, s));
        DevBuf<float4> qtmp(s);
        const float4 *dq = nullptr;
        RT_TRY(stage<float4>(queries, (size_t)q * 16, 16, s, qtmp, &dq));
        return range_select_host_begin(t, dq, q, sorted, mapping, order, s, offsets, ids, capacity, total,
                                       pending);
    } catch (...) {
        return fail(RTREE_ENOMEM, "%s: host allocation failed", name);
    }
}

}  // namespace

rtree_status rtree_range_select_host(const rtree_t *t, const float *queries, int64_t q,
                                     const rtree_select_opts_t *opts, void *stream, int64_t *offsets,
                                     int32_t *ids, int64_t capacity, int64_t *total)
{
    clear_error();
    rtree_pending_t *p = nullptr;
    rtree_status st = select_host_call("rtree_range_select_host", t, queries, q, opts, stream, offsets, ids,
                                       capacity, total, &p);
    if (p) {
        const rtree_status st2 = range_select_host_finish(p);
        st = st != RTREE_OK ? st : st2;
    }
    if (st == RTREE_OK) {
        DeviceGuard guard(t->device);
        cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
        if (e != cudaSuccess)
            st = fail(RTREE_ECUDA, "rtree_range_select_host: %s", cudaGetErrorString(e));
    }
    timing_resolve();
    return st;
}

rtree_status rtree_range_select_host_async(const rtree_t *t, const float *queries, int64_t q,
                                           const rtree_select_opts_t *opts, void *stream, int64_t *offsets,
                                           int32_t *ids, int64_t capacity, int64_t *total,
                                           rtree_pending_t **pending)
{
    clear_error();
    if (!pending)
        return fail(RTREE_EINVAL, "rtree_range_select_host_async: pending is NULL");
    *pending = nullptr;
    return select_host_call("rtree_range_select_host_async", t, queries, q, opts, stream, offsets, ids,
                            capacity, total, pending);
}

rtree_status rtree_pending_wait(rtree_pending_t *pending)
{
    clear_error();
    if (!pending)
        return RTREE_OK;
    const rtree_status st = range_select_host_finish(pending);
    timing_resolve();
    return st;
}

rtree_status rtree_range_select_stats(const rtree_t *t, const float *queries, int64_t q, void *stream,
                                      int64_t stats[8])
{
    clear_error();
    if (!t || !stats || q < 0 || (q > 0 && !queries))
        return fail(RTREE_EINVAL, "rtree_range_select_stats: bad argument");
    try {
        DeviceGuard guard(t->device);
        AllocScope scope(t->allocator());
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        RT_TRY(tree_ready_on(t, s));
        DevBuf<float4> qtmp(s);
        const float4 *dq = nullptr;
        RT_TRY(stage<float4>(queries, (size_t)q * 16, 16, s, qtmp, &dq));
        RT_TRY(select_stats(t, dq, q, s, stats));
        RT_CUDA(cudaStreamSynchronize(s));
        timing_resolve();
        return RTREE_OK;
    } catch (...) {
        return fail(RTREE_ENOMEM, "rtree_range_select_stats: host allocation failed");
    }
}

rtree_status rtree_join(const rtree_t *r, const rtree_t *s_tree, void *stream, rtree_result_t **out)
{
    return rtree_join_ex(r, s_tree, nullptr, stream, out);
}

namespace {
rtree_status join_impl(const rtree_t *r, const rtree_t *s_tree, const rtree_join_opts_t *opts,
                       void *stream, rtree_result_t **out, int64_t *stats);
}

rtree_status rtree_join_ex(const rtree_t *r, const rtree_t *s_tree, const rtree_join_opts_t *opts,
                           void *stream, rtree_result_t **out)
{
    return join_impl(r, s_tree, opts, stream, out, nullptr);
}

rtree_status rtree_join_stats(const rtree_t *r, const rtree_t *s_tree, const rtree_join_opts_t *opts,
                              void *stream, int64_t stats[8])
{
    if (!stats)
        return fail(RTREE_EINVAL, "rtree_join_stats: stats is NULL");
    for (int i = 0; i < 8; ++i)
        stats[i] = 0;
    rtree_result_t *res = nullptr;
    const rtree_status st = join_impl(r, s_tree, opts, stream, &res, stats);
    rtree_result_free(res);
    return st;
}

namespace {
rtree_status join_impl(const rtree_t *r, const rtree_t *s_tree, const rtree_join_opts_t *opts,
                       void *stream, rtree_result_t **out, int64_t *stats)
{
    clear_error();
    if (!out)
        return fail(RTREE_EINVAL, "rtree_join: out is NULL");
    *out = nullptr;
    if (!r || !s_tree)
        return fail(RTREE_EINVAL, "rtree_join: tree is NULL");
    if (r->device != s_tree->device)
        return fail(RTREE_EINVAL, "rtree_join: trees on devices %d and %d", r->device, s_tree->device);
    const int prune = opts ? opts->prune : RTREE_PRUNE_AUTO;
    if (prune != RTREE_PRUNE_AUTO && prune != RTREE_PRUNE_OFF && prune != RTREE_PRUNE_ON)
        return fail(RTREE_EINVAL, "rtree_join: unknown prune mode %d", prune);
    const bool both_sorted = r->sorted && s_tree->sorted;
    if (prune == RTREE_PRUNE_ON && !both_sorted)
        return fail(RTREE_EINVAL, "rtree_join: pruning needs both trees built with sort_children");
    const int traversal = opts ? opts->traversal : RTREE_JOIN_AUTO;
    if (traversal < RTREE_JOIN_AUTO || traversal > RTREE_JOIN_QUEUE)
        return fail(RTREE_EINVAL, "rtree_join: unknown traversal %d", traversal);
    // the counters come from the level-by-level form, which is also the
    // default (measured faster than the queued form on the 2M x 2M join)
    const bool queued = !stats && traversal == RTREE_JOIN_QUEUE;
    try {
        DeviceGuard guard(r->device);
        AllocScope scope(r->allocator());
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        rtree_result *res = new rtree_result();
        res->device = r->device;
        res->alloc = r->alloc;
        res->custom_alloc = r->custom_alloc;
        res->stream = stream;
        rtree_status st = tree_ready_on(r, s);
        if (st == RTREE_OK)
            st = tree_ready_on(s_tree, s);
        const bool pr = prune != RTREE_PRUNE_OFF && both_sorted;
        bool by_levels = !queued;
        if (st == RTREE_OK && queued)
            st = tree_join_queue(r, s_tree, pr, s, res, &by_levels);
        if (st == RTREE_OK && by_levels) {
            st = tree_join(r, s_tree, pr, s, res, stats);
            if (st == RTREE_OK) {
                cudaError_t e = cudaStreamSynchronize(s);
                if (e != cudaSuccess)
                    st = fail(RTREE_ECUDA, "rtree_join: %s", cudaGetErrorString(e));
            }
        } else if (st == RTREE_OK) {  // launch errors; the rest is reported by rtree_result_wait
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess)
                st = fail(RTREE_ECUDA, "rtree_join: %s", cudaGetErrorString(e));
        }
        if (st != RTREE_OK) {
            free_result_arrays(res);
            delete res;
            return st;
        }
        timing_resolve();
        *out = res;
        return RTREE_OK;
    } catch (...) {
        return fail(RTREE_ENOMEM, "rtree_join: host allocation failed");
    }
}
}  // namespace

int64_t rtree_result_total(const rtree_result_t *r) { return r ? r->total : 0; }
int64_t rtree_result_rows(const rtree_result_t *r) { return r ? r->rows : 0; }
const int64_t *rtree_result_offsets(const rtree_result_t *r) { return r ? r->offsets : nullptr; }
const int32_t *rtree_result_ids(const rtree_result_t *r) { return r ? r->ids : nullptr; }

rtree_status rtree_result_copy_to_host(const rtree_result_t *r, int64_t *offsets, int32_t *ids,
                                       void *stream)
{
    clear_error();
    if (!r)
        return fail(RTREE_EINVAL, "rtree_result_copy_to_host: result is NULL");
    DeviceGuard guard(r->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (r->status)  // after the producing call's work, whichever stream it ran on
        RT_CUDA(cudaStreamWaitEvent(s, r->status->ev, 0));
    if (offsets && r->offsets)
        RT_CUDA(cudaMemcpyAsync(offsets, r->offsets, (r->rows + 1) * sizeof(int64_t),
                                cudaMemcpyDeviceToHost, s));
    const int64_t nids = r->offsets ? r->total : 2 * r->total;
    if (ids && nids > 0)
        RT_CUDA(cudaMemcpyAsync(ids, r->ids, nids * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    RT_CUDA(cudaStreamSynchronize(s));
    return rtree_result_wait(r);
}

void rtree_result_free(rtree_result_t *r)
{
    if (!r)
        return;
    DeviceGuard guard(r->device);
    free_result_arrays(r);
    delete r;
}

void rtree_result_free_async(rtree_result_t *r, void *stream)
{
    if (!r)
        return;
    DeviceGuard guard(r->device);
    free_result_arrays(r, static_cast<cudaStream_t>(stream), true);
    delete r;
}

}  // extern "C"
