// internal.cuh -- shared declarations of the R-tree CUDA library (not public).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>

#include "rtree.h"

#define RT_FULL 0xffffffffu
#define RT_MAX_LEVELS 40

namespace rt {

// ------------------------------------------------------------------ errors
// Records a thread-local message and returns st.
rtree_status fail(rtree_status st, const char *fmt, ...) __attribute__((format(printf, 2, 3)));
void clear_error();

#define RT_CUDA(call)                                                                      \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return ::rt::fail(RTREE_ECUDA, "%s failed: %s (%s:%d)", #call,                 \
                              cudaGetErrorString(e_), __FILE__, __LINE__);                 \
    } while (0)
#define RT_LAUNCH() RT_CUDA(cudaGetLastError())
#define RT_TRY(x)                                                                          \
    do {                                                                                   \
        rtree_status s_ = (x);                                                             \
        if (s_ != RTREE_OK)                                                                \
            return s_;                                                                     \
    } while (0)

// Takes (and clears) the rtree_debug_wq_wait setting for the next
// work-queue pass: a wait limit in cycles (0: the default) and whether to
// count one never-published item.
void debug_wq_take(long long *cycles, int *hold);

// ------------------------------------------------------------------ memory
// The device-memory hook of the call in progress on this host thread (the
// tree's allocator), or null for the stream-ordered pool of the current
// device (cudaMallocAsync / cudaFreeAsync).  Entry points set it for their
// duration with an AllocScope.
extern thread_local const rtree_allocator_t *t_alloc;
struct AllocScope {
    const rtree_allocator_t *prev;
    explicit AllocScope(const rtree_allocator_t *a) : prev(t_alloc) { t_alloc = a; }
    ~AllocScope() { t_alloc = prev; }
    AllocScope(const AllocScope &) = delete;
    AllocScope &operator=(const AllocScope &) = delete;
};
// Device memory from t_alloc, usable in the order of stream s.  A host-side
// counter can make the k-th allocation fail (fault injection for tests; no
// GPU fault is involved).
rtree_status dmalloc(void **p, size_t bytes, cudaStream_t s, const char *what);
// Keeps freed blocks in the device's default pool between calls (once per device).
void setup_device_pool(int dev);
// Releases a tree's device arrays (not the struct): after the whole device
// has finished when s is null, else in the order of stream s.
void free_tree_arrays(rtree *t, cudaStream_t s = nullptr, bool ordered = false);
// The tree's bounding box, waiting (once) for the build that posted it.
rtree_status tree_root_box(const rtree *t, float box[4]);
// Orders stream s after the tree's build (the build returns before its
// packing has run; a call on another stream must not read the tree early).
rtree_status tree_ready_on(const rtree *t, cudaStream_t s);
// Releases a result's device arrays the same way.
void free_result_arrays(rtree_result *r, cudaStream_t s = nullptr, bool ordered = false);
bool fanout_ok(int f);

// Makes `dev` current for the scope, restoring the previous device after.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        cudaGetDevice(&prev);
        if (dev != prev)
            cudaSetDevice(dev);
    }
    ~DeviceGuard()
    {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev)
            cudaSetDevice(prev);
    }
};
void dfree(void *p, cudaStream_t s);

template <typename T>
struct DevBuf {
    T *p = nullptr;
    cudaStream_t s = nullptr;
    DevBuf() = default;
    explicit DevBuf(cudaStream_t st) : s(st) {}
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    ~DevBuf() { reset(); }
    rtree_status alloc(size_t n, const char *what)
    {
        reset();
        return dmalloc(reinterpret_cast<void **>(&p), (n ? n : 1) * sizeof(T), s, what);
    }
    void reset()
    {
        if (p) {
            dfree(p, s);
            p = nullptr;
        }
    }
    T *release()
    {
        T *q = p;
        p = nullptr;
        return q;
    }
};

int sm_count();

// Counts a kernel launch under `name` and, when timing is enabled, records
// CUDA events around it on stream s.  Scope it around the launch.
class KernelTimer {
  public:
    KernelTimer(const char *name, cudaStream_t s);
    ~KernelTimer();
    KernelTimer(const KernelTimer &) = delete;
    KernelTimer &operator=(const KernelTimer &) = delete;

  private:
    cudaStream_t s_;
    int entry_ = 0;
    cudaEvent_t a_ = nullptr, b_ = nullptr;
};
// Times a span of work on stream s under `name` (events on s at both ends)
// without counting it as a kernel launch; for spans whose kernels run
// concurrently on several streams, where per-kernel times overlap.
class PhaseTimer {
  public:
    PhaseTimer(const char *name, cudaStream_t s);
    ~PhaseTimer();
    PhaseTimer(const PhaseTimer &) = delete;
    PhaseTimer &operator=(const PhaseTimer &) = delete;

  private:
    cudaStream_t s_;
    int entry_ = 0;
    cudaEvent_t a_ = nullptr, b_ = nullptr;
};
// Resolves recorded event pairs into totals (call after a stream sync).
void timing_resolve();
// Graph capture on this thread: launches are counted, not timed; each replay
// of the captured graph adds its launch count under `name`.
void timing_capture_begin();
long long timing_capture_end();
void timing_add_replay(const char *name, long long launches);

// -------------------------------------------------------------------- tree
// Device view of a tree.  Nodes of all levels are numbered level by level
// from the root (node 0); leaves are the last level.
//   mbr : entry MBRs.  SOA: node g owns floats [g*4F, g*4F+4F): F lower-x,
//         F lower-y, F upper-x, F upper-y.  AOS: node g owns float4 slots
//         [g*F, g*F+F).  Unused slots hold (+inf, +inf, -inf, -inf).
//   meta: per node {first, count, elo, ehi}: first = global index of the
//         first child (internal) or index of the first entry in ids (leaf);
//         [elo, ehi) = the ids of all entries under the node.
//   nbox: per node, its bounding box (equal to its entry in the parent).
//   ids : entry ids, leaves in node order, entries in slot order.
struct Mailbox;

struct TreeDev {
    const float *mbr;
    const int4 *meta;
    const float4 *nbox;
    const int32_t *ids;
    int32_t leaf_base;
    int32_t nodes;
    int32_t levels;
    int32_t fanout;
    int32_t layout;
    int32_t sorted;  // entries of every node ascend by lx
    // The leaf level's one short leaf: {its position among the leaves (-1:
    // none), its count, how many leaves are short}.  With at most one short
    // leaf, leaf s holds entries [s*F - (s > pos ? F - count : 0), + F or
    // count) of the id array, without reading its metadata.
    const int64_t *leaf_part;
};

}  // namespace rt

struct rtree {
    int device = 0;
    rtree_allocator_t alloc{};  // the device-memory hook (custom_alloc), else the default pool
    bool custom_alloc = false;
    int32_t fanout = 16;
    int32_t layout = RTREE_LAYOUT_SOA;
    int32_t sorted = 0;  // built with sort_children
    int32_t levels = 0;
    int64_t n = 0;
    int64_t nodes = 0;
    int64_t level_nodes[RT_MAX_LEVELS] = {};  // root level first
    int64_t level_base[RT_MAX_LEVELS] = {};
    float *mbr = nullptr;
    int4 *meta = nullptr;
    float4 *nbox = nullptr;
    int32_t *ids = nullptr;
    int64_t *leaf_part = nullptr;  // see TreeDev::leaf_part
    float root_mbr[4] = {0, 0, 0, 0};  // valid once root_ready (see tree_root_box)
    bool root_ready = true;
    rt::Mailbox *root_mb = nullptr;     // the build's posted root box until it is read
    int64_t bytes = 0;

    const rtree_allocator_t *allocator() const { return custom_alloc ? &alloc : nullptr; }

    rt::TreeDev view() const
    {
        rt::TreeDev v;
        v.mbr = mbr;
        v.meta = meta;
        v.nbox = nbox;
        v.ids = ids;
        v.leaf_base = levels ? (int32_t)level_base[levels - 1] : 0;
        v.nodes = (int32_t)nodes;
        v.levels = levels;
        v.fanout = fanout;
        v.layout = layout;
        v.sorted = sorted;
        v.leaf_part = leaf_part;
        return v;
    }
};

struct rtree_result {
    int device = 0;
    int64_t rows = 0;   // queries (select) or 0 (join)
    int64_t total = 0;  // ids (select) or pairs (join)
    int64_t *offsets = nullptr;
    int32_t *ids = nullptr;
    rtree_allocator_t alloc{};  // where offsets and ids came from (custom_alloc)
    bool custom_alloc = false;
    void *stream = nullptr;     // the stream the result was produced on
    rt::Mailbox *status = nullptr;  // device flags of work still in flight, posted at its end
};

namespace rt {

// ------------------------------------------------------- device primitives
// Closed-interval intersection of two boxes (x=xmin, y=ymin, z=xmax, w=ymax).
__device__ __forceinline__ bool meets(float4 a, float4 b)
{
    return a.x <= b.z && b.x <= a.z && a.y <= b.w && b.y <= a.w;
}

// c lies inside q (every rectangle inside c then meets q).
__device__ __forceinline__ bool inside(float4 c, float4 q)
{
    return q.x <= c.x && c.z <= q.z && q.y <= c.y && c.w <= q.w;
}

__device__ __forceinline__ float4 empty_box()
{
    return make_float4(__int_as_float(0x7f800000), __int_as_float(0x7f800000),
                       __int_as_float(0xff800000), __int_as_float(0xff800000));
}

__device__ __forceinline__ unsigned lanemask_lt()
{
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Child box j of node g.
__device__ __forceinline__ float4 load_entry(const float *__restrict__ mbr, int layout, int F,
                                             int64_t g, int j)
{
    if (layout == RTREE_LAYOUT_AOS)
        return __ldg(reinterpret_cast<const float4 *>(mbr) + g * F + j);
    if (layout == RTREE_LAYOUT_LOHI) {
        const float2 *p = reinterpret_cast<const float2 *>(mbr + g * 4 * F);
        const float2 lo = __ldg(p + j), hi = __ldg(p + F + j);
        return make_float4(lo.x, lo.y, hi.x, hi.y);
    }
    const float *b = mbr + g * 4 * F + j;
    return make_float4(__ldg(b), __ldg(b + F), __ldg(b + 2 * F), __ldg(b + 3 * F));
}

template <int F, int LAYOUT>
__device__ __forceinline__ float4 load_entry_t(const float *__restrict__ mbr, int64_t g, int j)
{
    if (LAYOUT == RTREE_LAYOUT_AOS)
        return __ldg(reinterpret_cast<const float4 *>(mbr) + g * F + j);
    if (LAYOUT == RTREE_LAYOUT_LOHI) {
        const float2 *p = reinterpret_cast<const float2 *>(mbr + g * 4 * F);
        const float2 lo = __ldg(p + j), hi = __ldg(p + F + j);
        return make_float4(lo.x, lo.y, hi.x, hi.y);
    }
    const float *b = mbr + g * 4 * F + j;
    return make_float4(__ldg(b), __ldg(b + F), __ldg(b + 2 * F), __ldg(b + 3 * F));
}

// ------------------------------------------------------ host-side helpers
// Exclusive scan; out has n+1 entries and out[n] is the total.
rtree_status scan_exclusive(const int32_t *in, int64_t *out, int64_t n, cudaStream_t s);
rtree_status scan_exclusive(const uint32_t *in, uint32_t *out, int64_t n, cudaStream_t s);
rtree_status scan_exclusive(const int64_t *in, int64_t *out, int64_t n, cudaStream_t s);

// Fills t->leaf_part (allocated here from the tree's allocator) from the
// leaf level's metadata, on stream s.
rtree_status compute_leaf_part(rtree *t, cudaStream_t s);

// Stable LSD radix sort of (key, value) pairs on key bits [bit_lo, bit_hi).
// Inputs are not modified; outputs must not alias inputs.
rtree_status radix_sort_pairs(const uint32_t *kin, const uint32_t *vin, uint32_t *kout,
                              uint32_t *vout, int64_t n, int bit_lo, int bit_hi, cudaStream_t s);

// Outputs of one select pass kernel (unused fields are null).
struct SelIO {
    int32_t *counts;          // COUNT: ids per query
    int32_t *counts_leaf;     // COUNT, optional: ids found one by one in leaves
    int32_t *counts_rng;      // COUNT, optional: whole subtrees taken
    const int64_t *offsets;   // SCATTER: CSR offsets of the ids
    int32_t *out;             // SCATTER: the ids, traversal order
    const int64_t *off_leaf;  // DESC: offsets of the leaf hits
    const int64_t *off_rng;   // DESC: offsets of the whole-subtree ranges
    int32_t *leaf_out;        // DESC: leaf hits
    int2 *rng_out;            // DESC: (lo, hi) ranges of the tree's id array
    // Work-queue mapping only: per-query write cursors (zeroed before the
    // pass), because several warps may emit results for one query.
    int32_t *cur_ids;         // SCATTER
    int32_t *cur_leaf;        // DESC
    int32_t *cur_rng;         // DESC
    // Buffer capacities (entries); writes at or past them are dropped.  Only
    // the graph-captured plan sizes buffers before knowing the totals.
    int64_t out_cap;
    int64_t leaf_cap;
    int64_t rng_cap;
    // Optional traversal order: work item k is query order[k] (a permutation
    // of [0, Q)); results stay indexed by the query.
    const uint32_t *order;
};

// Caller-owned buffers for a select enqueued without host synchronization
// (q = number of queries): per-query counts [q], offsets [q+1], the leaf-hit,
// range and id outputs with their capacities, work-queue cursors [2q],
// flags [2] (select, sort) and work counters [2].  After the stream finishes,
// off[q], off_leaf[q] and off_rng[q] hold the totals; a total above its
// capacity means the outputs are incomplete.
struct SelectBuffers {
    int32_t *cnt, *cnt_leaf, *cnt_rng;
    int64_t *off, *off_leaf, *off_rng;
    int32_t *leaf;
    int64_t leaf_cap;
    int2 *rng;
    int64_t rng_cap;
    int32_t *ids;
    int64_t ids_cap;
    int32_t *cursors;
    int32_t *flags;
    unsigned long long *ctr;
    unsigned long long *wq_ctl;  // 3 words, work-queue mapping
    unsigned long long *wq_items;
    long long wq_cap;
};

// Enqueues a sorted range select into `b` on stream s (capturable in a CUDA
// graph: no host synchronization, no pageable copies).
rtree_status select_enqueue(const rtree *t, const float4 *queries, int64_t q, int mapping,
                            const SelectBuffers &b, cudaStream_t s);

// Where the ids of segment i come from: leaf[off_leaf[i] .. off_leaf[i+1])
// followed by tree_ids[lo .. hi) for every (lo, hi) in
// rng[off_rng[i] .. off_rng[i+1]).  rng may be null (no ranges).
struct SortSources {
    const int32_t *leaf;
    const int64_t *off_leaf;  // segment i's leaf hits start at off_leaf[i] and end at
    const int32_t *leaf_len;  // off_leaf[i] + leaf_len[i] if leaf_len is set, else off_leaf[i+1]
    const int2 *rng;
    const int64_t *off_rng;
    const int32_t *tree_ids;
    int64_t leaf_cap;  // 0: unchecked; else segments reaching past are skipped
    int64_t rng_cap;
};

// Writes segment i's ids, sorted ascending (signed), to
// out[off[i] .. off[i+1]).  out may be the leaf array itself (in place).
// Enqueues work only (no host synchronization); `total` must bound the sum
// of the segments' lengths (it sizes the scratch), and segments ending past
// out_cap (default: total) in `out` are skipped.  Offsets may be absolute
// positions in a larger `out`, so a run of segments can be sorted on its
// own.  Device-side capacity problems set bits in *flags.
rtree_status segmented_sort_gather(int32_t *out, const int64_t *off, int64_t nseg, int64_t total,
                                   const SortSources &src, cudaStream_t s, int32_t *flags,
                                   int64_t out_cap = -1);

// Sorts every segment ids[offsets[i] .. offsets[i+1]) ascending, in place.
rtree_status segmented_sort(int32_t *ids, const int64_t *offsets, int64_t nseg, int64_t total,
                            cudaStream_t s);

// Builds the tree from device rectangles (float4 rows) and device ids (or
// NULL); sort_children orders every node's entries by ascending lx.
rtree_status build_tree(const float4 *rects, const int32_t *ids, int64_t n, int fanout, int layout,
                        bool sort_children, cudaStream_t s, rtree *t);

// ------------------------------------------------------------- mailboxes
// Page-locked host words mapped into the device, plus an event: a kernel
// stores small results there and the host reads them once the event has
// completed, so such reads never queue behind large copies on a copy engine
// (mailbox.cu).  Mailboxes come from a per-device pool.
constexpr int kMailboxWords = 256;
struct Mailbox {
    uint32_t *h = nullptr;  // host view
    uint32_t *d = nullptr;  // device view
    cudaEvent_t ev = nullptr;
    int device = -1;
};
// Up to 8 device sources: words[i] 32-bit words from src[i] go to word at[i].
struct PostList {
    const void *src[8];
    int words[8];
    int at[8];
    int n;
};
// Enqueues the copy kernel only: words go to dst, a device view of mapped
// host memory (usable inside a graph capture).
rtree_status post_words(const PostList &l, uint32_t *dst, cudaStream_t s);
rtree_status mailbox_get(Mailbox *m);
void mailbox_put(Mailbox *m);
// Hands m back while a kernel may still post into it: it is reused only
// after its event has completed.
void mailbox_put_deferred(Mailbox *m);
// Enqueues the copy kernel on s, then records m.ev on s.
rtree_status mailbox_post(const Mailbox &m, const PostList &l, cudaStream_t s);
rtree_status mailbox_wait(const Mailbox &m);
// Posts two device words (flags) to a new mailbox of `res`, behind the work
// enqueued on s so far; rtree_result_wait reads them (word 0 bit 4: a
// bounded device wait ran out; any other bit: a consistency check failed).
rtree_status post_result_status(const int32_t *flags, cudaStream_t s, rtree_result *res);
// Reads nwords <= kMailboxWords device words listed in l on the host (one
// kernel stores them into a mailbox; the host waits for its event).
rtree_status read_words(const PostList &l, cudaStream_t s, uint32_t *out, int nwords);
struct MailboxRef {
    Mailbox m;
    MailboxRef() = default;
    MailboxRef(const MailboxRef &) = delete;
    MailboxRef &operator=(const MailboxRef &) = delete;
    ~MailboxRef() { mailbox_put(&m); }
};

// Range select whose result is copied, chunk by chunk, to host memory while
// later chunks are still being selected (see rtree_range_select_host).  On
// success *pending is the call still in flight (its copies run on a stream
// of its own), or null when nothing is left to wait for; finish it with
// range_select_host_finish.
rtree_status range_select_host_begin(const rtree *t, const float4 *queries, int64_t q, bool sorted,
                                     int mapping, int order, cudaStream_t s, int64_t *h_off,
                                     int32_t *h_ids, int64_t capacity, int64_t *h_total,
                                     rtree_pending **pending);
// Waits for the copies, checks the device flags, frees everything of p.
rtree_status range_select_host_finish(rtree_pending *p);

// Range select for device queries (float4 rows); order is RTREE_ORDER_*.
rtree_status range_select(const rtree *t, const float4 *queries, int64_t q, bool sorted,
                          int mapping, int order, cudaStream_t s, rtree_result *res);

// order[0 .. Q) = the queries' indices in Hilbert-curve order of their centres
// (scaled into the tree's bounding box); ties keep index order.
rtree_status hilbert_order(const rtree *t, const float4 *queries, int64_t Q, uint32_t *order,
                           cudaStream_t s);

// One pass of the range-select kernel on caller-provided buffers: the count
// pass when counts is non-null, else the scatter pass.  ctr (one zeroed
// work counter) and flags (zeroed) are caller-provided; nothing is allocated.
rtree_status select_pass(const rtree *t, const float4 *queries, int64_t q, int32_t *counts,
                         const int64_t *offsets, int32_t *out, unsigned long long *ctr,
                         int32_t *flags, cudaStream_t s);

// Traversal statistics of one count pass (see rtree_range_select_stats).
rtree_status select_stats(const rtree *t, const float4 *queries, int64_t q, cudaStream_t s,
                          int64_t out[8]);

// R-tree join of two trees on the same device; prune selects the sorted-node
// kernel for equal-height pairs (both trees must have sorted children).
// stats (optional, 8 zeroed words) receives node pairs tested at equal
// internal heights [0], with only R descending [1], only S descending [2],
// at the leaves [3], and the pairs found [4].
rtree_status tree_join(const rtree *r, const rtree *s_tree, bool prune, cudaStream_t s,
                       rtree_result *res, int64_t *stats = nullptr);
// The same join with the node pairs pulled by a persistent grid from a device
// work queue (count pass, one host read of the total, scatter pass, sort);
// returns with the scatter pass and sort in flight (the result's status
// mailbox gets their flags).  *redo_by_levels is set (and nothing produced)
// when the traversal needs more node pairs than the queue holds.
rtree_status tree_join_queue(const rtree *r, const rtree *s_tree, bool prune, cudaStream_t s,
                             rtree_result *res, bool *redo_by_levels);

}  // namespace rt

// A host-result select still in flight (rtree_range_select_host_async): its
// result copies run on `cs`; `ids` and `off` are the device buffers they
// read, freed on `cs` when the call is finished.
struct rtree_pending {
    int device = 0;
    rtree_allocator_t alloc{};  // the tree's device-memory hook (custom_alloc)
    bool custom_alloc = false;
    cudaStream_t cs = nullptr;
    cudaEvent_t ev[33] = {};
    rt::Mailbox flags;  // the device flags, posted behind the last chunk
    int32_t *ids = nullptr;
    int64_t *off = nullptr;
};

