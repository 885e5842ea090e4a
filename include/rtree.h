/*
 * rtree.h -- C ABI of the GB300 (sm_103a) R-tree library (librtree.so).
 *
 * Operations (arXiv 2309.16913, "SIMD-ified R-tree Query Processing and
 * Optimization"):
 *   - range select (Section 3): for each query rectangle q, the ids of all
 *     indexed rectangles r with r INTERSECTS q;
 *   - R-tree join (Section 4, after Brinkhoff, Kriegel and Seeger 1993): all
 *     (r_id, s_id) with R_r INTERSECTS S_s, found by traversing both trees
 *     top-down in step.
 * INTERSECTS is the closed-interval test on both axes:
 *     a.xmin <= b.xmax && b.xmin <= a.xmax && a.ymin <= b.ymax && b.ymin <= a.ymax
 * so rectangles that only touch intersect.  All tests are float32
 * comparisons; nothing is rounded, so results are exact.
 *
 * Data layout.  A rectangle is four float32 values [xmin, ymin, xmax, ymax];
 * an array of n rectangles is n*4 contiguous floats (16 bytes per row).  Ids
 * are int32.  Pointers passed in may be device pointers or host pointers
 * (pageable or pinned); the library tells them apart and copies host inputs
 * to the device on the given stream (device inputs that are not 16-byte
 * aligned are copied too).
 *
 * Streams.  `stream` is a cudaStream_t passed as void* (NULL = legacy default
 * stream).  rtree_build and rtree_range_select are stream-ordered: they
 * return once their work is enqueued on `stream`, after the one host read
 * each needs (the build's input check, the select's result sizes and total),
 * and their outputs may be used by later work on that stream, or by the
 * host once the stream has been synchronized (rtree_result_wait does that
 * and also reports device-side errors of the work still in flight).  The
 * other calls return only after their device work on `stream` has finished.
 *
 * Device memory.  A tree is built with an optional allocator
 * (rtree_allocator_t); every device buffer the library allocates for that
 * tree -- the tree itself, the scratch of calls on it, and their results --
 * is taken from it and given back to it.  NULL selects cudaMallocAsync and
 * cudaFreeAsync on the call's stream (the device's default memory pool).
 *
 * Errors.  Every call returns an rtree_status; on failure no output is
 * produced (output handles are set to NULL) and rtree_last_error() describes
 * the failure (per host thread).  No call aborts the process.
 *
 * Thread safety.  Distinct trees and results may be used from different host
 * threads.  A tree may be queried by several threads at once; rtree_free must
 * not race with queries on the same tree.
 */
#ifndef RTREE_H
#define RTREE_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define RTREE_API __attribute__((visibility("default")))
#else
#define RTREE_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum rtree_status {
    RTREE_OK = 0,
    RTREE_EINVAL = 1,    /* bad argument, NaN coordinate or xmin > xmax / ymin > ymax */
    RTREE_ENOMEM = 2,    /* a device or host allocation failed */
    RTREE_ECUDA = 3,     /* a CUDA runtime call failed (message has the CUDA error) */
    RTREE_ETIMEOUT = 4,  /* a bounded device-side wait gave up */
    RTREE_EOVERFLOW = 5, /* a size exceeds a fixed capacity (message says which) */
    RTREE_EINTERNAL = 6, /* a device-side consistency check failed */
    RTREE_EIO = 7        /* a file could not be opened, read or written (rtree_save/load) */
} rtree_status;

/* Node layouts (Section 2.3).  SOA is layout D1: per node, the F lower-x
 * values, then F lower-y, F upper-x, F upper-y.  AOS is layout D0: per node,
 * F entries of 16 bytes each (xmin, ymin, xmax, ymax).  LOHI is layout D2:
 * per node, the F lower-left points (xmin, ymin), then the F upper-right
 * points (xmax, ymax). */
enum { RTREE_LAYOUT_SOA = 0, RTREE_LAYOUT_AOS = 1, RTREE_LAYOUT_LOHI = 2 };

/* How range-select work is spread over the GPU. */
enum {
    RTREE_MAP_AUTO = 0,           /* library choice (currently WARP_PER_QUERY) */
    RTREE_MAP_WARP_PER_QUERY = 1, /* one warp walks one query's whole subtree */
    RTREE_MAP_WORK_QUEUE = 2      /* persistent warps share (query, node) items through a
                                     device work queue, so large queries are split */
};

/* Build configuration.  A zeroed struct (or NULL) selects the defaults. */
typedef struct rtree_config {
    int32_t fanout;        /* maximum entries per node F: 4, 8, 16, 32, 64 or 128; 0 -> 16 */
    int32_t layout;        /* RTREE_LAYOUT_*; default SOA */
    int32_t sort_children; /* 1: every node's entries ascend by xmin, ties in packing order
                              (the node order the join prunings of Section 4.2 assume);
                              0 (default): packing order */
    int32_t reserved[5];
} rtree_config_t;

/* Range-select options.  NULL selects the defaults. */
/* Traversal order of a batch (results are identical either way). */
enum {
    RTREE_ORDER_INPUT = 0,   /* queries are taken in the order given */
    RTREE_ORDER_HILBERT = 1  /* taken in Hilbert-curve order of their centres, so that warps
                                running together visit nearby nodes (an addition: the paper
                                has no such step; it carries the latency-hiding aim of its
                                prefetching, O2 in Section 3, over to the L2 cache) */
};

typedef struct rtree_select_opts {
    int32_t unsorted; /* 0 (default): ids of each query ascending; 1: traversal order */
    int32_t mapping;  /* RTREE_MAP_* */
    int32_t order;    /* RTREE_ORDER_*; rtree_range_select only (plans take INPUT) */
    int32_t reserved[5];
} rtree_select_opts_t;

typedef struct rtree rtree_t;               /* opaque; owns device memory */
typedef struct rtree_result rtree_result_t; /* opaque; owns device memory */
typedef struct rtree_pending rtree_pending_t; /* opaque; a host-result select in flight */

typedef struct rtree_info {
    int64_t n;            /* indexed rectangles */
    int64_t nodes;        /* nodes over all levels */
    int32_t levels;       /* tree height; 0 for an empty tree, 1 if the root is a leaf */
    int32_t fanout;       /* F */
    int32_t layout;       /* RTREE_LAYOUT_* */
    int32_t device;       /* CUDA device holding the tree */
    int64_t device_bytes; /* device memory held by the tree */
    float root_mbr[4];    /* bounding box of all rectangles (empty tree: +inf,+inf,-inf,-inf) */
    int32_t sort_children; /* as built (rtree_config_t) */
    int32_t reserved[3];
} rtree_info_t;

/*
 * Device-memory hook.  alloc(bytes, stream, ctx) returns device memory of
 * the tree's device usable by work enqueued on `stream` after the call (or
 * NULL on failure, which the library reports as RTREE_ENOMEM); free(p,
 * stream, ctx) gives it back, usable again once the work enqueued on
 * `stream` before the call has finished.  `stream` is a cudaStream_t as void*
 * (NULL = legacy default stream).  The functions may be called from any host
 * thread that calls into the library with this tree (serving workers
 * included), and `ctx` must stay valid until the tree and all its results
 * are freed.  The library copies the struct at rtree_build.
 */
typedef struct rtree_allocator {
    void *(*alloc)(size_t bytes, void *stream, void *ctx);
    void (*free)(void *p, void *stream, void *ctx);
    void *ctx;
} rtree_allocator_t;

/*
 * rtree_build -- bulk-load an R-tree with Sort-Tile-Recursive packing.
 *
 * The paper indexes a main-memory R-tree whose node holds up to F entries
 * (MBR, ptr) plus depth and count (Section 2.3) but does not say how it is
 * built.  This call packs it bottom-up with STR: at each level the m items
 * are sorted by the float32 centre key xmin+xmax (ties by item index), cut
 * into S = ceil(sqrt(ceil(m/F))) slabs of S*F items, each slab sorted by
 * ymin+ymax (ties by item index), and runs of F items become nodes; this is
 * repeated on the node MBRs until one node (the root) remains.  A centre key
 * that is NaN (-inf + inf) counts as 0 and -0 as +0.  With
 * cfg->sort_children the entries of every node are then reordered by
 * ascending xmin (stable; -0 equals +0), which changes neither the nodes'
 * contents nor any query result.
 *
 * rects: n*4 floats, ids: n int32 (NULL -> ids 0..n-1); host or device.
 * n = 0 builds a valid empty tree.  n must be < 2^31.
 * The inputs are copied; the caller keeps ownership and may free them once
 * the call returns.  alloc: the tree's device-memory hook (NULL: the default
 * pool).  *out receives the tree (free with rtree_free).  The call returns
 * once the inputs have been checked on the device (one host read) and the
 * packing is enqueued on `stream`; work enqueued on `stream` afterwards may
 * use the tree.
 * Errors: RTREE_EINVAL for a NaN coordinate, xmin > xmax or ymin > ymax in
 * any row, an unsupported fanout/layout, an allocator with a NULL function,
 * or NULL out; RTREE_ENOMEM.
 */
RTREE_API rtree_status rtree_build(const float *rects, const int32_t *ids, int64_t n,
                                   const rtree_config_t *cfg, const rtree_allocator_t *alloc,
                                   void *stream, rtree_t **out);

/* Releases the tree's device memory.  NULL is ignored. */
RTREE_API void rtree_free(rtree_t *tree);

/*
 * Releases the tree's device memory in the order of `stream`: work already
 * enqueued on that stream may still read the tree, and work on other
 * streams is not waited for (rtree_free may wait for the whole device).
 * The handle is invalid on return.  NULL is ignored.
 */
RTREE_API void rtree_free_async(rtree_t *tree, void *stream);

/* Fills *info.  Errors: RTREE_EINVAL for NULL arguments. */
RTREE_API rtree_status rtree_get_info(const rtree_t *tree, rtree_info_t *info);

/*
 * rtree_export -- copy the tree to caller-owned host arrays, level by level
 * from the root.  Within a level, nodes come in the order their parents list
 * them; entries keep their packing order.
 *   level_nodes[levels]       nodes per level, root level first
 *   counts[nodes]             entries per node
 *   mbrs[nodes * F * 4]       entry MBRs; unused slots are (+inf,+inf,-inf,-inf)
 *   leaf_ids[n]               ids of the leaf entries, leaves in export order
 * Used to compare the device-built tree with an independently built one.
 */
RTREE_API rtree_status rtree_export(const rtree_t *tree, int64_t *level_nodes, int32_t *counts,
                          float *mbrs, int32_t *leaf_ids, void *stream);

/*
 * rtree_range_select -- batched range select (Section 3).
 *
 * For every query i (queries: q*4 floats, host or device) returns the ids of
 * all indexed rectangles that intersect it, as CSR: offsets[q+1] (int64) and
 * ids[total] (int32), query i owning ids[offsets[i] .. offsets[i+1]).  Ids of
 * one query are ascending unless opts->unsorted.  Queries may be degenerate
 * (points, lines) or infinite.  A query is used as given: the predicate is
 * evaluated literally, so a query with a NaN coordinate matches nothing and
 * an inverted query (xmin > xmax) matches whatever the four comparisons
 * accept; neither is an error.
 *
 * The traversal is the paper's vectorized select recast for a warp: a
 * query's node is tested against all F child MBRs at once (one lane per
 * child), qualifying children are compacted with a ballot into a per-warp
 * stack (the queue insertion of step 4), and a child whose MBR lies inside
 * the query contributes its whole subtree without further tests.  Output is
 * written in two passes (count, exclusive scan, scatter) and then sorted per
 * query.
 *
 * *out receives the result (free with rtree_result_free), resident on the
 * tree's device, its buffers from the tree's allocator.  Stream order: the
 * call reads two small values on the host (the sizes of the traversal's
 * outputs, then the result's total) and returns while the last pass and the
 * per-query sort still run on `stream`; rtree_result_total is valid on
 * return, the offsets and ids once `stream` has reached the end of the call
 * (rtree_result_wait, rtree_result_copy_to_host, or a stream
 * synchronization).  Errors found on the device after the return (internal
 * consistency checks, a work-queue wait that ran out) are reported by
 * rtree_result_wait and rtree_result_copy_to_host.
 * Errors: RTREE_EINVAL (NULL tree/out, q < 0), RTREE_ENOMEM,
 * RTREE_EINTERNAL, RTREE_ETIMEOUT, RTREE_ECUDA.
 */
RTREE_API rtree_status rtree_range_select(const rtree_t *tree, const float *queries, int64_t q,
                                const rtree_select_opts_t *opts, void *stream,
                                rtree_result_t **out);

/*
 * Plans: batched range select captured in CUDA graphs (the persistent
 * batched form of the select).
 *
 * A plan owns every device buffer a sorted select needs, sized for at most
 * max_queries queries and max_ids result ids per batch (and, for the
 * warp-per-query mapping, 2*max_ids + 4*F*max_queries leaf-hit slots: its
 * sizing pass stops above the leaves and reserves F slots per leaf a query
 * meets), and records the whole
 * device pipeline of rtree_range_select (sizing pass, scans, descriptor pass,
 * segmented sort, store of the totals) as one CUDA graph per batch-size bucket
 * (powers of two from 256 up to max_queries); a batch is padded to its bucket
 * with NaN queries, which match nothing.  Unlike rtree_range_select, a run
 * needs no host round trip between kernels, so small batches cost one graph
 * launch.  opts->mapping selects warp-per-query or the work queue; plans
 * always sort.  The tree must outlive the plan.
 *
 * rtree_plan_run copies q <= max_queries queries (host or device) into the
 * plan, runs the batch on `stream` and returns when it has finished; *total
 * receives the number of ids.  The results are rtree_plan_offsets (device
 * int64[q+1]) and rtree_plan_ids (device int32[total]), valid until the next
 * run.  If the batch needs more than max_ids ids, the run returns
 * RTREE_EOVERFLOW with *total set to the size needed and incomplete outputs.
 * The first run of each bucket records its graph (it must not itself be
 * inside a stream capture).  A plan is used by one host thread at a time.
 * The plan's buffers come from the tree's allocator; scratch that the
 * recorded pipeline allocates is graph memory, owned by the graphs.
 */
typedef struct rtree_plan rtree_plan_t;
RTREE_API rtree_status rtree_plan_create(const rtree_t *tree, int64_t max_queries, int64_t max_ids,
                                         const rtree_select_opts_t *opts, rtree_plan_t **out);
RTREE_API rtree_status rtree_plan_run(rtree_plan_t *plan, const float *queries, int64_t q,
                                      void *stream, int64_t *total);
RTREE_API const int64_t *rtree_plan_offsets(const rtree_plan_t *plan);
RTREE_API const int32_t *rtree_plan_ids(const rtree_plan_t *plan);
RTREE_API void rtree_plan_free(rtree_plan_t *plan);

/*
 * Serving: a request loop over a device-resident index with continuous
 * batching.
 *
 * rtree_server_start launches `workers` host threads, each with its own CUDA
 * stream and plan (max_batch_queries queries, max_batch_ids ids), so several
 * batches run on the device at once.  Requests wait in a queue; a free worker
 * takes the waiting requests in arrival order while the batch's queries fit
 * its plan and their expected result (a running mean of ids per query) fits
 * 80% of the plan's id capacity -- admission by output memory.  A batch that
 * still overflows is split in two and rerun; a single request too large for
 * a plan is answered by rtree_range_select.  Requests arriving while batches
 * are in flight join the next batch a worker forms.
 *
 * Request kinds: RTREE_REQ_SELECT (range select of q query rectangles) and
 * RTREE_REQ_PROBE_JOIN (join of q probe rectangles with the index).  Both
 * replies are CSR in host memory: row i lists, ascending, the ids of indexed
 * rectangles meeting query/probe i -- for a probe join, the pairs (i, id) in
 * lexicographic order.  A reply's latency runs from submission until its
 * results are in host memory.  submit and wait may be called from any host
 * threads; the tree must outlive the server.
 */
enum { RTREE_REQ_SELECT = 0, RTREE_REQ_PROBE_JOIN = 1 };

typedef struct rtree_server_config {
    int32_t workers;           /* concurrent batches (streams); 0 -> 2 */
    int32_t max_batch_queries; /* per batch; 0 -> 16384 */
    int64_t max_batch_ids;     /* output ids per batch (the memory budget); 0 -> 16M */
    int32_t mapping;           /* RTREE_MAP_* for the batches */
    int32_t reserved[5];
} rtree_server_config_t;

typedef struct rtree_reply {
    int32_t kind;
    int32_t reserved;
    int64_t rows;       /* queries or probes in the request */
    int64_t total;      /* ids */
    int64_t *offsets;   /* host, rows+1 */
    int32_t *ids;       /* host, total */
    double latency_us;  /* submission to results in host memory */
} rtree_reply_t;

typedef struct rtree_server_stats {
    int64_t completed;     /* requests answered since start/reset */
    int64_t batches;
    int64_t batch_queries; /* queries run in batches */
    int64_t splits;        /* batches split after an overflow */
    int64_t fallbacks;     /* requests answered by rtree_range_select */
    int64_t pending;       /* requests waiting now */
    double p50_us, p99_us, max_us;
    double elapsed_s;      /* since start/reset */
} rtree_server_stats_t;

typedef struct rtree_server rtree_server_t;
RTREE_API rtree_status rtree_server_start(const rtree_t *tree, const rtree_server_config_t *cfg,
                                          rtree_server_t **out);
/* Copies the q rectangles (host memory); *ticket identifies the reply. */
RTREE_API rtree_status rtree_server_submit(rtree_server_t *server, const float *rects, int64_t q,
                                           int32_t kind, uint64_t *ticket);
/* Waits for a reply (timeout_us < 0: no limit; RTREE_ETIMEOUT otherwise).
 * Fills *reply; free its arrays with rtree_reply_free.  Each ticket's reply
 * can be taken once. */
RTREE_API rtree_status rtree_server_wait(rtree_server_t *server, uint64_t ticket, int64_t timeout_us,
                                         rtree_reply_t *reply);
RTREE_API void rtree_reply_free(rtree_reply_t *reply);
RTREE_API rtree_status rtree_server_get_stats(rtree_server_t *server, rtree_server_stats_t *stats);
RTREE_API rtree_status rtree_server_reset_stats(rtree_server_t *server);
/* Answers every request already submitted, then stops the workers. */
RTREE_API void rtree_server_stop(rtree_server_t *server);

/*
 * rtree_range_select_noalloc -- range select that allocates no device memory.
 * (An addition of this library; the paper has no counterpart.)
 *
 * For callers that cannot allocate once running: an application that has
 * reserved all of the GPU's memory for its own pool, or a request loop that
 * must neither block in nor fail from the CUDA allocator mid-request.  The
 * caller passes every buffer; the library's temporary storage lives in one
 * fixed device array (about 256 KiB) compiled into the library, which each
 * GPU that loads the library holds until the process exits.
 *
 * queries: q*4 floats in device memory, 16-byte aligned, q <= 65536
 *          (larger q: RTREE_EOVERFLOW; split the batch).
 * offsets: device int64[q+1], receives the CSR offsets.
 * ids:     device int32[capacity], receives the ids of query i at
 *          ids[offsets[i] .. offsets[i+1]) in traversal order (not sorted;
 *          the same order rtree_range_select gives with opts->unsorted = 1).
 * total:   host int64, receives the number of ids.  If it exceeds capacity
 *          the call returns RTREE_EOVERFLOW with offsets and *total valid
 *          and ids unwritten, so the caller can retry with a larger buffer.
 * The first call on a device looks up the array's device address (a
 * runtime call, no allocation); make that first call before any stream
 * capture.  Calls share the array: calls whose device work overlaps (other
 * streams or host threads) race on it and must be serialized by the caller.
 * Returns when the results are ready on `stream`.
 */
RTREE_API rtree_status rtree_range_select_noalloc(const rtree_t *tree, const float *queries, int64_t q,
                                                  int64_t *offsets, int32_t *ids, int64_t capacity,
                                                  int64_t *total, void *stream);

/*
 * rtree_range_select_stats -- traversal counters of one count pass over the
 * same queries (no output is produced).  stats[0..5] receive: queries, nodes
 * visited, leaf nodes visited, children taken whole because their MBR lies
 * inside the query, ids found, ids found through such whole children;
 * stats[6..7] are 0.  Used to turn kernel times into bytes per second.
 */
RTREE_API rtree_status rtree_range_select_stats(const rtree_t *tree, const float *queries, int64_t q,
                                                void *stream, int64_t stats[8]);

/*
 * rtree_join -- R-tree join (Section 4).
 *
 * Returns every pair (r_id, s_id) of rectangles from tree r and tree s that
 * intersect, sorted lexicographically, as ids[2*total] (int32 pairs).  Both
 * trees are walked top-down together from their roots, following entry pairs
 * whose MBRs intersect; where the heights differ, only the taller tree
 * descends until the heights match.  Each node pair is tested by one warp:
 * every outer child's MBR is broadcast to all lanes and compared with the
 * inner children held one per lane (the one-to-many comparison of Section
 * 4.1).  The trees may have different fanouts and layouts but must be on the
 * same device.  A join returns at most 2^31-1 pairs (the pair sort is a
 * 32-bit-indexed radix sort); a larger result is RTREE_EOVERFLOW.
 * Errors: RTREE_EINVAL, RTREE_ENOMEM, RTREE_ECUDA, RTREE_EOVERFLOW.
 */
/*
 * rtree_range_select_host -- rtree_range_select with the result written to
 * caller-owned host memory, the copy overlapped with the work.  One count
 * pass over the batch fixes every query's offset (written to `offsets`
 * first); the batch is then cut into chunks of about equal id counts (about
 * 128M ids each, at most 32), and
 * while the second pass and sort of one chunk run on `stream`, the ids of
 * the chunk before are copied to `ids` on a second stream.  Same ids, order
 * and options as rtree_range_select.
 * queries: q*4 floats, host or device.  offsets: host int64[q+1].  ids: host
 * int32[capacity]; page-locked memory lets the copies overlap the work.
 * *total receives the number of ids.  If it exceeds capacity the call
 * returns RTREE_EOVERFLOW with offsets and *total written and ids untouched
 * (resize and call again).  Errors otherwise as rtree_range_select.
 */
RTREE_API rtree_status rtree_range_select_host(const rtree_t *tree, const float *queries, int64_t q,
                                               const rtree_select_opts_t *opts, void *stream,
                                               int64_t *offsets, int32_t *ids, int64_t capacity,
                                               int64_t *total);

/*
 * rtree_range_select_host_async -- rtree_range_select_host that returns
 * once all of its work and copies are enqueued, so that the caller can start
 * the next call (or build the next tree) while this call's results are
 * still travelling to host memory.  The count pass still runs before the
 * return: *total is valid on return (and RTREE_EOVERFLOW is reported then,
 * as by rtree_range_select_host).  On RTREE_OK, *pending is the call in
 * flight, or NULL if it completed already (an empty result); offsets and ids
 * are valid only after rtree_pending_wait(*pending) returns RTREE_OK.  The
 * tree, the queries and `stream` may be reused or freed (rtree_free_async on
 * `stream`) right away.  Small results the host needs during the call (the
 * total, chunk bounds, error flags) travel through page-locked mapped
 * memory written by a kernel, not through a copy, so they never wait behind
 * the copies of earlier calls.
 */
RTREE_API rtree_status rtree_range_select_host_async(const rtree_t *tree, const float *queries, int64_t q,
                                                     const rtree_select_opts_t *opts, void *stream,
                                                     int64_t *offsets, int32_t *ids, int64_t capacity,
                                                     int64_t *total, rtree_pending_t **pending);

/*
 * Waits until a pending host-result select has written its offsets and ids,
 * releases it and returns its status (device-side errors of the call, e.g.
 * RTREE_ETIMEOUT, are reported here).  NULL returns RTREE_OK.  Every pending
 * call must be waited for exactly once.
 */
RTREE_API rtree_status rtree_pending_wait(rtree_pending_t *pending);

RTREE_API rtree_status rtree_join(const rtree_t *r, const rtree_t *s, void *stream, rtree_result_t **out);

/*
 * rtree_join_ex -- rtree_join with options: the sorted-node prunings of
 * Section 4.2 for trees built with sort_children.
 *
 * On equal-height node pairs the outer node's children are taken 32 at a
 * time, one per lane, in ascending xmin.  O3: an outer child whose xmin lies
 * right of every inner child (right of the inner node's MBR) fails for all
 * of them, and so does every later outer child, so the rest of the outer
 * node is skipped; an outer child that misses the inner node's MBR is also
 * not paired (the search-space restriction of Brinkhoff, Kriegel and Seeger
 * 1993).  O4/O5: each remaining outer child finds, with the batched search
 * of the many-to-many comparison (log2(P)+1 rounds over the inner children's
 * xmin, P = inner count rounded up to a power of two), the number f of inner
 * children that start left of its xmax; only those f are tested, the pairs
 * of all 32 lanes packed densely onto the warp.  The result is identical to
 * rtree_join's.
 *
 * opts NULL -> RTREE_PRUNE_AUTO, RTREE_JOIN_AUTO.  Errors: as rtree_join, and
 * RTREE_EINVAL for RTREE_PRUNE_ON when either tree was built without
 * sort_children, or an unknown option; RTREE_ETIMEOUT if a bounded
 * work-queue wait ran out (RTREE_JOIN_QUEUE).
 */
enum { RTREE_PRUNE_AUTO = 0, /* prune when both trees have sorted children */
       RTREE_PRUNE_OFF = 1,  /* plain one-to-many comparison */
       RTREE_PRUNE_ON = 2 };
/* How the node pairs of the traversal are scheduled (same pairs either way). */
enum { RTREE_JOIN_AUTO = 0,   /* the library's choice (RTREE_JOIN_LEVELS: faster on the joins measured;
                                 the queue's counters see one atomic per node pair or more, while a
                                 level costs one launch and one host read) */
       RTREE_JOIN_LEVELS = 1, /* one launch per tree level over that level's node pairs, the pairs
                                 found on one level being the next level's work (count, scan and
                                 scatter per level; the call returns when its work has finished) */
       RTREE_JOIN_QUEUE = 2 };/* a persistent grid pulls node pairs from a device work queue and
                                 publishes the qualifying child pairs to it; a count pass, one host
                                 read of the total, a scatter pass and the pair sort.  The call
                                 returns with the scatter pass and sort in flight on `stream`
                                 (rtree_result_wait).  If the traversal needs more node pairs
                                 than the queue holds (8 per node of the two trees, at least
                                 4M), the join is redone by levels */
typedef struct rtree_join_opts {
    int32_t prune;     /* RTREE_PRUNE_* */
    int32_t traversal; /* RTREE_JOIN_* */
    int32_t reserved[6];
} rtree_join_opts_t;
RTREE_API rtree_status rtree_join_ex(const rtree_t *r, const rtree_t *s, const rtree_join_opts_t *opts,
                                     void *stream, rtree_result_t **out);

/*
 * rtree_join_stats -- runs rtree_join_ex and, instead of the pairs, returns
 * the traversal's counters: stats[0] node pairs tested with both trees at
 * the same internal level, [1] node pairs where only r descends (r taller),
 * [2] where only s descends, [3] leaf node pairs, [4] pairs found; [5..7]
 * are 0.  Used to turn the join kernels' times into bytes and tests per
 * second.  Errors: as rtree_join_ex, and RTREE_EINVAL for NULL stats.
 */
RTREE_API rtree_status rtree_join_stats(const rtree_t *r, const rtree_t *s, const rtree_join_opts_t *opts,
                                        void *stream, int64_t stats[8]);

/* Result accessors.  Pointers are device pointers owned by the result. */
RTREE_API int64_t rtree_result_total(const rtree_result_t *res);         /* ids (select) or pairs (join) */
RTREE_API int64_t rtree_result_rows(const rtree_result_t *res);          /* q for select, 0 for join */
RTREE_API const int64_t *rtree_result_offsets(const rtree_result_t *res); /* q+1 entries, NULL for join */
RTREE_API const int32_t *rtree_result_ids(const rtree_result_t *res);     /* total (select) or 2*total (join) */

/* Copies a result to caller-owned host arrays (offsets may be NULL; sized as
 * the accessors above say), on `stream` after the work that produced the
 * result (whichever stream that ran on), and returns once the copies are
 * done, with the device-side status of that work (see rtree_result_wait). */
RTREE_API rtree_status rtree_result_copy_to_host(const rtree_result_t *res, int64_t *offsets,
                                       int32_t *ids, void *stream);

/* Waits until the device work that produces the result has finished and
 * returns its status: RTREE_OK, RTREE_EINTERNAL if a device-side consistency
 * check failed, RTREE_ETIMEOUT if a bounded work-queue wait ran out (the
 * result is then incomplete).  Results of calls that return only after their
 * work has finished (a join by levels) return RTREE_OK at once. */
RTREE_API rtree_status rtree_result_wait(const rtree_result_t *res);

/* Releases a result (after the whole device has finished; the buffers go
 * back to the allocator they came from).  NULL is ignored. */
RTREE_API void rtree_result_free(rtree_result_t *res);

/* Releases a result in the order of `stream`: work already enqueued on that
 * stream (the producing call's, if it ran there) may still read it; work on
 * other streams is not waited for.  The handle is invalid on return.  NULL
 * is ignored. */
RTREE_API void rtree_result_free_async(rtree_result_t *res, void *stream);

/* Description of the last failure on this host thread ("" if none). */
RTREE_API const char *rtree_last_error(void);

/* Library version string. */
RTREE_API const char *rtree_version(void);

/*
 * rtree_autotune -- choose fanout, node layout and thread mapping by timing.
 *
 * Builds a tree over rects/ids for every fanout in fanouts[0 .. n_fanouts)
 * (NULL or 0 -> {16, 32, 64}; at most 8) and all three layouts, and times a
 * sorted rtree_range_select of the q queries under both mappings with CUDA
 * events on `stream` (one untimed run first).  flags & RTREE_TUNE_INCLUDE_BUILD
 * adds the build time to each configuration's time; flags & RTREE_TUNE_ORDERS
 * also tries every configuration with RTREE_ORDER_HILBERT.  *out receives the
 * fastest configuration and every configuration's time (at most 64).  Inputs
 * may be host or device memory; callers pass a representative sample.
 */
enum { RTREE_TUNE_INCLUDE_BUILD = 1, RTREE_TUNE_ORDERS = 2 };

typedef struct rtree_tune_result {
    int32_t fanout, layout, mapping, order, tried, reserved;
    double ms;              /* time of the chosen configuration */
    double ms_all[64];      /* every configuration tried, in order */
    int32_t fanout_all[64];
    int32_t layout_all[64];
    int32_t mapping_all[64];
    int32_t order_all[64];
} rtree_tune_result_t;

/*
 * rtree_save / rtree_load -- keep a built tree in a file (an addition: the
 * paper's index lives in memory only; a serving process restarts from the
 * file instead of rebuilding).
 *
 * The file is a 1 KiB little-endian header (magic "RTREEGB3", version 1,
 * fanout, layout, sorted flag, level sizes, root MBR, payload size and
 * checksums) followed by the node entries, node metadata, node boxes and
 * leaf-entry ids exactly as held on the device.  rtree_save waits for the
 * tree's stream work, writes a temporary file beside `path` and renames it,
 * so `path` is only ever replaced by a complete file.  rtree_load reads and
 * checks the header and the file size before any device work, copies the
 * payload to `device` (-1: the current device) through pinned staging
 * buffers, verifies the payload checksum and checks on the device that the
 * node structure is a tree (children in the next level, entry ranges inside
 * the leaf level).  The loaded tree answers every call as the saved one.
 * Errors: RTREE_EIO (cannot open, read, write or rename), RTREE_EINVAL (not
 * a tree file of this version, wrong size, checksum or structure mismatch:
 * nothing is returned), RTREE_ENOMEM, RTREE_ECUDA.
 */
RTREE_API rtree_status rtree_save(const rtree_t *tree, const char *path, void *stream);
RTREE_API rtree_status rtree_load(const char *path, int device, void *stream, rtree_t **out);

RTREE_API rtree_status rtree_autotune(const float *rects, const int32_t *ids, int64_t n,
                                      const float *queries, int64_t q, const int32_t *fanouts,
                                      int32_t n_fanouts, int32_t flags, void *stream,
                                      rtree_tune_result_t *out);

/*
 * Kernel accounting.  Every kernel launch the library makes is counted under
 * a short name ("select_count", "sort_mid", ...).  With timing enabled, CUDA
 * events recorded on the launching stream bracket each launch and their
 * elapsed times are summed per name (this adds two event records per
 * launch).  rtree_timing_get returns 0 past the last name; name strings stay
 * valid until the library is unloaded.
 */
RTREE_API void rtree_timing_enable(int on);
RTREE_API void rtree_timing_reset(void);
RTREE_API int rtree_timing_get(int index, const char **name, long long *launches, double *ms);
RTREE_API long long rtree_launch_count(void);

/* Testing hook: the k-th device allocation after this call fails with
 * RTREE_ENOMEM (k = 0: the next one); k < 0 disables.  The failure is made
 * on the host, before cudaMallocAsync is called; no GPU fault is involved. */
RTREE_API void rtree_debug_fail_alloc_after(long long k);

/* Testing hook for the bounded waits of the device work queues (the
 * select's RTREE_MAP_WORK_QUEUE and the join's RTREE_JOIN_QUEUE): the next
 * work-queue pass launched by any host thread (for the join, its count pass)
 * limits each device-side wait for work to `cycles` GPU clock cycles
 * (<= 0: the default, about one second), and with hold != 0 it counts one
 * work item that is never published, so the pass cannot end by running out
 * of work: every waiting warp's wait runs out, the warp records the timeout
 * and returns, and the call reports RTREE_ETIMEOUT.  The waits end by
 * themselves; no GPU fault or trap is involved and the context stays usable.
 * The setting applies to one pass, then resets. */
RTREE_API void rtree_debug_wq_wait(long long cycles, int hold);

#ifdef __cplusplus
}
#endif

#endif /* RTREE_H */
