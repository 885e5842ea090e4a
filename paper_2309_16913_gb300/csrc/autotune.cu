// autotune.cu -- pick fanout, node layout and thread mapping by measurement.
//
// For each candidate fanout and layout the tree is built from the caller's
// rectangles and the caller's queries are selected (sorted) under each
// thread mapping (and, on request, each traversal order); every
// configuration is timed with CUDA events on the
// caller's stream after one untimed run, optionally including the build.
// The fastest configuration is returned with all the times.  (The select's
// per-warp stack needs no tuning: its depth has an exact bound.)
#include <cstring>

#include "internal.cuh"

using namespace rt;

extern "C" rtree_status rtree_autotune(const float *rects, const int32_t *ids, int64_t n,
                                       const float *queries, int64_t q, const int32_t *fanouts,
                                       int32_t n_fanouts, int32_t flags, void *stream,
                                       rtree_tune_result_t *out)
{
    clear_error();
    if (!out || (n > 0 && !rects) || (q > 0 && !queries) || n_fanouts < 0 || n_fanouts > 8)
        return fail(RTREE_EINVAL, "rtree_autotune: bad argument");
    memset(out, 0, sizeof(*out));
    static const int32_t kDefault[3] = {16, 32, 64};
    if (!fanouts || n_fanouts == 0) {
        fanouts = kDefault;
        n_fanouts = 3;
    }
    const bool with_build = (flags & RTREE_TUNE_INCLUDE_BUILD) != 0;
    const int n_orders = (flags & RTREE_TUNE_ORDERS) ? 2 : 1;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        return fail(RTREE_ECUDA, "rtree_autotune: cudaEventCreate failed");
    }
    rtree_status st = RTREE_OK;
    double best = 1e300;
    int k = 0;
    for (int fi = 0; fi < n_fanouts && st == RTREE_OK; ++fi) {
        for (int layout = RTREE_LAYOUT_SOA; layout <= RTREE_LAYOUT_LOHI && st == RTREE_OK; ++layout) {
            rtree_config_t cfg{};
            cfg.fanout = fanouts[fi];
            cfg.layout = layout;
            rtree_t *tree = nullptr;
            float build_ms = 0.f;
            cudaEventRecord(e0, s);
            st = rtree_build(rects, ids, n, &cfg, nullptr, stream, &tree);
            cudaEventRecord(e1, s);
            if (st != RTREE_OK)
                break;
            cudaEventSynchronize(e1);
            cudaEventElapsedTime(&build_ms, e0, e1);
            for (int combo = 0; combo < 2 * n_orders && st == RTREE_OK; ++combo) {
                const int mapping = RTREE_MAP_WARP_PER_QUERY + combo % 2;
                const int order = combo / 2 ? RTREE_ORDER_HILBERT : RTREE_ORDER_INPUT;
                rtree_select_opts_t opts{};
                opts.mapping = mapping;
                opts.order = order;
                float sel_ms = 0.f;
                for (int rep = 0; rep < 2 && st == RTREE_OK; ++rep) {  // untimed, then timed
                    rtree_result_t *res = nullptr;
                    cudaEventRecord(e0, s);
                    st = rtree_range_select(tree, queries, q, &opts, stream, &res);
                    cudaEventRecord(e1, s);
                    if (st == RTREE_OK) {
                        cudaEventSynchronize(e1);
                        cudaEventElapsedTime(&sel_ms, e0, e1);
                        rtree_result_free(res);
                    }
                }
                if (st != RTREE_OK)
                    break;
                const double ms = sel_ms + (with_build ? build_ms : 0.f);
                if (k < 64) {
                    out->ms_all[k] = ms;
                    out->fanout_all[k] = cfg.fanout;
                    out->layout_all[k] = layout;
                    out->mapping_all[k] = mapping;
                    out->order_all[k] = order;
                }
                ++k;
                if (ms < best) {
                    best = ms;
                    out->fanout = cfg.fanout;
                    out->layout = layout;
                    out->mapping = mapping;
                    out->order = order;
                    out->ms = ms;
                }
            }
            rtree_free(tree);
        }
    }
    out->tried = k < 64 ? k : 64;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return st;
}
