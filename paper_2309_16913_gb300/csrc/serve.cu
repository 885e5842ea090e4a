// serve.cu -- request loop over a device-resident index (continuous batching).
//
// Clients submit range-select requests (a few query rectangles) and probe-join
// requests (a set of rectangles joined with the index); workers turn the
// waiting requests into batches.  Each worker owns a CUDA stream and a
// graph-captured plan (plan.cu), so several batches run on the device at once
// and a request that arrives while batches are in flight joins the next batch
// a free worker forms.  Admission is by output memory: a worker adds requests
// while the batch's expected result (running mean of ids per query) fits its
// plan's id capacity; a batch that still overflows is split in two and run
// again, and a single request too large for any plan is answered by the
// allocating rtree_range_select.  Results are copied to host memory; the
// reply's latency runs from submission to the copy being complete.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t ticket;
    int32_t kind;
    std::vector<float4> queries;
    Clock::time_point submitted;
};

struct Reply {
    rtree_status status = RTREE_OK;
    int32_t kind = 0;
    std::vector<int64_t> offsets;
    std::vector<int32_t> ids;
    double latency_us = 0;
};

}  // namespace

struct rtree_server {
    const rtree *tree = nullptr;
    rtree_server_config_t cfg{};
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request> pending;
    std::unordered_map<uint64_t, Reply> done;
    std::vector<std::thread> workers;
    uint64_t next_ticket = 1;
    bool stopping = false;
    rtree_status worker_error = RTREE_OK;
    // statistics
    std::vector<double> latencies;
    long long batches = 0, batch_queries = 0, splits = 0, fallbacks = 0, completed = 0;
    double ids_per_query = 64.0;  // running estimate for admission
    Clock::time_point started;
};

namespace rt {
namespace {

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

// Runs the queries of `reqs` (concatenated) and writes their replies.
void run_batch(rtree_server *srv, rtree_plan_t *plan, cudaStream_t s, std::vector<Request> &reqs,
               int64_t *h_off, int32_t *h_ids, int64_t ids_cap, std::vector<Reply> &replies,
               long long *splits, long long *fallbacks)
{
    std::vector<float4> q;
    for (const Request &r : reqs)
        q.insert(q.end(), r.queries.begin(), r.queries.end());
    const int64_t nq = (int64_t)q.size();
    int64_t total = 0;
    rtree_status st = rtree_plan_run(plan, reinterpret_cast<const float *>(q.data()), nq, s, &total);
    if (st == RTREE_EOVERFLOW && reqs.size() > 1) {  // split and retry
        ++*splits;
        std::vector<Request> a(reqs.begin(), reqs.begin() + reqs.size() / 2);
        std::vector<Request> b(reqs.begin() + reqs.size() / 2, reqs.end());
        std::vector<Reply> ra, rb;
        run_batch(srv, plan, s, a, h_off, h_ids, ids_cap, ra, splits, fallbacks);
        run_batch(srv, plan, s, b, h_off, h_ids, ids_cap, rb, splits, fallbacks);
        replies = ra;
        replies.insert(replies.end(), rb.begin(), rb.end());
        return;
    }
    replies.assign(reqs.size(), Reply{});
    if (st == RTREE_EOVERFLOW) {  // one request larger than the plan: allocate for it
        ++*fallbacks;
        rtree_result_t *res = nullptr;
        st = rtree_range_select(srv->tree, reinterpret_cast<const float *>(q.data()), nq, nullptr, s, &res);
        if (st == RTREE_OK) {
            Reply &r = replies[0];
            r.kind = reqs[0].kind;
            r.offsets.resize(nq + 1);
            r.ids.resize(rtree_result_total(res));
            st = rtree_result_copy_to_host(res, r.offsets.data(), r.ids.empty() ? nullptr : r.ids.data(), s);
            rtree_result_free_async(res, s);
        }
        replies[0].status = st;
        return;
    }
    if (st != RTREE_OK) {
        for (Reply &r : replies)
            r.status = st;
        return;
    }
    cudaError_t e1 = cudaMemcpyAsync(h_off, rtree_plan_offsets(plan), (nq + 1) * sizeof(int64_t),
                                     cudaMemcpyDeviceToHost, s);
    cudaError_t e2 = total ? cudaMemcpyAsync(h_ids, rtree_plan_ids(plan), total * sizeof(int32_t),
                                             cudaMemcpyDeviceToHost, s)
                           : cudaSuccess;
    cudaError_t e3 = cudaStreamSynchronize(s);
    if (e1 || e2 || e3) {
        for (Reply &r : replies)
            r.status = RTREE_ECUDA;
        return;
    }
    int64_t qpos = 0;
    for (size_t k = 0; k < reqs.size(); ++k) {
        const int64_t n = (int64_t)reqs[k].queries.size();
        const int64_t b0 = h_off[qpos], b1 = h_off[qpos + n];
        Reply &r = replies[k];
        r.kind = reqs[k].kind;
        r.offsets.resize(n + 1);
        for (int64_t i = 0; i <= n; ++i)
            r.offsets[i] = h_off[qpos + i] - b0;
        r.ids.assign(h_ids + b0, h_ids + b1);
        qpos += n;
    }
    (void)ids_cap;
}

void worker_main(rtree_server *srv, int index)
{
    CurrentDevice guard(srv->tree->device);
    cudaStream_t s = nullptr;
    rtree_plan_t *plan = nullptr;
    int64_t *h_off = nullptr;
    int32_t *h_ids = nullptr;
    const int64_t maxq = srv->cfg.max_batch_queries, cap = srv->cfg.max_batch_ids;
    rtree_select_opts_t opts{};
    opts.mapping = srv->cfg.mapping;
    rtree_status st = RTREE_OK;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
        cudaMallocHost(reinterpret_cast<void **>(&h_off), (maxq + 1) * sizeof(int64_t)) != cudaSuccess ||
        cudaMallocHost(reinterpret_cast<void **>(&h_ids), cap * sizeof(int32_t)) != cudaSuccess)
        st = RTREE_ENOMEM;
    if (st == RTREE_OK)
        st = rtree_plan_create(srv->tree, maxq, cap, &opts, &plan);
    if (st != RTREE_OK) {
        std::lock_guard<std::mutex> g(srv->mu);
        srv->worker_error = st;
        srv->cv_done.notify_all();
    }
    (void)index;
    while (st == RTREE_OK) {
        std::vector<Request> batch;
        {
            std::unique_lock<std::mutex> g(srv->mu);
            srv->cv_work.wait(g, [&] { return srv->stopping || !srv->pending.empty(); });
            if (srv->pending.empty() && srv->stopping)
                break;
            // admission: queries and expected ids must fit this worker's plan
            int64_t nq = 0;
            double expect = 0;
            while (!srv->pending.empty()) {
                const Request &r = srv->pending.front();
                const int64_t n = (int64_t)r.queries.size();
                const double e = n * srv->ids_per_query;
                if (!batch.empty() && (nq + n > maxq || expect + e > 0.8 * (double)cap))
                    break;
                if (n > maxq && batch.empty()) {  // never fits a plan: run it alone
                    batch.push_back(std::move(srv->pending.front()));
                    srv->pending.pop_front();
                    break;
                }
                nq += n;
                expect += e;
                batch.push_back(std::move(srv->pending.front()));
                srv->pending.pop_front();
            }
        }
        std::vector<Reply> replies;
        long long splits = 0, fallbacks = 0;
        int64_t nq = 0, nids = 0;
        for (const Request &r : batch)
            nq += (int64_t)r.queries.size();
        if (nq > maxq) {  // a request larger than a plan
            replies.assign(1, Reply{});
            rtree_result_t *res = nullptr;
            const Request &r = batch[0];
            rtree_status rs = rtree_range_select(srv->tree, reinterpret_cast<const float *>(r.queries.data()),
                                                 (int64_t)r.queries.size(), nullptr, s, &res);
            replies[0].kind = r.kind;
            if (rs == RTREE_OK) {
                replies[0].offsets.resize(r.queries.size() + 1);
                replies[0].ids.resize(rtree_result_total(res));
                rs = rtree_result_copy_to_host(res, replies[0].offsets.data(),
                                               replies[0].ids.empty() ? nullptr : replies[0].ids.data(), s);
                rtree_result_free_async(res, s);
            }
            replies[0].status = rs;
            fallbacks = 1;
        } else {
            run_batch(srv, plan, s, batch, h_off, h_ids, cap, replies, &splits, &fallbacks);
        }
        const Clock::time_point now = Clock::now();
        std::lock_guard<std::mutex> g(srv->mu);
        for (size_t k = 0; k < batch.size(); ++k) {
            Reply &r = replies[k];
            r.latency_us = std::chrono::duration<double, std::micro>(now - batch[k].submitted).count();
            nids += (int64_t)r.ids.size();
            srv->latencies.push_back(r.latency_us);
            srv->done[batch[k].ticket] = std::move(r);
        }
        srv->batches += 1;
        srv->batch_queries += nq;
        srv->splits += splits;
        srv->fallbacks += fallbacks;
        srv->completed += (long long)batch.size();
        if (nq > 0)
            srv->ids_per_query = 0.8 * srv->ids_per_query + 0.2 * ((double)nids / (double)nq);
        srv->cv_done.notify_all();
    }
    if (plan)
        rtree_plan_free(plan);
    if (h_off)
        cudaFreeHost(h_off);
    if (h_ids)
        cudaFreeHost(h_ids);
    if (s)
        cudaStreamDestroy(s);
}

double percentile(std::vector<double> v, double p)
{
    if (v.empty())
        return 0.0;
    std::sort(v.begin(), v.end());
    size_t k = (size_t)(p * (double)(v.size() - 1) + 0.5);
    return v[std::min(k, v.size() - 1)];
}

}  // namespace
}  // namespace rt

using namespace rt;

extern "C" {

rtree_status rtree_server_start(const rtree_t *tree, const rtree_server_config_t *cfg,
                                rtree_server_t **out)
{
    clear_error();
    if (!out || !tree)
        return fail(RTREE_EINVAL, "rtree_server_start: NULL tree or out");
    *out = nullptr;
    try {
        rtree_server *srv = new rtree_server();
        srv->tree = tree;
        if (cfg)
            srv->cfg = *cfg;
        if (srv->cfg.workers <= 0)
            srv->cfg.workers = 2;
        if (srv->cfg.max_batch_queries <= 0)
            srv->cfg.max_batch_queries = 16384;
        if (srv->cfg.max_batch_ids <= 0)
            srv->cfg.max_batch_ids = 16 << 20;
        if (srv->cfg.mapping < RTREE_MAP_AUTO || srv->cfg.mapping > RTREE_MAP_WORK_QUEUE) {
            delete srv;
            return fail(RTREE_EINVAL, "rtree_server_start: unknown mapping");
        }
        srv->started = Clock::now();
        for (int i = 0; i < srv->cfg.workers; ++i)
            srv->workers.emplace_back(worker_main, srv, i);
        *out = srv;
        return RTREE_OK;
    } catch (...) {
        return fail(RTREE_ENOMEM, "rtree_server_start: host allocation failed");
    }
}

rtree_status rtree_server_submit(rtree_server_t *srv, const float *queries, int64_t q, int32_t kind,
                                 uint64_t *ticket)
{
    clear_error();
    if (!srv || !ticket || q < 0 || (q > 0 && !queries) || kind < 0 || kind > 1)
        return fail(RTREE_EINVAL, "rtree_server_submit: bad argument");
    try {
        Request r;
        r.kind = kind;
        r.queries.resize(q);
        if (q)
            memcpy(r.queries.data(), queries, q * sizeof(float4));
        r.submitted = Clock::now();
        std::lock_guard<std::mutex> g(srv->mu);
        if (srv->worker_error != RTREE_OK)
            return fail(srv->worker_error, "rtree_server_submit: the server's workers failed to start");
        if (srv->stopping)
            return fail(RTREE_EINVAL, "rtree_server_submit: the server is stopping");
        r.ticket = srv->next_ticket++;
        *ticket = r.ticket;
        srv->pending.push_back(std::move(r));
        srv->cv_work.notify_one();
        return RTREE_OK;
    } catch (...) {
        return fail(RTREE_ENOMEM, "rtree_server_submit: host allocation failed");
    }
}

rtree_status rtree_server_wait(rtree_server_t *srv, uint64_t ticket, int64_t timeout_us,
                               rtree_reply_t *out)
{
    clear_error();
    if (!srv || !out)
        return fail(RTREE_EINVAL, "rtree_server_wait: NULL argument");
    memset(out, 0, sizeof(*out));
    std::unique_lock<std::mutex> g(srv->mu);
    auto ready = [&] { return srv->done.count(ticket) || srv->worker_error != RTREE_OK; };
    if (timeout_us < 0)
        srv->cv_done.wait(g, ready);
    else if (!srv->cv_done.wait_for(g, std::chrono::microseconds(timeout_us), ready))
        return fail(RTREE_ETIMEOUT, "rtree_server_wait: ticket %llu not done within %lld us",
                    (unsigned long long)ticket, (long long)timeout_us);
    auto it = srv->done.find(ticket);
    if (it == srv->done.end())
        return fail(srv->worker_error, "rtree_server_wait: the server's workers failed");
    Reply r = std::move(it->second);
    srv->done.erase(it);
    g.unlock();
    if (r.status != RTREE_OK)
        return fail(r.status, "rtree_server_wait: the request failed");
    out->kind = r.kind;
    out->rows = r.offsets.empty() ? 0 : (int64_t)r.offsets.size() - 1;
    out->total = (int64_t)r.ids.size();
    out->latency_us = r.latency_us;
    out->offsets = static_cast<int64_t *>(malloc((out->rows + 1) * sizeof(int64_t)));
    out->ids = static_cast<int32_t *>(malloc((out->total ? out->total : 1) * sizeof(int32_t)));
    if (!out->offsets || !out->ids) {
        free(out->offsets);
        free(out->ids);
        memset(out, 0, sizeof(*out));
        return fail(RTREE_ENOMEM, "rtree_server_wait: host allocation failed");
    }
    if (r.offsets.empty())
        out->offsets[0] = 0;
    else
        memcpy(out->offsets, r.offsets.data(), r.offsets.size() * sizeof(int64_t));
    if (out->total)
        memcpy(out->ids, r.ids.data(), out->total * sizeof(int32_t));
    return RTREE_OK;
}

void rtree_reply_free(rtree_reply_t *r)
{
    if (!r)
        return;
    free(r->offsets);
    free(r->ids);
    r->offsets = nullptr;
    r->ids = nullptr;
}

rtree_status rtree_server_get_stats(rtree_server_t *srv, rtree_server_stats_t *st)
{
    clear_error();
    if (!srv || !st)
        return fail(RTREE_EINVAL, "rtree_server_get_stats: NULL argument");
    std::lock_guard<std::mutex> g(srv->mu);
    memset(st, 0, sizeof(*st));
    st->completed = srv->completed;
    st->batches = srv->batches;
    st->batch_queries = srv->batch_queries;
    st->splits = srv->splits;
    st->fallbacks = srv->fallbacks;
    st->pending = (int64_t)srv->pending.size();
    st->p50_us = percentile(srv->latencies, 0.50);
    st->p99_us = percentile(srv->latencies, 0.99);
    st->max_us = percentile(srv->latencies, 1.0);
    st->elapsed_s = std::chrono::duration<double>(Clock::now() - srv->started).count();
    return RTREE_OK;
}

rtree_status rtree_server_reset_stats(rtree_server_t *srv)
{
    if (!srv)
        return fail(RTREE_EINVAL, "rtree_server_reset_stats: NULL server");
    std::lock_guard<std::mutex> g(srv->mu);
    srv->latencies.clear();
    srv->batches = srv->batch_queries = srv->splits = srv->fallbacks = srv->completed = 0;
    srv->started = Clock::now();
    return RTREE_OK;
}

void rtree_server_stop(rtree_server_t *srv)
{
    if (!srv)
        return;
    {
        std::lock_guard<std::mutex> g(srv->mu);
        srv->stopping = true;
        srv->cv_work.notify_all();
    }
    for (std::thread &t : srv->workers)
        t.join();
    delete srv;
}

}  // extern "C"
