// timing.cu -- per-kernel launch counts and (optionally) device time.
//
// Every kernel launch site declares a KernelTimer with a name.  Launches are
// always counted.  When timing is enabled, a pair of CUDA events is recorded
// around the launch on the launching stream; elapsed times are resolved once
// the stream has been synchronized (at the end of every C-ABI call, or when
// the totals are read).  Resolving at the end of a call only takes the pairs
// whose work has finished; reading the totals waits for all of them.
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "internal.cuh"

namespace rt {
namespace {

struct Entry {
    std::string name;
    long long launches = 0;
    double ms = 0.0;
};

struct Pending {
    int entry;
    cudaEvent_t a, b;
};

std::mutex g_mu;
std::vector<Entry> g_entries;
std::vector<Pending> g_pending;
std::vector<cudaEvent_t> g_pool;
bool g_enabled = false;
long long g_total_launches = 0;

int entry_for(const char *name)
{
    for (size_t i = 0; i < g_entries.size(); ++i)
        if (g_entries[i].name == name)
            return (int)i;
    g_entries.push_back(Entry{name, 0, 0.0});
    return (int)g_entries.size() - 1;
}

cudaEvent_t get_event()
{
    if (!g_pool.empty()) {
        cudaEvent_t e = g_pool.back();
        g_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

// Adds the times of the recorded pairs.  wait: every pair, waiting for its
// events; else only pairs whose end event has completed (the others stay
// pending), so that a call can resolve without waiting for its own work
// still in flight.
void resolve_locked(bool wait)
{
    size_t keep = 0;
    for (size_t i = 0; i < g_pending.size(); ++i) {
        const Pending p = g_pending[i];
        if (!wait) {
            const cudaError_t q = cudaEventQuery(p.b);
            if (q == cudaErrorNotReady) {
                cudaGetLastError();
                g_pending[keep++] = p;
                continue;
            }
        }
        float ms = 0.f;
        if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess)
            g_entries[p.entry].ms += ms;
        else
            cudaGetLastError();
        g_pool.push_back(p.a);
        g_pool.push_back(p.b);
    }
    g_pending.resize(keep);
}

}  // namespace

// While this thread captures a CUDA graph, launches are counted here (the
// graph's replays add them later) and no events are recorded.
thread_local long long t_capture_launches = -1;

void timing_capture_begin() { t_capture_launches = 0; }

long long timing_capture_end()
{
    const long long n = t_capture_launches;
    t_capture_launches = -1;
    return n < 0 ? 0 : n;
}

void timing_add_replay(const char *name, long long launches)
{
    std::lock_guard<std::mutex> g(g_mu);
    const int e = entry_for(name);
    g_entries[e].launches += launches;
    g_total_launches += launches;
}

KernelTimer::KernelTimer(const char *name, cudaStream_t s) : s_(s)
{
    if (t_capture_launches >= 0) {
        ++t_capture_launches;
        return;
    }
    std::lock_guard<std::mutex> g(g_mu);
    entry_ = entry_for(name);
    g_entries[entry_].launches++;
    g_total_launches++;
    if (g_enabled) {
        a_ = get_event();
        b_ = get_event();
        if (a_ && b_)
            cudaEventRecord(a_, s_);
    }
}

KernelTimer::~KernelTimer()
{
    if (!a_ || !b_)
        return;
    std::lock_guard<std::mutex> g(g_mu);
    cudaEventRecord(b_, s_);
    g_pending.push_back(Pending{entry_, a_, b_});
}

PhaseTimer::PhaseTimer(const char *name, cudaStream_t s) : s_(s)
{
    if (t_capture_launches >= 0)
        return;
    std::lock_guard<std::mutex> g(g_mu);
    entry_ = entry_for(name);
    g_entries[entry_].launches++;  // counts spans, not kernel launches
    if (g_enabled) {
        a_ = get_event();
        b_ = get_event();
        if (a_ && b_)
            cudaEventRecord(a_, s_);
    }
}

PhaseTimer::~PhaseTimer()
{
    if (!a_ || !b_)
        return;
    std::lock_guard<std::mutex> g(g_mu);
    cudaEventRecord(b_, s_);
    g_pending.push_back(Pending{entry_, a_, b_});
}

void timing_resolve()
{
    std::lock_guard<std::mutex> g(g_mu);
    resolve_locked(false);
}

}  // namespace rt

using namespace rt;

extern "C" {

void rtree_timing_enable(int on)
{
    std::lock_guard<std::mutex> g(g_mu);
    g_enabled = on != 0;
}

void rtree_timing_reset(void)
{
    std::lock_guard<std::mutex> g(g_mu);
    resolve_locked(true);
    for (Entry &e : g_entries) {
        e.launches = 0;
        e.ms = 0.0;
    }
    g_total_launches = 0;
}

int rtree_timing_get(int index, const char **name, long long *launches, double *ms)
{
    std::lock_guard<std::mutex> g(g_mu);
    resolve_locked(true);
    if (index < 0 || index >= (int)g_entries.size())
        return 0;
    if (name)
        *name = g_entries[index].name.c_str();
    if (launches)
        *launches = g_entries[index].launches;
    if (ms)
        *ms = g_entries[index].ms;
    return 1;
}

long long rtree_launch_count(void)
{
    std::lock_guard<std::mutex> g(g_mu);
    return g_total_launches;
}

}  // extern "C"
