// mailbox.cu -- small device results delivered to the host without a copy
// engine.
//
// A mailbox is a block of page-locked host memory mapped into the device's
// address space, plus an event.  A kernel stores the values into it, the
// event is recorded behind that kernel, and the host waits for the event and
// reads the words.  A cudaMemcpyAsync of a few bytes would instead wait in a
// copy engine's queue behind every larger copy already queued there (such as
// gigabytes of an earlier call's results still going to the host), which
// would serialize calls that are meant to overlap.  Mailboxes are pooled per
// device: allocating page-locked memory synchronizes the device, so it only
// happens the first time a mailbox is needed.
#include <mutex>
#include <vector>

#include "internal.cuh"

namespace rt {
namespace {

std::mutex g_mu;
std::vector<Mailbox> g_free[64];
std::vector<Mailbox> g_deferred[64];  // handed back while a post into them may still be pending

__global__ void k_post(PostList l, uint32_t *__restrict__ dst)
{
    const int i = threadIdx.x;
    if (i >= l.n)
        return;
    const uint32_t *src = static_cast<const uint32_t *>(l.src[i]);
    for (int w = 0; w < l.words[i]; ++w)
        dst[l.at[i] + w] = src[w];
}

}  // namespace

rtree_status mailbox_get(Mailbox *m)
{
    int dev = 0;
    RT_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64)
        return fail(RTREE_EINVAL, "device %d out of range", dev);
    {
        std::lock_guard<std::mutex> g(g_mu);
        for (size_t i = 0; i < g_deferred[dev].size();) {  // reclaim those whose post has run
            if (cudaEventQuery(g_deferred[dev][i].ev) == cudaSuccess) {
                g_free[dev].push_back(g_deferred[dev][i]);
                g_deferred[dev][i] = g_deferred[dev].back();
                g_deferred[dev].pop_back();
            } else {
                cudaGetLastError();  // cudaErrorNotReady
                ++i;
            }
        }
        if (!g_free[dev].empty()) {
            *m = g_free[dev].back();
            g_free[dev].pop_back();
            return RTREE_OK;
        }
    }
    Mailbox n;
    n.device = dev;
    void *h = nullptr;
    RT_CUDA(cudaHostAlloc(&h, kMailboxWords * sizeof(uint32_t), cudaHostAllocMapped | cudaHostAllocPortable));
    n.h = static_cast<uint32_t *>(h);
    void *d = nullptr;
    cudaError_t e = cudaHostGetDevicePointer(&d, h, 0);
    if (e == cudaSuccess)
        e = cudaEventCreateWithFlags(&n.ev, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        cudaFreeHost(h);
        return fail(RTREE_ECUDA, "mailbox: %s", cudaGetErrorString(e));
    }
    n.d = static_cast<uint32_t *>(d);
    *m = n;
    return RTREE_OK;
}

void mailbox_put(Mailbox *m)
{
    if (!m->h)
        return;
    std::lock_guard<std::mutex> g(g_mu);
    g_free[m->device].push_back(*m);
    *m = Mailbox{};
}

void mailbox_put_deferred(Mailbox *m)
{
    if (!m->h)
        return;
    std::lock_guard<std::mutex> g(g_mu);
    g_deferred[m->device].push_back(*m);
    *m = Mailbox{};
}

rtree_status post_words(const PostList &l, uint32_t *dst, cudaStream_t s)
{
    if (l.n > 0) {
        KernelTimer kt_("mailbox_post", s);
        k_post<<<1, 32, 0, s>>>(l, dst);
        RT_LAUNCH();
    }
    return RTREE_OK;
}

rtree_status mailbox_post(const Mailbox &m, const PostList &l, cudaStream_t s)
{
    RT_TRY(post_words(l, m.d, s));
    RT_CUDA(cudaEventRecord(m.ev, s));
    return RTREE_OK;
}

rtree_status mailbox_wait(const Mailbox &m)
{
    RT_CUDA(cudaEventSynchronize(m.ev));
    return RTREE_OK;
}

rtree_status post_result_status(const int32_t *flags, cudaStream_t s, rtree_result *res)
{
    Mailbox *mb = new Mailbox();
    rtree_status st = mailbox_get(mb);
    if (st != RTREE_OK) {
        delete mb;
        return st;
    }
    PostList pl{};
    pl.src[0] = flags;
    pl.words[0] = 2;
    pl.at[0] = 0;
    pl.n = 1;
    st = mailbox_post(*mb, pl, s);
    if (st != RTREE_OK) {
        cudaEventSynchronize(mb->ev);
        mailbox_put(mb);
        delete mb;
        return st;
    }
    res->status = mb;
    return RTREE_OK;
}

rtree_status read_words(const PostList &l, cudaStream_t s, uint32_t *out, int nwords)
{
    MailboxRef mb;
    RT_TRY(mailbox_get(&mb.m));
    RT_TRY(mailbox_post(mb.m, l, s));
    RT_TRY(mailbox_wait(mb.m));
    for (int i = 0; i < nwords; ++i)
        out[i] = ((const volatile uint32_t *)mb.m.h)[i];
    return RTREE_OK;
}

}  // namespace rt
