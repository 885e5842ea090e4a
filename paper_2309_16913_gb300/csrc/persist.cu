// persist.cu -- save a built tree to a file and load it back.
//
// An addition (the paper keeps its index in memory and says nothing about
// storing it): a serving process can restart from the file instead of
// rebuilding.  The file holds the device arrays exactly as the traversal
// kernels read them, so loading is a checked copy, not a rebuild.
//
// Layout (little-endian, every field fixed-width):
//   header, kHeaderBytes bytes:
//     magic[8] "RTREEGB3", u32 version, u32 endian marker 0x01020304,
//     i32 fanout, i32 layout, i32 sorted, i32 levels,
//     i64 n, i64 nodes, f32 root_mbr[4], i64 level_nodes[40],
//     u64 payload_bytes, u64 payload_hash, u64 header_hash, zero padding;
//   payload: node entries (nodes*F*16 bytes, in the tree's layout), node
//     metadata (nodes x {first, count, elo, ehi} i32), node boxes
//     (nodes x 4 f32), leaf-entry ids (n x i32).
// Hash: 64-bit words of the byte stream (little-endian, the tail padded with
// zeros), h = (rotl(h, 27) ^ w) * 0x9E3779B97F4A7C15 from h = 0x243F6A8885A308D3,
// then h ^= byte count; header_hash covers the header with that field zero.
//
// rtree_save writes a temporary file next to the target and renames it, so
// an existing file is replaced only by a complete one.  rtree_load checks the
// header and the file size before touching the device, streams the payload
// through two pinned staging buffers (reading one while the other is copied
// to the device), compares the checksum, and runs a device check that every
// node's children lie in the next level and every entry range inside the
// leaf level, so a damaged or hand-made file cannot send a traversal out of
// bounds.
#include <cerrno>
#include <cstdio>
#include <cstring>
#include <string>
#include <unistd.h>
#include <vector>

#include "internal.cuh"

namespace rt {
namespace {

const char kMagic[8] = {'R', 'T', 'R', 'E', 'E', 'G', 'B', '3'};
constexpr uint32_t kVersion = 1;
constexpr uint32_t kEndian = 0x01020304u;
constexpr size_t kHeaderBytes = 1024;
constexpr size_t kChunk = size_t(16) << 20;  // staging chunk; a multiple of 8

// Serialized header fields (written and read field by field at fixed offsets).
struct Header {
    int32_t fanout = 0, layout = 0, sorted = 0, levels = 0;
    int64_t n = 0, nodes = 0;
    float root_mbr[4] = {0, 0, 0, 0};
    int64_t level_nodes[RT_MAX_LEVELS] = {};
    uint64_t payload_bytes = 0, payload_hash = 0, header_hash = 0;
};

// Byte offsets inside the header.
enum : size_t {
    O_MAGIC = 0, O_VERSION = 8, O_ENDIAN = 12, O_FANOUT = 16, O_LAYOUT = 20, O_SORTED = 24,
    O_LEVELS = 28, O_N = 32, O_NODES = 40, O_ROOT = 48, O_LEVEL_NODES = 64,
    O_PAYLOAD_BYTES = O_LEVEL_NODES + 8 * RT_MAX_LEVELS, O_PAYLOAD_HASH = O_PAYLOAD_BYTES + 8,
    O_HEADER_HASH = O_PAYLOAD_HASH + 8, O_END = O_HEADER_HASH + 8
};
static_assert(O_END <= kHeaderBytes, "header fields overflow the header");

struct Hasher {
    uint64_t h = 0x243F6A8885A308D3ull;
    uint64_t count = 0;
    unsigned char carry[8];
    int nc = 0;
    void word(uint64_t w)
    {
        h = ((h << 27) | (h >> 37)) ^ w;
        h *= 0x9E3779B97F4A7C15ull;
    }
    static uint64_t load_le(const unsigned char *p)
    {
        uint64_t w = 0;
        for (int i = 7; i >= 0; --i)
            w = (w << 8) | p[i];
        return w;
    }
    void add(const void *data, size_t len)
    {
        const unsigned char *p = static_cast<const unsigned char *>(data);
        count += len;
        while (nc > 0 && len > 0) {
            carry[nc++] = *p++;
            --len;
            if (nc == 8) {
                word(load_le(carry));
                nc = 0;
            }
        }
        for (; len >= 8; p += 8, len -= 8)
            word(load_le(p));
        for (; len > 0; --len)
            carry[nc++] = *p++;
    }
    uint64_t finish()
    {
        if (nc > 0) {
            memset(carry + nc, 0, 8 - nc);
            word(load_le(carry));
            nc = 0;
        }
        return h ^ count;
    }
};

template <typename T>
void put(unsigned char *buf, size_t off, T v)
{
    memcpy(buf + off, &v, sizeof(T));
}
template <typename T>
T get(const unsigned char *buf, size_t off)
{
    T v;
    memcpy(&v, buf + off, sizeof(T));
    return v;
}

void encode(const Header &h, unsigned char *buf)
{
    memset(buf, 0, kHeaderBytes);
    memcpy(buf + O_MAGIC, kMagic, 8);
    put<uint32_t>(buf, O_VERSION, kVersion);
    put<uint32_t>(buf, O_ENDIAN, kEndian);
    put<int32_t>(buf, O_FANOUT, h.fanout);
    put<int32_t>(buf, O_LAYOUT, h.layout);
    put<int32_t>(buf, O_SORTED, h.sorted);
    put<int32_t>(buf, O_LEVELS, h.levels);
    put<int64_t>(buf, O_N, h.n);
    put<int64_t>(buf, O_NODES, h.nodes);
    for (int i = 0; i < 4; ++i)
        put<float>(buf, O_ROOT + 4 * i, h.root_mbr[i]);
    for (int i = 0; i < RT_MAX_LEVELS; ++i)
        put<int64_t>(buf, O_LEVEL_NODES + 8 * i, h.level_nodes[i]);
    put<uint64_t>(buf, O_PAYLOAD_BYTES, h.payload_bytes);
    put<uint64_t>(buf, O_PAYLOAD_HASH, h.payload_hash);
    Hasher hh;
    hh.add(buf, kHeaderBytes);  // header_hash field still zero
    put<uint64_t>(buf, O_HEADER_HASH, hh.finish());
}

// Sizes of the four payload sections, in file order.
void sections(int64_t nodes, int F, int64_t n, size_t out[4])
{
    out[0] = (size_t)nodes * F * 16;
    out[1] = (size_t)nodes * sizeof(int4);
    out[2] = (size_t)nodes * sizeof(float4);
    out[3] = (size_t)n * sizeof(int32_t);
}

// Parses and checks a header; fills *h.  No CUDA call.
rtree_status decode(const unsigned char *buf, size_t got, Header *h)
{
    if (got < kHeaderBytes)
        return fail(RTREE_EINVAL, "rtree_load: file too short for a tree header (%zu bytes)", got);
    if (memcmp(buf + O_MAGIC, kMagic, 8) != 0)
        return fail(RTREE_EINVAL, "rtree_load: not an rtree file (bad magic)");
    if (get<uint32_t>(buf, O_VERSION) != kVersion)
        return fail(RTREE_EINVAL, "rtree_load: file version %u, this library reads %u",
                    get<uint32_t>(buf, O_VERSION), kVersion);
    if (get<uint32_t>(buf, O_ENDIAN) != kEndian)
        return fail(RTREE_EINVAL, "rtree_load: byte order of the file differs from this host");
    unsigned char tmp[kHeaderBytes];
    memcpy(tmp, buf, kHeaderBytes);
    put<uint64_t>(tmp, O_HEADER_HASH, 0);
    Hasher hh;
    hh.add(tmp, kHeaderBytes);
    if (hh.finish() != get<uint64_t>(buf, O_HEADER_HASH))
        return fail(RTREE_EINVAL, "rtree_load: header checksum mismatch (damaged file)");
    h->fanout = get<int32_t>(buf, O_FANOUT);
    h->layout = get<int32_t>(buf, O_LAYOUT);
    h->sorted = get<int32_t>(buf, O_SORTED);
    h->levels = get<int32_t>(buf, O_LEVELS);
    h->n = get<int64_t>(buf, O_N);
    h->nodes = get<int64_t>(buf, O_NODES);
    for (int i = 0; i < 4; ++i)
        h->root_mbr[i] = get<float>(buf, O_ROOT + 4 * i);
    for (int i = 0; i < RT_MAX_LEVELS; ++i)
        h->level_nodes[i] = get<int64_t>(buf, O_LEVEL_NODES + 8 * i);
    h->payload_bytes = get<uint64_t>(buf, O_PAYLOAD_BYTES);
    h->payload_hash = get<uint64_t>(buf, O_PAYLOAD_HASH);
    if (!fanout_ok(h->fanout) || h->layout < RTREE_LAYOUT_SOA || h->layout > RTREE_LAYOUT_LOHI ||
        (h->sorted != 0 && h->sorted != 1))
        return fail(RTREE_EINVAL, "rtree_load: bad fanout/layout/sorted fields");
    if (h->n < 0 || h->n >= (int64_t)INT32_MAX || h->nodes < 0 || h->nodes >= (int64_t)INT32_MAX ||
        h->levels < 0 || h->levels > RT_MAX_LEVELS || (h->n == 0) != (h->levels == 0))
        return fail(RTREE_EINVAL, "rtree_load: bad size fields");
    int64_t sum = 0;
    for (int e = 0; e < h->levels; ++e) {
        const int64_t c = h->level_nodes[e];
        if (c < 1 || c > h->nodes || (e == 0 && c != 1))
            return fail(RTREE_EINVAL, "rtree_load: bad node count on level %d", e);
        sum += c;
    }
    if (sum != h->nodes)
        return fail(RTREE_EINVAL, "rtree_load: level sizes do not add up to the node count");
    size_t sec[4];
    sections(h->nodes, h->fanout, h->n, sec);
    if (h->payload_bytes != sec[0] + sec[1] + sec[2] + sec[3])
        return fail(RTREE_EINVAL, "rtree_load: payload size field does not match the tree shape");
    return RTREE_OK;
}

struct LevelInfo {
    int64_t base[RT_MAX_LEVELS + 1];  // first node of each level; base[levels] = nodes
    int32_t levels;
};

// Structure check of loaded metadata: counts in [1, F]; an internal node's
// children lie in the next level; leaf entries, and every node's entry range,
// inside [0, n).
__global__ void k_check_meta(const int4 *__restrict__ meta, LevelInfo L, int F, int64_t n,
                             unsigned long long *__restrict__ bad)
{
    const int64_t nodes = L.base[L.levels];
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < nodes;
         g += (int64_t)gridDim.x * blockDim.x) {
        int e = 0;
        while (e + 1 < L.levels && L.base[e + 1] <= g)
            ++e;
        const int4 m = meta[g];
        bool ok = m.y >= 1 && m.y <= F && m.z >= 0 && m.z < m.w && m.w <= n;
        if (e + 1 < L.levels)
            ok = ok && m.x >= L.base[e + 1] && (int64_t)m.x + m.y <= L.base[e + 2];
        else
            ok = ok && m.x >= 0 && (int64_t)m.x + m.y <= n;
        if (!ok)
            atomicMin(bad, (unsigned long long)g);
    }
}

struct File {
    FILE *f = nullptr;
    ~File()
    {
        if (f)
            fclose(f);
    }
};

struct Pinned {
    void *p[2] = {nullptr, nullptr};
    cudaEvent_t ev[2] = {nullptr, nullptr};
    ~Pinned()
    {
        for (int i = 0; i < 2; ++i) {
            if (ev[i]) {
                cudaEventSynchronize(ev[i]);
                cudaEventDestroy(ev[i]);
            }
            if (p[i])
                cudaFreeHost(p[i]);
        }
    }
    rtree_status init()
    {
        for (int i = 0; i < 2; ++i) {
            RT_CUDA(cudaMallocHost(&p[i], kChunk));
            RT_CUDA(cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming));
        }
        return RTREE_OK;
    }
};

rtree_status save_impl(const rtree *t, const char *path, cudaStream_t s)
{
    Header h;
    h.fanout = t->fanout;
    h.layout = t->layout;
    h.sorted = t->sorted;
    h.levels = t->levels;
    h.n = t->n;
    h.nodes = t->nodes;
    RT_TRY(tree_root_box(t, h.root_mbr));
    for (int e = 0; e < t->levels; ++e)
        h.level_nodes[e] = t->level_nodes[e];
    size_t sec[4];
    sections(t->nodes, t->fanout, t->n, sec);
    h.payload_bytes = sec[0] + sec[1] + sec[2] + sec[3];
    const void *src[4] = {t->mbr, t->meta, t->nbox, t->ids};

    const std::string tmp = std::string(path) + ".tmp" + std::to_string((long long)getpid());
    File out;
    out.f = fopen(tmp.c_str(), "wb");
    if (!out.f)
        return fail(RTREE_EIO, "rtree_save: cannot create %s: %s", tmp.c_str(), strerror(errno));
    unsigned char hdr[kHeaderBytes];
    memset(hdr, 0, sizeof(hdr));
    bool ok = fwrite(hdr, 1, kHeaderBytes, out.f) == kHeaderBytes;  // placeholder
    Pinned st;
    rtree_status rs = ok ? st.init() : RTREE_OK;
    Hasher ph;
    // chunks of all sections in order; copy chunk k+1 while chunk k is written
    struct Piece {
        const char *p;
        size_t len;
    };
    std::vector<Piece> pieces;
    for (int i = 0; i < 4; ++i)
        for (size_t off = 0; off < sec[i]; off += kChunk)
            pieces.push_back({static_cast<const char *>(src[i]) + off,
                              sec[i] - off < kChunk ? sec[i] - off : kChunk});
    if (ok && rs == RTREE_OK && !pieces.empty()) {
        RT_CUDA(cudaMemcpyAsync(st.p[0], pieces[0].p, pieces[0].len, cudaMemcpyDeviceToHost, s));
        RT_CUDA(cudaEventRecord(st.ev[0], s));
        for (size_t k = 0; k < pieces.size() && ok; ++k) {
            const int b = (int)(k & 1);
            if (k + 1 < pieces.size()) {
                RT_CUDA(cudaMemcpyAsync(st.p[b ^ 1], pieces[k + 1].p, pieces[k + 1].len,
                                        cudaMemcpyDeviceToHost, s));
                RT_CUDA(cudaEventRecord(st.ev[b ^ 1], s));
            }
            RT_CUDA(cudaEventSynchronize(st.ev[b]));
            ph.add(st.p[b], pieces[k].len);
            ok = fwrite(st.p[b], 1, pieces[k].len, out.f) == pieces[k].len;
        }
        RT_CUDA(cudaStreamSynchronize(s));
    }
    if (rs != RTREE_OK) {
        remove(tmp.c_str());
        return rs;
    }
    h.payload_hash = ph.finish();
    encode(h, hdr);
    ok = ok && fseek(out.f, 0, SEEK_SET) == 0 && fwrite(hdr, 1, kHeaderBytes, out.f) == kHeaderBytes;
    ok = ok && fflush(out.f) == 0 && fsync(fileno(out.f)) == 0;
    const int close_rc = fclose(out.f);
    out.f = nullptr;
    if (!ok || close_rc != 0) {
        const int err = errno;
        remove(tmp.c_str());
        return fail(RTREE_EIO, "rtree_save: writing %s failed: %s", tmp.c_str(), strerror(err));
    }
    if (rename(tmp.c_str(), path) != 0) {
        const int err = errno;
        remove(tmp.c_str());
        return fail(RTREE_EIO, "rtree_save: cannot rename to %s: %s", path, strerror(err));
    }
    return RTREE_OK;
}

rtree_status load_payload(FILE *f, const Header &h, rtree *t, cudaStream_t s)
{
    size_t sec[4];
    sections(h.nodes, h.fanout, h.n, sec);
    DevBuf<float> mbr(s);
    DevBuf<int4> meta(s);
    DevBuf<float4> nbox(s);
    DevBuf<int32_t> ids(s);
    RT_TRY(mbr.alloc((size_t)h.nodes * h.fanout * 4, "node entries"));
    RT_TRY(meta.alloc(h.nodes, "node metadata"));
    RT_TRY(nbox.alloc(h.nodes, "node boxes"));
    RT_TRY(ids.alloc(h.n, "entry ids"));
    char *dst[4] = {reinterpret_cast<char *>(mbr.p), reinterpret_cast<char *>(meta.p),
                    reinterpret_cast<char *>(nbox.p), reinterpret_cast<char *>(ids.p)};
    Pinned st;
    RT_TRY(st.init());
    Hasher ph;
    bool used[2] = {false, false};
    int b = 0;
    for (int i = 0; i < 4; ++i) {
        for (size_t off = 0; off < sec[i]; off += kChunk) {
            const size_t len = sec[i] - off < kChunk ? sec[i] - off : kChunk;
            if (used[b])
                RT_CUDA(cudaEventSynchronize(st.ev[b]));  // its previous copy is done
            if (fread(st.p[b], 1, len, f) != len)
                return fail(RTREE_EIO, "rtree_load: short read in the payload");
            ph.add(st.p[b], len);
            RT_CUDA(cudaMemcpyAsync(dst[i] + off, st.p[b], len, cudaMemcpyHostToDevice, s));
            RT_CUDA(cudaEventRecord(st.ev[b], s));
            used[b] = true;
            b ^= 1;
        }
    }
    RT_CUDA(cudaStreamSynchronize(s));
    if (ph.finish() != h.payload_hash)
        return fail(RTREE_EINVAL, "rtree_load: payload checksum mismatch (damaged file)");
    LevelInfo L{};
    L.levels = h.levels;
    int64_t base = 0;
    for (int e = 0; e < h.levels; ++e) {
        L.base[e] = base;
        base += h.level_nodes[e];
    }
    L.base[h.levels] = base;
    if (h.nodes > 0) {
        DevBuf<unsigned long long> bad(s);
        RT_TRY(bad.alloc(1, "load check flag"));
        RT_CUDA(cudaMemsetAsync(bad.p, 0xff, sizeof(unsigned long long), s));
        {
            KernelTimer kt_("check_meta", s);
            int64_t blocks = (h.nodes + 255) / 256;
            k_check_meta<<<(unsigned)(blocks > 65536 ? 65536 : blocks), 256, 0, s>>>(meta.p, L, h.fanout,
                                                                                   h.n, bad.p);
            RT_LAUNCH();
        }
        unsigned long long hb = 0;
        RT_CUDA(cudaMemcpyAsync(&hb, bad.p, sizeof(hb), cudaMemcpyDeviceToHost, s));
        RT_CUDA(cudaStreamSynchronize(s));
        if (hb != ~0ull)
            return fail(RTREE_EINVAL, "rtree_load: node %llu breaks the tree structure", hb);
    }
    t->fanout = h.fanout;
    t->layout = h.layout;
    t->sorted = h.sorted;
    t->levels = h.levels;
    t->n = h.n;
    t->nodes = h.nodes;
    for (int e = 0; e < h.levels; ++e) {
        t->level_nodes[e] = h.level_nodes[e];
        t->level_base[e] = L.base[e];
    }
    memcpy(t->root_mbr, h.root_mbr, sizeof(h.root_mbr));
    t->bytes = (int64_t)h.nodes * h.fanout * 16 + h.nodes * 32 + h.n * 4;
    t->mbr = mbr.release();
    t->meta = meta.release();
    t->nbox = nbox.release();
    t->ids = ids.release();
    // the load returns with its work finished (calls on any stream may use
    // the tree at once): wait for the leaf record too
    RT_TRY(compute_leaf_part(t, s));
    RT_CUDA(cudaStreamSynchronize(s));
    return RTREE_OK;
}

}  // namespace
}  // namespace rt

using namespace rt;

extern "C" rtree_status rtree_save(const rtree_t *tree, const char *path, void *stream)
{
    clear_error();
    if (!tree || !path)
        return fail(RTREE_EINVAL, "rtree_save: NULL argument");
    try {
        DeviceGuard guard(tree->device);
        return save_impl(tree, path, static_cast<cudaStream_t>(stream));
    } catch (...) {
        return fail(RTREE_ENOMEM, "rtree_save: host allocation failed");
    }
}

extern "C" rtree_status rtree_load(const char *path, int device, void *stream, rtree_t **out)
{
    clear_error();
    if (!out)
        return fail(RTREE_EINVAL, "rtree_load: out is NULL");
    *out = nullptr;
    if (!path)
        return fail(RTREE_EINVAL, "rtree_load: path is NULL");
    File in;
    in.f = fopen(path, "rb");
    if (!in.f)
        return fail(RTREE_EIO, "rtree_load: cannot open %s: %s", path, strerror(errno));
    unsigned char hdr[kHeaderBytes];
    const size_t got = fread(hdr, 1, kHeaderBytes, in.f);
    Header h;
    RT_TRY(decode(hdr, got, &h));
    // the file must be exactly header + payload
    if (fseek(in.f, 0, SEEK_END) != 0)
        return fail(RTREE_EIO, "rtree_load: cannot seek in %s", path);
    const long long size = ftell(in.f);
    if (size < 0 || (unsigned long long)size != kHeaderBytes + h.payload_bytes)
        return fail(RTREE_EINVAL, "rtree_load: file is %lld bytes, the header describes %llu",
                    size, (unsigned long long)(kHeaderBytes + h.payload_bytes));
    if (fseek(in.f, (long)kHeaderBytes, SEEK_SET) != 0)
        return fail(RTREE_EIO, "rtree_load: cannot seek in %s", path);
    try {
        int dev = device;
        if (dev < 0)
            RT_CUDA(cudaGetDevice(&dev));
        DeviceGuard guard(dev);
        setup_device_pool(dev);
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        rtree *t = new rtree();
        t->device = dev;
        rtree_status st = load_payload(in.f, h, t, s);
        if (st != RTREE_OK) {
            free_tree_arrays(t);
            delete t;
            return st;
        }
        timing_resolve();
        *out = t;
        return RTREE_OK;
    } catch (...) {
        return fail(RTREE_ENOMEM, "rtree_load: host allocation failed");
    }
}
