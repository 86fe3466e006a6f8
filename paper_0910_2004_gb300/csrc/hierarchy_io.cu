// Saving a hierarchy to a file and loading it back onto the device, so a
// coarsened graph (every level, every map, a batch's offsets) can be kept
// and refined later without coarsening again.  The file is little-endian:
//
//   u64 magic "KPHIER01", i32 version, i32 levels L, i32 num_graphs G,
//   i32 reserved; then for l = 0..L-1 the level's sizes and row offsets --
//   version 1 (32-bit offsets): i32 n, i32 nnz, int32 xadj[n+1]; version 2
//   (64-bit offsets): i32 n, i32 0, i64 nnz, int64 xadj[n+1] -- then
//   adjncy[nnz], ewgt[nnz], vwgt[n], and for l < L-1 map[n]; for a batch
//   (G > 0) also goff[G+1] per level, then glevels[G] and gid0[n_0].  A
//   library writes the version of its own offset width and reads both (a
//   32-bit build refuses a level of 2^31 entries or more).
#include <cstdio>
#include <cstring>
#include <new>
#include <type_traits>
#include <vector>

#include "kp_internal.cuh"

using namespace kp;

namespace {

constexpr uint64_t KP_HIER_MAGIC = 0x313052454948504bull;   // "KPHIER01"
constexpr int32_t KP_HIER_VERSION = KP_OFFSET_BITS == 64 ? 2 : 1;

struct File {
    FILE *f = nullptr;
    ~File() {
        if (f) fclose(f);
    }
};

kp_status put(FILE *f, const void *p, size_t bytes) {
    if (bytes && fwrite(p, 1, bytes, f) != bytes) return set_error(KP_ERR_INVALID, "write failed");
    return KP_OK;
}

kp_status get(FILE *f, void *p, size_t bytes) {
    if (bytes && fread(p, 1, bytes, f) != bytes) return set_error(KP_ERR_INVALID, "truncated hierarchy file");
    return KP_OK;
}

// A device array to the file through a host buffer.
template <class T>
kp_status put_dev(FILE *f, const T *d, int64_t count, std::vector<T> &buf) {
    if (count <= 0) return KP_OK;
    buf.resize((size_t)count);
    KP_CUDA(cudaMemcpy(buf.data(), d, sizeof(T) * (size_t)count, cudaMemcpyDeviceToHost));
    return put(f, buf.data(), sizeof(T) * (size_t)count);
}

}  // namespace

static kp_status hierarchy_save_impl(const kp_hierarchy *h, const char *path) {
    if (!h || !path) return set_error(KP_ERR_INVALID, "null argument");
    if (h->stream && cudaStreamSynchronize(h->stream) != cudaSuccess)
        return cuda_error(cudaGetLastError(), "sync");
    File file;
    file.f = fopen(path, "wb");
    if (!file.f) return set_error(KP_ERR_INVALID, std::string("cannot open for writing: ") + path);
    FILE *f = file.f;
    const int32_t L = (int32_t)h->levels.size(), G = h->num_graphs;
    const uint64_t magic = KP_HIER_MAGIC;
    const int32_t head[4] = {KP_HIER_VERSION, L, G, 0};
    KP_TRY(put(f, &magic, 8));
    KP_TRY(put(f, head, sizeof head));
    std::vector<int32_t> buf;
    std::vector<eoff> xbuf;
    for (int32_t l = 0; l < L; l++) {
        const kp_level &lv = h->levels[(size_t)l];
        if (KP_HIER_VERSION == 1) {
            const int32_t sz[2] = {lv.n, (int32_t)lv.nnz};
            KP_TRY(put(f, sz, sizeof sz));
        } else {
            const int32_t sz[2] = {lv.n, 0};
            const int64_t nnz = lv.nnz;
            KP_TRY(put(f, sz, sizeof sz));
            KP_TRY(put(f, &nnz, sizeof nnz));
        }
        KP_TRY(put_dev(f, lv.xadj, (int64_t)lv.n + 1, xbuf));
        KP_TRY(put_dev(f, lv.adjncy, lv.nnz, buf));
        KP_TRY(put_dev(f, lv.ewgt, lv.nnz, buf));
        KP_TRY(put_dev(f, lv.vwgt, lv.n, buf));
        if (l < L - 1) KP_TRY(put_dev(f, lv.map, lv.n, buf));
        if (G > 0) KP_TRY(put_dev(f, lv.goff, (int64_t)G + 1, buf));
    }
    if (G > 0) {
        KP_TRY(put(f, h->glevels.data(), sizeof(int32_t) * (size_t)G));
        KP_TRY(put_dev(f, h->gid0, L > 0 ? h->levels[0].n : 0, buf));
    }
    if (fflush(f) != 0) return set_error(KP_ERR_INVALID, "write failed");
    return KP_OK;
}

// A level of a hierarchy file, read and checked on the host.
struct HostLevel {
    int32_t n = 0;
    int64_t nnz = 0;
    std::vector<int64_t> xadj;   // the file's offsets, widened
    std::vector<int32_t> adjncy, ewgt, vwgt, map, goff;
};

// Uploads the checked host arrays into h (which it frees on an error).
static kp_status upload_hierarchy(kp_hierarchy *h, const std::vector<HostLevel> &lv, const std::vector<std::vector<eoff>> &xs,
                                  const std::vector<int32_t> &glevels, const std::vector<int32_t> &gid0, int32_t L,
                                  int32_t G, cudaStream_t s, kp_hierarchy **out) {
    h->stream = s;
    h->num_graphs = G;
    auto fail = [&](kp_status st) {
        kp_hierarchy_free(h);
        return st;
    };
    if (cudaGetDevice(&h->device) != cudaSuccess) return fail(cuda_error(cudaGetLastError(), "device"));
    auto up = [&](auto **dst, const auto &src) -> kp_status {
        using T = typename std::remove_reference<decltype(src)>::type::value_type;
        KP_TRY(dev_alloc_n(dst, (int64_t)src.size(), s));
        h->allocations.push_back(*dst);
        if (!src.empty())
            KP_CUDA(cudaMemcpyAsync(*dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice, s));
        return KP_OK;
    };
    for (int32_t l = 0; l < L; l++) {
        const HostLevel &H = lv[(size_t)l];
        kp_level k;
        k.n = H.n;
        k.nnz = (eoff)H.nnz;
        k.owned = true;
        kp_status st = up(&k.xadj, xs[(size_t)l]);
        if (st == KP_OK) st = up(&k.adjncy, H.adjncy);
        if (st == KP_OK) st = up(&k.ewgt, H.ewgt);
        if (st == KP_OK) st = up(&k.vwgt, H.vwgt);
        if (st == KP_OK && l < L - 1) st = up(&k.map, H.map);
        if (st == KP_OK && G > 0) st = up(&k.goff, H.goff);
        if (st != KP_OK) return fail(st);
        h->levels.push_back(k);
    }
    if (G > 0) {
        h->glevels = glevels;
        kp_status st = up(&h->glevels_dev, glevels);
        if (st == KP_OK) st = up(&h->gid0, gid0);
        if (st != KP_OK) return fail(st);
    }
    h->per_level.assign((size_t)(L - 1), kp_level_profile{});
    for (int32_t l = 0; l + 1 < L; l++) {
        h->per_level[(size_t)l].n = h->levels[(size_t)l].n;
        h->per_level[(size_t)l].nnz = h->levels[(size_t)l].nnz;
        h->total_matched += (int64_t)h->levels[(size_t)l].n - h->levels[(size_t)l + 1].n;
    }
    h->total.n = h->levels[0].n;
    h->total.nnz = h->levels[0].nnz;
    // the host vectors are the copies' sources: wait before they go
    if (cudaStreamSynchronize(s) != cudaSuccess) return fail(cuda_error(cudaGetLastError(), "sync"));
    *out = h;
    return KP_OK;
}

static kp_status hierarchy_load_impl(const char *path, kp_stream stream, kp_hierarchy **out) {
    if (!path || !out) return set_error(KP_ERR_INVALID, "null argument");
    *out = nullptr;
    cudaStream_t s = (cudaStream_t)stream;
    File file;
    file.f = fopen(path, "rb");
    if (!file.f) return set_error(KP_ERR_INVALID, std::string("cannot open: ") + path);
    FILE *f = file.f;
    // the file's size bounds every array before a buffer is sized for it, so
    // a damaged header cannot make the loader take more host memory than the
    // file holds (a stream that cannot seek is read without the bound)
    long fsize = -1;
    if (fseek(f, 0, SEEK_END) == 0) fsize = ftell(f);
    if (fseek(f, 0, SEEK_SET) != 0) {
        clearerr(f);
        fsize = -1;
    }
    auto room = [&](int64_t bytes) {
        if (fsize < 0) return true;
        const long pos = ftell(f);
        return pos >= 0 && pos <= fsize && bytes <= (int64_t)(fsize - pos);
    };
    uint64_t magic = 0;
    int32_t head[4] = {0, 0, 0, 0};
    KP_TRY(get(f, &magic, 8));
    KP_TRY(get(f, head, sizeof head));
    if (magic != KP_HIER_MAGIC) return set_error(KP_ERR_INVALID, "not a hierarchy file");
    if (head[0] != 1 && head[0] != 2) return set_error(KP_ERR_UNSUPPORTED, "hierarchy file version");
    const bool wide_file = head[0] == 2;
    const int32_t L = head[1], G = head[2];
    if (L < 1 || L > 128 || G < 0) return set_error(KP_ERR_INVALID, "bad hierarchy header");   // at most 128 levels

    // everything is read and checked on the host before anything reaches the
    // device: the kernels index with these arrays
    std::vector<HostLevel> lv((size_t)L);
    auto rd = [&](std::vector<int32_t> &v, int64_t count) -> kp_status {
        if (count < 0 || count > (1ll << 32)) return set_error(KP_ERR_INVALID, "bad array size in hierarchy file");
        if (!room((int64_t)sizeof(int32_t) * count)) return set_error(KP_ERR_INVALID, "truncated hierarchy file");
        v.resize((size_t)count);
        return get(f, v.data(), sizeof(int32_t) * (size_t)count);
    };
    for (int32_t l = 0; l < L; l++) {
        HostLevel &H = lv[(size_t)l];
        int32_t sz[2];
        KP_TRY(get(f, sz, sizeof sz));
        H.n = sz[0];
        H.nnz = sz[1];
        if (wide_file) KP_TRY(get(f, &H.nnz, sizeof H.nnz));
        if (H.n < 0 || H.nnz < 0 || (l > 0 && H.n > lv[(size_t)l - 1].n))
            return set_error(KP_ERR_INVALID, "bad level sizes in hierarchy file");
        if (H.nnz >= NNZ_LIMIT)
            return set_error(KP_ERR_OVERFLOW, "a level of the hierarchy file has more entries than this library's offsets hold");
        if (wide_file) {
            if (!room((int64_t)sizeof(int64_t) * ((int64_t)H.n + 1)))
                return set_error(KP_ERR_INVALID, "truncated hierarchy file");
            H.xadj.resize((size_t)H.n + 1);
            KP_TRY(get(f, H.xadj.data(), sizeof(int64_t) * H.xadj.size()));
        } else {
            std::vector<int32_t> x32;
            KP_TRY(rd(x32, (int64_t)H.n + 1));
            H.xadj.assign(x32.begin(), x32.end());
        }
        KP_TRY(rd(H.adjncy, H.nnz));
        KP_TRY(rd(H.ewgt, H.nnz));
        KP_TRY(rd(H.vwgt, H.n));
        if (l < L - 1) KP_TRY(rd(H.map, H.n));
        if (G > 0) KP_TRY(rd(H.goff, (int64_t)G + 1));
    }
    std::vector<int32_t> glevels, gid0;
    if (G > 0) {
        KP_TRY(rd(glevels, G));
        KP_TRY(rd(gid0, lv[0].n));
    }
    char extra;
    if (fread(&extra, 1, 1, f) != 0) return set_error(KP_ERR_INVALID, "trailing bytes in hierarchy file");
    for (int32_t l = 0; l < L; l++) {
        const HostLevel &H = lv[(size_t)l];
        bool ok = H.xadj[0] == 0 && H.xadj[(size_t)H.n] == H.nnz;
        for (int32_t v = 0; ok && v < H.n; v++) ok = H.xadj[(size_t)v] <= H.xadj[(size_t)v + 1];
        for (int64_t e = 0; ok && e < H.nnz; e++) ok = H.adjncy[(size_t)e] >= 0 && H.adjncy[(size_t)e] < H.n;
        if (G > 0) {
            ok = ok && H.goff[0] == 0 && H.goff[(size_t)G] == H.n;
            for (int32_t g = 0; ok && g < G; g++) ok = H.goff[(size_t)g] <= H.goff[(size_t)g + 1];
        } else if (l < L - 1) {
            // one graph: every node is carried to the next level
            const int32_t n2 = lv[(size_t)l + 1].n;
            for (int32_t v = 0; ok && v < H.n; v++) ok = H.map[(size_t)v] >= 0 && H.map[(size_t)v] < n2;
        }
        if (!ok) return set_error(KP_ERR_INVALID, "inconsistent level in hierarchy file");
    }
    for (int32_t v : glevels)
        if (v < 1 || v > L) return set_error(KP_ERR_INVALID, "bad graph level count in hierarchy file");
    if (G > 0) {
        // the projection follows a node's maps inside its own graph: the
        // input node of graph g lies in g's range of level 0 and carries g's
        // id; on every level before g's coarsest, g's nodes map into g's range
        // of the next level.  On g's coarsest and later levels a map is never
        // followed: -1 (not carried), or into g's range (the copy a level that
        // matched nothing leaves behind)
        for (int32_t g = 0; g < G; g++)
            for (int32_t v = lv[0].goff[(size_t)g]; v < lv[0].goff[(size_t)g + 1]; v++)
                if (gid0[(size_t)v] != g) return set_error(KP_ERR_INVALID, "bad graph id in hierarchy file");
        for (int32_t l = 0; l + 1 < L; l++) {
            const HostLevel &H = lv[(size_t)l], &N = lv[(size_t)l + 1];
            for (int32_t g = 0; g < G; g++) {
                const bool carried = l < glevels[(size_t)g] - 1;
                const int32_t lo = N.goff[(size_t)g], hi = N.goff[(size_t)g + 1];
                for (int32_t v = H.goff[(size_t)g]; v < H.goff[(size_t)g + 1]; v++) {
                    const int32_t m = H.map[(size_t)v];
                    const bool inside = m >= lo && m < hi;
                    if (carried ? !inside : !(inside || m == -1))
                        return set_error(KP_ERR_INVALID, "map leaves its graph in hierarchy file");
                }
            }
        }
    }

    // the offsets in this library's width (every value is below NNZ_LIMIT)
    std::vector<std::vector<eoff>> xs((size_t)L);
    for (int32_t l = 0; l < L; l++) xs[(size_t)l].assign(lv[(size_t)l].xadj.begin(), lv[(size_t)l].xadj.end());

    kp_hierarchy *h = new kp_hierarchy();
    try {
        return upload_hierarchy(h, lv, xs, glevels, gid0, L, G, s, out);
    } catch (...) {
        kp_hierarchy_free(h);
        throw;
    }
}

// The host buffers of a large file may not fit host memory: an allocation
// failure is an error code, not an exception leaving the C ABI.
extern "C" kp_status kp_hierarchy_save(const kp_hierarchy *h, const char *path) {
    try {
        return hierarchy_save_impl(h, path);
    } catch (const std::bad_alloc &) {
        return set_error(KP_ERR_OOM, "host buffer for the hierarchy file");
    }
}

extern "C" kp_status kp_hierarchy_load(const char *path, kp_stream stream, kp_hierarchy **out) {
    try {
        return hierarchy_load_impl(path, stream, out);
    } catch (const std::bad_alloc &) {
        if (out) *out = nullptr;
        return set_error(KP_ERR_OOM, "host buffer for the hierarchy file");
    }
}
