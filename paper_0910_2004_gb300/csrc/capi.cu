// C ABI entry points (include/kp.h), error state, allocation and the
// device-side input check of Section 2's requirements (omega > 0, c >= 0,
// undirected graph stored symmetrically, no self loops).
#include <atomic>
#include <cstdio>
#include <mutex>
#include <new>
#include <string>

#include "kp_internal.cuh"

namespace kp {

namespace {
// a fixed buffer per thread: reporting an error allocates nothing, so it
// also works when a host allocation is what failed
thread_local char g_last_error[2048];
}

kp_status set_error(kp_status st, const char *msg) {
    snprintf(g_last_error, sizeof g_last_error, "%s", msg ? msg : "");
    return st;
}

kp_status set_error(kp_status st, const std::string &msg) { return set_error(st, msg.c_str()); }

kp_status cuda_error(cudaError_t e, const char *what) {
    cudaGetLastError();   // clear a non-sticky error
    char buf[512];
    snprintf(buf, sizeof buf, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
    return set_error(e == cudaErrorMemoryAllocation ? KP_ERR_OOM : KP_ERR_CUDA, buf);
}

int num_sms() {
    static std::atomic<int> cached[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
    int c = cached[dev].load(std::memory_order_relaxed);
    if (c == 0) {
        int v = 0;
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        c = v > 0 ? v : 1;
        cached[dev].store(c, std::memory_order_relaxed);
    }
    return c;
}

// Test hook: the allocation after `g_fail_after` more successful ones fails
// with KP_ERR_OOM (-1: never), then the hook switches itself off.
static std::mutex g_inject_mu;
static int64_t g_fail_after = -1;

static bool injected_failure() {
    std::lock_guard<std::mutex> lock(g_inject_mu);
    if (g_fail_after < 0) return false;
    if (g_fail_after == 0) {
        g_fail_after = -1;
        return true;
    }
    g_fail_after--;
    return false;
}

kp_status dev_alloc(void **p, size_t bytes, cudaStream_t s) {
    static std::mutex mu;
    static std::atomic<bool> configured[64];
    int dev = 0;
    KP_CUDA(cudaGetDevice(&dev));
    if (dev >= 0 && dev < 64 && !configured[dev]) {
        std::lock_guard<std::mutex> lock(mu);
        if (!configured[dev]) {
            cudaMemPool_t pool;
            if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
                uint64_t threshold = ~0ull;   // keep freed blocks for reuse
                cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &threshold);
            }
            configured[dev] = true;
        }
    }
    if (injected_failure()) {
        *p = nullptr;
        return set_error(KP_ERR_OOM, "injected allocation failure");
    }
    const cudaError_t e = cudaMallocAsync(p, bytes, s);
    if (e != cudaSuccess) {
        *p = nullptr;
        return cuda_error(e, "cudaMallocAsync");
    }
    return KP_OK;
}

void dev_free(void *p, cudaStream_t s) {
    if (p) cudaFreeAsync(p, s);
}

ArenaObserver &arena_observer() {
    thread_local ArenaObserver o;
    return o;
}

// ---------------------------------------------------------------------------
// input check
// ---------------------------------------------------------------------------
struct CheckAcc {
    unsigned long long csum;
    unsigned long long wsum;
    int32_t err;
    int32_t pad;
};

// Input check in two kernels.  Nodes: row bounds, c >= 0 and the sum of c.
__global__ void k_validate_nodes(int32_t n, eoff nnz, const eoff *__restrict__ xadj,
                                 const int32_t *__restrict__ vwgt, CheckAcc *acc) {
    int bad = 0;
    unsigned long long csum = 0;
    if (blockIdx.x == 0 && threadIdx.x == 0 && (xadj[0] != 0 || xadj[n] != nnz)) bad = 1;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const eoff beg = xadj[v], end = xadj[v + 1];
        if (beg < 0 || end < beg || end > nnz) bad = 1;
        const int32_t c = vwgt[v];
        if (c < 0) bad = 1;
        else csum += (unsigned long long)c;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) csum += __shfl_xor_sync(0xffffffffu, csum, o);
    if ((threadIdx.x & 31) == 0 && csum) atomicAdd(&acc->csum, csum);
    if (bad) atomicOr(&acc->err, ERR_GRAPH_INVALID);
}

// Entries, in chunks of VALIDATE_CHUNK consecutive ones per thread, so hub
// rows spread over many threads: the row of the chunk's first entry by a
// binary search over xadj, then for every entry: neighbour in range, no self
// loop, omega > 0, the row ascending, and the reverse entry with the same
// weight (a binary search in the neighbour's row).  Every index is checked
// before it is used, whatever the input (the node kernel reports bad rows).
constexpr int VALIDATE_CHUNK = 8;

__global__ void k_validate_entries(int32_t n, eoff nnz, const eoff *__restrict__ xadj,
                                   const int32_t *__restrict__ adjncy, const int32_t *__restrict__ ewgt,
                                   CheckAcc *acc) {
    int bad = 0;
    unsigned long long wsum = 0;
    const int64_t chunks = ((int64_t)nnz + VALIDATE_CHUNK - 1) / VALIDATE_CHUNK;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < chunks; c += stride) {
        const int64_t e0 = c * VALIDATE_CHUNK, e1 = min((int64_t)nnz, e0 + VALIDATE_CHUNK);
        int32_t lo = 0, hi = n - 1;   // the last row starting at or before e0
        while (lo < hi) {
            const int32_t mid = lo + (hi - lo + 1) / 2;
            if ((int64_t)xadj[mid] <= e0) lo = mid;
            else hi = mid - 1;
        }
        int32_t v = lo;
        for (int64_t e = e0; e < e1; e++) {
            while (v + 1 < n && (int64_t)xadj[v + 1] <= e) v++;
            const int32_t u = adjncy[e];
            const int32_t w = ewgt[e];
            if (u < 0 || u >= n || u == v || w <= 0) {
                bad = 1;
                continue;
            }
            if (e > 0 && e > xadj[v] && adjncy[e - 1] >= u) bad = 1;
            eoff a = xadj[u], b = xadj[u + 1] - 1;
            if (a < 0 || b >= nnz) {
                bad = 1;
                continue;
            }
            eoff found = -1;
            while (a <= b) {
                const eoff mid = a + (b - a) / 2;
                const int32_t t = adjncy[mid];
                if (t == v) {
                    found = mid;
                    break;
                }
                if (t < v) a = mid + 1;
                else b = mid - 1;
            }
            if (found < 0 || ewgt[found] != w) bad = 1;
            if (u > v) wsum += (unsigned long long)w;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) wsum += __shfl_xor_sync(0xffffffffu, wsum, o);
    if ((threadIdx.x & 31) == 0 && wsum) atomicAdd(&acc->wsum, wsum);
    if (bad) atomicOr(&acc->err, ERR_GRAPH_INVALID);
}

kp_status validate_graph(const kp_graph *g, cudaStream_t s, int64_t) {
    CheckAcc *acc = nullptr;
    KP_TRY(dev_alloc_n(&acc, 1, s));
    thread_local CheckAcc *host = nullptr;
    if (!host && cudaMallocHost((void **)&host, sizeof(CheckAcc)) != cudaSuccess) {
        host = nullptr;
        dev_free(acc, s);
        return set_error(KP_ERR_OOM, "pinned host buffer");
    }
    cudaError_t e = cudaMemsetAsync(acc, 0, sizeof(CheckAcc), s);
    if (e == cudaSuccess) {
        const int cap = num_sms() * 16;
        const int grid_n = (int)std::max<int64_t>(1, std::min<int64_t>(((int64_t)g->n + 255) / 256, cap));
        const int64_t chunks = ((int64_t)g->nnz + VALIDATE_CHUNK - 1) / VALIDATE_CHUNK;
        const int grid_e = (int)std::max<int64_t>(1, std::min<int64_t>((chunks + 255) / 256, cap));
        k_validate_nodes<<<grid_n, 256, 0, s>>>(g->n, g->nnz, g->xadj, g->vwgt, acc);
        if (g->nnz > 0) k_validate_entries<<<grid_e, 256, 0, s>>>(g->n, g->nnz, g->xadj, g->adjncy, g->ewgt, acc);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(host, acc, sizeof(CheckAcc), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    dev_free(acc, s);
    if (e != cudaSuccess) return cuda_error(e, "graph check");
    if (host->err) return set_error(KP_ERR_INVALID, "graph is not a valid symmetric sorted CSR with omega > 0, c >= 0");
    if (host->csum >= (1ull << 31)) return set_error(KP_ERR_OVERFLOW, "sum of node weights >= 2^31");
    if (host->wsum >= (1ull << 31)) return set_error(KP_ERR_OVERFLOW, "sum of edge weights >= 2^31");
    return KP_OK;
}

kp_status project_impl(const kp_hierarchy *h, const int32_t *coarse_part, int32_t *fine_part, cudaStream_t s);
kp_status project_batch_impl(const kp_hierarchy *h, const int32_t *coarse_part, const int32_t *coarse_offsets,
                             int32_t *fine_part, cudaStream_t s);
kp_status batch_coarsest_impl(const kp_hierarchy *h, int32_t *sizes, cudaStream_t s);
kp_status cut_gain_impl(const kp_graph *g, const int32_t *part, int32_t k, double eps, kp_cut_gain_out *out,
                        cudaStream_t s);
kp_status cut_gain_noalloc_impl(const kp_graph *g, const int32_t *part, int32_t k, double eps,
                                kp_cut_gain_out *out, cudaStream_t s);
kp_status pipeline_host_impl(const kp_graph *hg, const kp_options *o, int32_t k, double eps,
                             kp_initial_partition_fn ip, void *user, int32_t *fine_part, int64_t *gain,
                             int32_t *target, int64_t *block_w, kp_cut_gain_out *out, int32_t *num_levels,
                             cudaStream_t s);

}  // namespace kp

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
using namespace kp;

#define KP_GUARD(expr)                                              \
    try {                                                           \
        return (expr);                                              \
    } catch (const std::bad_alloc &) {                              \
        return set_error(KP_ERR_OOM, "host allocation failed");     \
    } catch (...) {                                                 \
        return set_error(KP_ERR_CUDA, "unexpected exception");      \
    }

extern "C" {

void kp_options_default(kp_options *o) {
    if (!o) return;
    o->rating = KP_RATING_EXPANSION_STAR2;
    o->seed = 1;
    o->stop_size = 40;
    o->max_levels = 64;
    o->min_shrink_permille = 50;
    o->spin_limit = 1ll << 22;
    o->validate = 1;
    o->profile = 0;
    o->matcher = KP_MATCHER_SUITOR;
    o->arena_bytes = 0;
    o->tail_nodes = 0;
    o->suitor_lanes = 0;
    o->suitor_blocks = 0;
    o->tail_block_nodes = 0;
    o->sort_shared_max = 0;
    o->radix_bits = 0;
    o->cluster_nodes = 0;
}

kp_status kp_coarsen(const kp_graph *g, const kp_options *o, kp_stream s, kp_hierarchy **out) {
    kp::TraceRange trace("kp_coarsen");
    if (!g || !out) return set_error(KP_ERR_INVALID, "null argument");
    *out = nullptr;
    kp_options def;
    kp_options_default(&def);
    if (o && o->max_levels > 120) return set_error(KP_ERR_UNSUPPORTED, "max_levels above 120");
    g_last_error[0] = 0;
    KP_GUARD(coarsen_impl(g, o ? o : &def, (cudaStream_t)s, out));
}

kp_status kp_coarsen_batch(const kp_graph *g, int32_t num_graphs, const int32_t *node_offsets,
                           const uint64_t *seeds, const int32_t *stop_sizes, const kp_options *o, kp_stream s,
                           kp_hierarchy **out) {
    kp::TraceRange trace("kp_coarsen_batch");
    if (!g || !out) return set_error(KP_ERR_INVALID, "null argument");
    *out = nullptr;
    kp_options def;
    kp_options_default(&def);
    if (o && o->max_levels > 120) return set_error(KP_ERR_UNSUPPORTED, "max_levels above 120");
    g_last_error[0] = 0;
    BatchSpec b;
    b.num_graphs = num_graphs;
    b.node_offsets = node_offsets;
    b.seeds = seeds;
    b.stop_sizes = stop_sizes;
    KP_GUARD(coarsen_impl(g, o ? o : &def, (cudaStream_t)s, out, &b));
}

kp_status kp_hierarchy_batch(const kp_hierarchy *h, int32_t *num_graphs, int32_t *levels) {
    if (!h) return set_error(KP_ERR_INVALID, "null argument");
    if (num_graphs) *num_graphs = h->num_graphs;
    if (levels)
        for (int32_t i = 0; i < h->num_graphs; i++) levels[i] = h->glevels[(size_t)i];
    return KP_OK;
}

kp_status kp_hierarchy_batch_coarsest(const kp_hierarchy *h, int32_t *sizes, kp_stream s) {
    KP_GUARD(batch_coarsest_impl(h, sizes, (cudaStream_t)s));
}

kp_status kp_hierarchy_level_offsets(const kp_hierarchy *h, int32_t l, const int32_t **node_offsets) {
    if (!h || !node_offsets) return set_error(KP_ERR_INVALID, "null argument");
    if (h->num_graphs == 0) return set_error(KP_ERR_INVALID, "not a batch hierarchy");
    if (l < 0 || l >= (int32_t)h->levels.size()) return set_error(KP_ERR_INVALID, "level out of range");
    *node_offsets = h->levels[(size_t)l].goff;
    return KP_OK;
}

kp_status kp_project_batch(const kp_hierarchy *h, const int32_t *coarse_part, const int32_t *coarse_offsets,
                           int32_t *fine_part, kp_stream s) {
    kp::TraceRange trace("kp_project_batch");
    KP_GUARD(project_batch_impl(h, coarse_part, coarse_offsets, fine_part, (cudaStream_t)s));
}

kp_status kp_hierarchy_num_levels(const kp_hierarchy *h, int32_t *num_levels) {
    if (!h || !num_levels) return set_error(KP_ERR_INVALID, "null argument");
    *num_levels = (int32_t)h->levels.size();
    return KP_OK;
}

kp_status kp_hierarchy_level(const kp_hierarchy *h, int32_t l, kp_graph *view, const int32_t **map) {
    if (!h || !view) return set_error(KP_ERR_INVALID, "null argument");
    if (l < 0 || l >= (int32_t)h->levels.size()) return set_error(KP_ERR_INVALID, "level out of range");
    const kp_level &L = h->levels[(size_t)l];
    view->n = L.n;
    view->nnz = L.nnz;
    view->xadj = L.xadj;
    view->adjncy = L.adjncy;
    view->ewgt = L.ewgt;
    view->vwgt = L.vwgt;
    if (map) *map = L.map;
    return KP_OK;
}

kp_status kp_hierarchy_stats(const kp_hierarchy *h, int32_t *total_rounds, int64_t *total_matched) {
    if (!h) return set_error(KP_ERR_INVALID, "null argument");
    if (total_rounds) *total_rounds = h->total_rounds;
    if (total_matched) *total_matched = h->total_matched;
    return KP_OK;
}

kp_status kp_hierarchy_profile(const kp_hierarchy *h, int32_t l, kp_level_profile *out) {
    if (!h || !out) return set_error(KP_ERR_INVALID, "null argument");
    if (l == -1) {
        *out = h->total;
        return KP_OK;
    }
    if (l < 0 || l >= (int32_t)h->per_level.size()) return set_error(KP_ERR_INVALID, "level out of range");
    *out = h->per_level[(size_t)l];
    return KP_OK;
}

void kp_hierarchy_free(kp_hierarchy *h) {
    if (!h) return;
    for (void *p : h->allocations) dev_free(p, h->stream);
    cudaStreamSynchronize(h->stream);
    delete h;
}

kp_status kp_project(const kp_hierarchy *h, const int32_t *coarse_part, int32_t *fine_part, kp_stream s) {
    kp::TraceRange trace("kp_project");
    KP_GUARD(project_impl(h, coarse_part, fine_part, (cudaStream_t)s));
}

kp_status kp_cut_gain(const kp_graph *g, const int32_t *part, int32_t k, double eps, kp_cut_gain_out *out,
                      kp_stream s) {
    kp::TraceRange trace("kp_cut_gain");
    KP_GUARD(cut_gain_impl(g, part, k, eps, out, (cudaStream_t)s));
}

kp_status kp_cut_gain_noalloc(const kp_graph *g, const int32_t *part, int32_t k, double eps,
                              kp_cut_gain_out *out, kp_stream s) {
    KP_GUARD(cut_gain_noalloc_impl(g, part, k, eps, out, (cudaStream_t)s));
}

kp_status kp_pipeline_host(const kp_graph *g, const kp_options *o, int32_t k, double eps,
                           kp_initial_partition_fn ip, void *user, int32_t *fine_part, int64_t *gain,
                           int32_t *target, int64_t *block_w, kp_cut_gain_out *out, int32_t *num_levels,
                           kp_stream s) {
    kp::TraceRange trace("kp_pipeline_host");
    kp_options def;
    kp_options_default(&def);
    if (o && o->max_levels > 120) return set_error(KP_ERR_UNSUPPORTED, "max_levels above 120");
    KP_GUARD(pipeline_host_impl(g, o ? o : &def, k, eps, ip, user, fine_part, gain, target, block_w, out,
                                num_levels, (cudaStream_t)s));
}

const char *kp_last_error(void) { return g_last_error; }

const char *kp_version(void) {
    return KP_OFFSET_BITS == 64 ? "kp-gb300 0.1 (sm_103a, 64-bit offsets)" : "kp-gb300 0.1 (sm_103a)";
}

int32_t kp_offset_bits(void) { return KP_OFFSET_BITS; }

}  // extern "C"

extern "C" void kp_test_fail_allocation(int64_t after) {
    std::lock_guard<std::mutex> lock(kp::g_inject_mu);
    kp::g_fail_after = after < 0 ? -1 : after;
}

extern "C" int64_t kp_test_device_bytes_in_use(void) {
    int dev = 0;
    cudaMemPool_t pool;
    uint64_t used = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetDefaultMemPool(&pool, dev) != cudaSuccess ||
        cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used) != cudaSuccess)
        return -1;
    return (int64_t)used;
}
