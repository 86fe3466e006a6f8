// Internal declarations shared by the library's translation units.
// Device helpers: exact rating comparison, tie-break hash, a bounded grid
// barrier for persistent kernels, and the block-wide scan of the scans.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "kp.h"

namespace kp {

// A named range on the host timeline for tracing tools (NVTX; free when no
// tool is attached): entry points, levels, server groups.
struct TraceRange {
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};

}  // namespace kp

namespace kp {

// Entry offsets and counts (CSR row offsets, entry indices, nnz): int32 in
// the default build, int64 in the wide build (KP_WIDE_OFFSETS).  Node ids,
// degrees and weights stay int32 in both.
using eoff = kp_eoff;
// Inputs have nnz below this: the int32 range, or in the wide build 2^32
// (nnz = 2|E|, omega >= 1 and the sum of omega below 2^31).
constexpr int64_t NNZ_LIMIT = KP_OFFSET_BITS == 64 ? (1ll << 32) : (1ll << 31);

// ---------------------------------------------------------------------------
// error state (host)
// ---------------------------------------------------------------------------
kp_status set_error(kp_status st, const char *msg);
kp_status set_error(kp_status st, const std::string &msg);
kp_status cuda_error(cudaError_t e, const char *what);

#define KP_CUDA(call)                                                  \
    do {                                                               \
        cudaError_t _e = (call);                                       \
        if (_e != cudaSuccess) return ::kp::cuda_error(_e, #call);     \
    } while (0)

#define KP_TRY(call)                                                   \
    do {                                                               \
        kp_status _s = (call);                                         \
        if (_s != KP_OK) return _s;                                    \
    } while (0)

int num_sms();

// A batch of independent graphs stored as one disjoint union.
struct BatchSpec {
    int32_t num_graphs;
    const int32_t *node_offsets;   // device [num_graphs+1]: graph i is [off[i], off[i+1])
    const uint64_t *seeds;         // device [num_graphs] or null
    const int32_t *stop_sizes = nullptr;   // device [num_graphs] or null
};

kp_status coarsen_impl(const kp_graph *g, const kp_options *o, cudaStream_t s, kp_hierarchy **out,
                       const BatchSpec *batch = nullptr);

// Stream-ordered device allocation from the device's default memory pool
// (its release threshold is raised once so freed blocks are reused).
kp_status dev_alloc(void **p, size_t bytes, cudaStream_t s);
void dev_free(void *p, cudaStream_t s);

// Device bytes a coarsening takes beyond its first arena (spare chunks for
// slowly shrinking graphs, a larger arena after an overflow) are reported to
// this thread's observer, if one is set (the request server charges them to
// its device budget while the allocation is in use).
struct ArenaObserver {
    void (*grew)(void *ctx, int64_t bytes) = nullptr;
    void *ctx = nullptr;
};
ArenaObserver &arena_observer();
inline void report_arena_growth(int64_t bytes) {
    ArenaObserver &o = arena_observer();
    if (o.grew) o.grew(o.ctx, bytes);
}

template <class T>
kp_status dev_alloc_n(T **p, int64_t count, cudaStream_t s) {
    return dev_alloc(reinterpret_cast<void **>(p), sizeof(T) * (size_t)(count > 0 ? count : 1), s);
}

// ---------------------------------------------------------------------------
// device-side status flags
// ---------------------------------------------------------------------------
enum : int32_t {
    ERR_TIMEOUT = 1,
    ERR_BAD_PART = 2,
    ERR_GRAPH_INVALID = 4,
};

// ---------------------------------------------------------------------------
// exact comparison of ratings num/den (Section 3.1)
// ---------------------------------------------------------------------------
// a/b against c/d by the 128-bit cross products a*d and c*b.  Numerators are
// > 0 and denominators >= 0, so a zero denominator (rating +infinity) wins
// against any finite rating and ties with another infinity.  When all four
// fit in 32 bits (small weights: the common case), the products fit in 64
// bits and are formed by single widening multiplies (not in the persistent
// tail's unit, KP_FRAC_WIDE_ONLY: at its register cap the extra branch
// measured slower there).
__device__ __forceinline__ int cmp_frac(uint64_t a, uint64_t b, uint64_t c, uint64_t d) {
#ifndef KP_FRAC_WIDE_ONLY
    if (((a | b | c | d) >> 32) == 0) {
        const uint64_t l = (uint64_t)(uint32_t)a * (uint32_t)d, r = (uint64_t)(uint32_t)c * (uint32_t)b;
        return (l > r) - (l < r);
    }
#endif
    const uint64_t lh = __umul64hi(a, d), ll = a * d;
    const uint64_t rh = __umul64hi(c, b), rl = c * b;
    if (lh != rh) return lh > rh ? 1 : -1;
    if (ll != rl) return ll > rl ? 1 : -1;
    return 0;
}

// splitmix64 output function (Steele, Lea, Flood, OOPSLA 2014).
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
    uint64_t z = x + 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ uint64_t edge_hash(uint64_t seed, int32_t u, int32_t v) {
    const uint32_t lo = (uint32_t)min(u, v), hi = (uint32_t)max(u, v);
    return splitmix64(seed ^ (((uint64_t)lo << 32) | hi));
}

// ---------------------------------------------------------------------------
// bounded grid barrier for cooperative (co-resident) grids
// ---------------------------------------------------------------------------
struct GridBarrier {
    unsigned int count;
    unsigned int generation;
};

__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int *p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_u32(unsigned int *p, unsigned int v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ int ld_relaxed_i32(const int32_t *p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// All blocks of the grid meet here.  Returns false (and every block returns
// false soon after) when a wait exceeded spin_limit iterations or another
// block already flagged an error; the error flag then holds ERR_TIMEOUT.
__device__ __forceinline__ unsigned cluster_ctas() {
    unsigned r;
    asm("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ void cluster_barrier() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// A word every block of a one-cluster grid reads with the same value: read
// between two cluster barriers (no block writes it in between).
__device__ __forceinline__ int32_t cluster_uniform_read(const int32_t *p) {
    cluster_barrier();
    const int32_t v = ld_relaxed_i32(p);
    cluster_barrier();
    return v;
}

__device__ __forceinline__ bool grid_sync(GridBarrier *bar, int32_t *err, long long spin_limit) {
    __shared__ int s_ok;
    if (gridDim.x == 1) {   // one block: a block barrier is a grid barrier
        __syncthreads();
        return ld_relaxed_i32(err) == 0;
    }
    if (cluster_ctas() == gridDim.x) {
        // the grid is one thread-block cluster: the hardware cluster barrier
        // (release/acquire at cluster scope; every CTA of a cluster is
        // resident together).  The error flag is read between two barriers,
        // where no block runs a phase, so every block takes the same
        // decision and none leaves while the others wait.
        cluster_barrier();
        const bool ok = ld_relaxed_i32(err) == 0;
        cluster_barrier();
        return ok;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned int gen = ld_acquire_u32(&bar->generation);
        // arrive: acquire-release at gpu scope.  Releasing covers the writes
        // of the whole block (ordered before by the block barrier above); the
        // last arriver has acquired every earlier arrival through the
        // counter's read-modify-write chain and releases them all with the
        // new generation, which the waiters acquire.
        unsigned int arrived;
        asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], 1;" : "=r"(arrived) : "l"(&bar->count) : "memory");
        if (arrived == gridDim.x - 1) {
            atomicExch(&bar->count, 0u);
            st_release_u32(&bar->generation, gen + 1);
        } else {
            long long it = 0;
            while (ld_acquire_u32(&bar->generation) == gen) {
                if (ld_relaxed_i32(err) != 0) { ok = 0; break; }
                if (++it > spin_limit) {
                    atomicOr(err, ERR_TIMEOUT);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        if (ok && ld_relaxed_i32(err) != 0) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// ---------------------------------------------------------------------------
// warp helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Mask of the G-lane group that contains this lane (G divides 32).
template <int G>
__device__ __forceinline__ unsigned group_mask() {
    if constexpr (G == 32) {
        return 0xffffffffu;
    } else {
        const unsigned lane = threadIdx.x & 31u;
        return ((1u << G) - 1u) << (lane & ~(unsigned)(G - 1));
    }
}

// ---------------------------------------------------------------------------
// tiles of the device-wide scans (engine.cuh: single pass, decoupled
// look-back) and the block-wide exclusive scan they use
// ---------------------------------------------------------------------------
constexpr int SCAN_BLOCK = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_BLOCK * SCAN_ITEMS;

template <int BLOCK>
__device__ __forceinline__ uint64_t block_exclusive_scan(uint64_t v, uint64_t *total) {
    __shared__ uint64_t warp_sums[BLOCK / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t x = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        uint64_t y = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint64_t s = lane < BLOCK / 32 ? warp_sums[lane] : 0;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            uint64_t y = __shfl_up_sync(0xffffffffu, s, d);
            if (lane >= d) s += y;
        }
        if (lane < BLOCK / 32) warp_sums[lane] = s;
    }
    __syncthreads();
    const uint64_t warp_prefix = warp > 0 ? warp_sums[warp - 1] : 0;
    *total = warp_sums[BLOCK / 32 - 1];
    __syncthreads();
    return warp_prefix + x - v;
}

inline int64_t scan_tiles(int64_t count) { return (count + SCAN_TILE - 1) / SCAN_TILE; }

}  // namespace kp

// The hierarchy handle (opaque to C callers).
struct kp_level {
    int32_t n = 0;
    kp_eoff nnz = 0;
    kp_eoff *xadj = nullptr;
    int32_t *adjncy = nullptr;
    int32_t *ewgt = nullptr;
    int32_t *vwgt = nullptr;
    int32_t *map = nullptr;   // to the next level; nullptr on the coarsest
    int32_t *goff = nullptr;  // batches: first node of each graph on this level
    bool owned = false;
};

struct kp_hierarchy {
    std::vector<kp_level> levels;
    std::vector<void *> allocations;
    cudaStream_t stream = nullptr;
    int device = 0;
    int32_t total_rounds = 0;
    int64_t total_matched = 0;
    kp_level_profile total = {};
    std::vector<kp_level_profile> per_level;
    // batches of independent graphs
    int32_t num_graphs = 0;             // 0: one graph
    std::vector<int32_t> glevels;       // per graph: number of levels
    int32_t *glevels_dev = nullptr;     // the same on the device
    int32_t *gid0 = nullptr;            // graph of every input node (device)
};

namespace kp {

// Records CUDA events at phase boundaries on one stream when enabled; the
// elapsed times are summed per phase once the stream has been synchronised.
class PhaseTimer {
  public:
    PhaseTimer(bool on, cudaStream_t s) : on_(on), s_(s) {}
    ~PhaseTimer() {   // the events go back to this thread's pool
        for (auto &m : marks_) pool().push_back(m.ev);
    }
    // Starts `phase_starting` (-1: only ends the running interval) of level
    // `level` (-1: outside the level loop).
    void mark(int phase_starting, int level = -1) {
        if (!on_) return;
        cudaEvent_t e;
        if (!pool().empty()) {
            e = pool().back();
            pool().pop_back();
        } else if (cudaEventCreate(&e) != cudaSuccess) {
            return;
        }
        cudaEventRecord(e, s_);
        marks_.push_back({e, phase_starting, level});
    }
    // After the stream is synchronised: add each interval to the phase that
    // began at its start mark, per level and in total.
    void accumulate(kp_level_profile *total, std::vector<kp_level_profile> &levels) {
        for (size_t i = 0; i + 1 < marks_.size(); i++) {
            if (marks_[i].phase < 0) continue;
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, marks_[i].ev, marks_[i + 1].ev) != cudaSuccess) continue;
            total->phase_ms[marks_[i].phase] += ms;
            const int l = marks_[i].level;
            if (l >= 0 && l < (int)levels.size()) levels[(size_t)l].phase_ms[marks_[i].phase] += ms;
        }
    }

  private:
    // Events are created once per thread and reused (creating one per mark
    // costs host time inside the enqueue loop).  They belong to the device
    // that was current when they were made; the pool is per thread.
    static std::vector<cudaEvent_t> &pool() {
        thread_local std::vector<cudaEvent_t> p;
        return p;
    }
    struct Mark {
        cudaEvent_t ev;
        int phase;
        int level;
    };
    bool on_;
    cudaStream_t s_;
    std::vector<Mark> marks_;
};

}  // namespace kp
