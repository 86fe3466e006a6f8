// Device-side state of the coarsening engine, shared by the matching and the
// contraction translation units.
//
// The level loop is driven from device memory: a table of level descriptors
// (sizes, array pointers, flags), per-level counters and a bump arena from
// which coarse levels are carved once their sizes are known on the device.
// Every kernel of level l reads its sizes and pointers from the table, skips
// itself when level l is not being contracted, and the stop rule is decided
// on the device, so the host can enqueue levels ahead without waiting.
#pragma once

#include "kp_internal.cuh"

// Read-only loads.  A persistent launch (the tail kernel) reads data that
// other blocks wrote earlier in the same launch, so its translation unit
// defines KP_COHERENT_LOADS: no read-only cache path, no __restrict__
// aliasing promises, and (with -dlcm=cg) every global load served from L2.
#ifdef KP_COHERENT_LOADS
#define KP_LDG(p) (*(p))
#define KP_RESTRICT
#else
#define KP_LDG(p) __ldg(p)
#define KP_RESTRICT __restrict__
#endif

namespace kp {

constexpr int32_t SENT = 0x7fffffff;   // sorts after every node id
constexpr int MID_MAX = 2048;          // longest row handled in shared memory
constexpr int SORT_SHARED_DEFAULT = 256;   // kp_options.sort_shared_max = 0
constexpr int MATCH_BLOCK = 256;
constexpr int CONTRACT_BLOCK = 256;
constexpr int MAX_LEVELS = 128;        // level table size (kp_options.max_levels <= 120)
// proposals: rows up to SUITOR_WARP_ROW that the first pass parks are
// searched by one warp each, longer ones by one block each; rows longer than
// SUITOR_CACHE_ROW keep up to SUITOR_CACHE_K candidates between searches
constexpr int32_t SUITOR_WARP_ROW = 1024;
constexpr int32_t SUITOR_CACHE_ROW = 4096;
constexpr int SUITOR_CACHE_K = 8;
// contraction: rows of more gathered entries than this are sorted by a
// thread-block cluster each (levels launched one kernel per phase)
constexpr int32_t HUGE_ROW = 32768;

// level flags
enum : int32_t { LV_ACTIVE = 1, LV_BUILT = 2, LV_NOMATCH = 4 };

struct Counters {   // one per level, zeroed before the level runs
    GridBarrier bar;
    int32_t err;
    int32_t list_size[4];  // proposals: [0],[1] middle pass list and counter, [2],[3] wide pass
    int32_t rounds;
    int32_t cn;            // coarse node count
    eoff U;                // sum of coarse row upper bounds
    int32_t nclass[7];     // class lists: [1] <=32, [2] <=128, [3] <=MID_MAX, [4] longer, [5] > huge_row,
                           // [6] 129..warp_row (taken out of [3] where a warp kernel runs)
    eoff nnz_out;          // coarse entry count
    int32_t tile_counter[2];
    int32_t maxdeg;        // largest coarse degree if it is at least 1024, else 0
    unsigned long long searches;     // rating passes over a row
    unsigned long long failed_cas;   // lost proposal races
    unsigned long long start_next;   // proposals: next start node handed to a warp
    int32_t class_next[2];           // contraction: next row of classes 3 and 4 handed to a block
};

struct DevLevel {
    int32_t n, flags;
    eoff nnz, U;
    eoff *xadj;
    int32_t *adjncy, *ewgt, *vwgt;
    int32_t *map;    // to level l+1 (-1: the node's graph has stopped)
    int32_t *outw;   // Out(v) (innerOuter only)
    int32_t *gid;    // batches: graph of each node
    int32_t *goff;   // batches: first node of each graph, [num_graphs+1]
};

// What the host needs to steer the loop, written by the device into mapped
// pinned host memory when a level ends (no copy on the stream).
struct LevelSnap {
    int32_t stop;
    int32_t cn;
    eoff nnz;
    int32_t done;
    unsigned long long room;   // arena bytes left after the level
    int32_t arena_gen;         // spare chunks taken so far
    int32_t maxdeg;            // Counters::maxdeg of the level
};

struct DevState {
    DevLevel lv[MAX_LEVELS];
    Counters ctr[MAX_LEVELS];
    char *arena;
    unsigned long long arena_cap, arena_used;
    // a spare chunk the host supplies ahead of need (stream-ordered copy of
    // these two words); the arena continues there when a carve does not fit
    char *arena_next;
    unsigned long long arena_next_cap;
    int32_t stop_size, max_levels, min_shrink_permille, inner_outer;
    int32_t stop;       // coarsening has ended
    int32_t overflow;   // 1 + the level whose arrays did not fit the arena
    int32_t err;        // ERR_TIMEOUT from a bounded wait
    int32_t suitor_lanes;      // 0: from the mean degree
    int32_t sort_shared_max;   // longest row sorted in shared memory
    int32_t radix_bits;        // bits per radix pass (4..8)
    int32_t tail_resume;       // first level left to the cluster tail (-1: none)
    int32_t arena_gen;         // spare chunks taken so far
    int32_t maxdeg0;           // the input's largest degree (level 0's start)
    int32_t maxdeg0_warps;     // warps that have added theirs
    LevelSnap *snap;    // host-mapped, one per level
    GridBarrier tail_bar;
};

// Ends the loop: the level is not contracted further and the host is told.
__device__ __forceinline__ void stop_at(DevState *st, int level, int32_t err_bits) {
    if (err_bits) atomicOr(&st->err, err_bits);
    atomicAnd(&st->lv[level].flags, ~LV_ACTIVE);
    st->stop = 1;
    volatile LevelSnap *s = st->snap + level;
    s->stop = 1;
    s->done = 1;
}

// Offer record of node u for the proposal matching (16 bytes, one 128-bit
// CAS): current suitor s (-1 none), omega(s,u), rating attribute of s, and
// u's own rating attribute (c, or Out for innerOuter).
struct __align__(16) Offer {
    int32_t s;
    int32_t w;
    int32_t as;
    int32_t au;
};

// Decoupled look-back scan status of one tile; the flag carries the scan's
// epoch so the array never needs clearing between scans.
struct TileStatus {
    unsigned long long agg;
    unsigned long long incl;
    int32_t flag;   // (epoch << 2) | 1 aggregate ready, | 2 inclusive prefix ready
    int32_t pad;
};

// Scratch sized for level 0 and reused by every level.
struct Work {
    Offer *offer;
    int32_t *match, *cand, *list0, *list1;
    int32_t *first, *second, *degp;
    eoff *off;   // slot of every coarse row in tmp/big (upper bounds, scanned)
    int32_t *tmp_adj, *tmp_w, *big_adj, *big_w;
    int32_t *lists[7];
    // proposals: candidate caches of the rows searched by the wide pass,
    // one slot per entry of list1 (wslot: node -> slot, checked on use)
    int32_t *wslot;
    int2 *cache;       // SUITOR_CACHE_K candidates {node, edge weight} per slot
    int2 *cache_hdr;   // per slot {candidates kept, next to try}
    int32_t cache_slots;
    // Global Path Algorithm: the collected neighbours of every node (two
    // slots, -1 empty), per directed entry whether the edge was refused for
    // closing an odd cycle, the other end of a cycle's closing edge, the
    // dynamic programme's take flags, and the pending cycle checks with their
    // decisions
    int32_t *gnb;
    uint8_t *grej;
    int32_t *gclose;
    uint8_t *gtake;
    int32_t *gpend;
    int8_t *gdec;
    int32_t *ghub;   // rows of more than GPA_HUB_ROW entries (at most nnz / GPA_HUB_ROW)
    // the input's largest degree + 1, written by level 0's start into mapped
    // host memory (null: not wanted)
    int32_t *deg0_host;
    TileStatus *status;
    uint64_t seed;
    long long spin_limit;
    // batches of independent graphs (batch = 0: one graph)
    int32_t batch;
    int32_t num_graphs;
    const uint64_t *seeds;   // per graph, or null: `seed` for all
    const int32_t *stops;    // per graph stop sizes, or null: the state's for all
    int32_t *gactive;        // per graph: contracted at the current level
    int32_t *glevels;        // per graph: levels of its hierarchy (input included)
};

// Tie-break hash context of a node: the seed of its graph and the id offset
// that makes ids graph-local, so a graph's result does not depend on where it
// sits in a batch.
struct HashCtx {
    uint64_t seed;
    int32_t base;
};

__device__ __forceinline__ HashCtx hash_ctx(const Work &w, const DevLevel &L, int32_t v) {
    HashCtx h;
    h.seed = w.seed;
    h.base = 0;
    if (w.batch) {
        const int32_t g = L.gid[v];
        if (w.seeds) h.seed = w.seeds[g];
        h.base = L.goff[g];
    }
    return h;
}

__device__ __forceinline__ uint64_t edge_hash_in(const HashCtx &h, int32_t u, int32_t v) {
    return edge_hash(h.seed, u - h.base, v - h.base);
}

// ---------------------------------------------------------------------------
// ratings (Section 3.1) as exact fractions
// ---------------------------------------------------------------------------
// The rating of an edge of weight w whose ends carry attributes a and b
// (c for the c-based ratings, Out for innerOuter); symmetric in a and b.
template <int R>
__device__ __forceinline__ void rating_ab(int32_t w, int32_t a, int32_t b, uint64_t &num, uint64_t &den) {
    const uint64_t W = (uint64_t)(uint32_t)w;
    if (R == KP_RATING_EXPANSION_STAR2) {
        num = W * W;
        den = (uint64_t)(uint32_t)a * (uint64_t)(uint32_t)b;
    } else if (R == KP_RATING_INNER_OUTER) {
        num = W;
        den = (uint64_t)((int64_t)a + (int64_t)b - 2 * (int64_t)w);
    } else if (R == KP_RATING_WEIGHT) {
        num = W;
        den = 1;
    } else if (R == KP_RATING_EXPANSION) {
        num = W;
        den = (uint64_t)(uint32_t)a + (uint64_t)(uint32_t)b;
    } else {
        num = W;
        den = (uint64_t)(uint32_t)a * (uint64_t)(uint32_t)b;
    }
}

template <int R>
__device__ __forceinline__ int32_t rating_attr(const int32_t *vwgt, const int32_t *outw, int32_t v) {
    if (R == KP_RATING_INNER_OUTER) return outw[v];
    if (R == KP_RATING_WEIGHT) return 0;
    return vwgt[v];
}

// A candidate edge {v,u} seen from v.
struct Cand {
    uint64_t num, den, h;
    int32_t u;
};

// Strict order: higher rating, then higher hash, then smaller (min,max) ids.
__device__ __forceinline__ bool better(const Cand &a, const Cand &b, int32_t v) {
    if (b.u < 0) return a.u >= 0;
    if (a.u < 0) return false;
    const int c = cmp_frac(a.num, a.den, b.num, b.den);
    if (c != 0) return c > 0;
    if (a.h != b.h) return a.h > b.h;
    const int32_t alo = min(v, a.u), ahi = max(v, a.u), blo = min(v, b.u), bhi = max(v, b.u);
    if (alo != blo) return alo < blo;
    return ahi < bhi;
}

// ---------------------------------------------------------------------------
// memory-model helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ int ld_acquire_i32(const int32_t *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_i32(int32_t *p, int v) {
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed_u64(unsigned long long *p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Before a level carves anything (one thread): when the rest of the arena
// may be too small for the level's arrays (`need` bytes at most), continue
// in the spare chunk the host supplied, if there is one and it is large
// enough.  Arrays carved before stay where they are.
__device__ __forceinline__ void arena_reserve(DevState *st, unsigned long long need) {
    if (st->arena_used + need <= st->arena_cap || !st->arena_next || need > st->arena_next_cap) return;
    st->arena = st->arena_next;
    st->arena_cap = st->arena_next_cap;
    st->arena_used = 0;
    st->arena_next = nullptr;
    st->arena_next_cap = 0;
    st->arena_gen++;
}

// Carves `bytes` (256-byte aligned) from the arena; nullptr when full.
__device__ __forceinline__ char *arena_carve(DevState *st, unsigned long long bytes) {
    const unsigned long long b = (bytes + 255ull) & ~255ull;
    const unsigned long long at = st->arena_used;
    if (at + b > st->arena_cap) return nullptr;
    st->arena_used = at + b;
    return st->arena + at;
}

// ---------------------------------------------------------------------------
// single-pass exclusive scan (decoupled look-back) over 64-bit values
//   bool     Op::prepare()                 false: the level is not active
//   int64_t  Op::count()
//   int32_t *Op::tile_counter()            zero before the scan
//   uint64_t Op::load(int64_t i)
//   void     Op::store(int64_t i, uint64_t excl, uint64_t v)
//   void     Op::total(uint64_t t)         once, with the sum of all items
//   void     Op::fail()                    a look-back wait ran out
// Tiles are taken in order from a counter, so every tile's predecessors are
// held by running blocks; each wait for a predecessor is bounded.  The look
// back reads 32 predecessors at a time (one per lane of the first warp).
// ---------------------------------------------------------------------------
// Returns false when a look-back wait gave up (op.fail() has been called).
template <class Op>
__device__ bool scan_lb_phase(Op &op, TileStatus *status, int32_t epoch, long long spin_limit) {
    __shared__ int64_t s_tile;
    __shared__ unsigned long long s_prefix;
    __shared__ int s_abort;
    if (!op.prepare()) return true;
    const int64_t count = op.count();
    const int64_t tiles = (count + SCAN_TILE - 1) / SCAN_TILE;
    if (tiles == 0) {
        if (blockIdx.x == 0 && threadIdx.x == 0) op.total(0);
        return true;
    }
    int32_t *counter = op.tile_counter();
    for (;;) {
        if (threadIdx.x == 0) s_tile = atomicAdd(counter, 1);
        __syncthreads();
        const int64_t tile = s_tile;
        __syncthreads();
        if (tile >= tiles) break;
        const int64_t base = tile * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
        uint64_t v[SCAN_ITEMS];
        uint64_t sum = 0;
#pragma unroll
        for (int j = 0; j < SCAN_ITEMS; j++) {
            v[j] = base + j < count ? op.load(base + j) : 0;
            sum += v[j];
        }
        uint64_t total;
        const uint64_t excl = block_exclusive_scan<SCAN_BLOCK>(sum, &total);
        if (threadIdx.x < 32) {
            // the first warp publishes the tile and looks back over its
            // predecessors 32 at a time (lane i reads tile base - i); the
            // nearest one with an inclusive prefix ends the walk, the
            // aggregates of those after it are added
            const int lane = threadIdx.x;
            unsigned long long prefix = 0;
            int ok = 1;
            TileStatus *me = status + tile;
            if (tile == 0) {
                if (lane == 0) {
                    st_relaxed_u64(&me->incl, total);
                    st_release_i32(&me->flag, (epoch << 2) | 2);
                }
            } else {
                if (lane == 0) {
                    st_relaxed_u64(&me->agg, total);
                    st_release_i32(&me->flag, (epoch << 2) | 1);
                }
                int64_t base = tile - 1;
                long long it = 0;
                for (;;) {
                    const int64_t j = base - lane;
                    const int f = j >= 0 ? ld_acquire_i32(&status[j].flag) : ((epoch << 2) | 2);
                    const bool ready = (f >> 2) == epoch && (f & 3) != 0;
                    if (!__all_sync(0xffffffffu, ready)) {   // the same decision in every lane
                        if (++it > spin_limit) {
                            ok = 0;
                            break;
                        }
                        __nanosleep(32);
                        continue;
                    }
                    // tile 0 is inclusive, so a window that reaches it finds one
                    const unsigned inc = __ballot_sync(0xffffffffu, j >= 0 && (f & 3) == 2);
                    const int stop = inc ? __ffs(inc) - 1 : 32;
                    unsigned long long v = 0;
                    if (j >= 0 && lane < stop) v = ld_relaxed_u64(&status[j].agg);
                    if (j >= 0 && lane == stop) v = ld_relaxed_u64(&status[j].incl);
#pragma unroll
                    for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
                    prefix += v;
                    if (inc) break;
                    base -= 32;
                }
                if (lane == 0 && ok) {
                    st_relaxed_u64(&me->incl, prefix + total);
                    st_release_i32(&me->flag, (epoch << 2) | 2);
                }
            }
            if (lane == 0) {
                s_prefix = prefix;
                s_abort = !ok;
                if (!ok) op.fail();
                else if (tile == tiles - 1) op.total(prefix + total);
            }
        }
        __syncthreads();
        if (s_abort) return false;
        uint64_t p = s_prefix + excl;
#pragma unroll
        for (int j = 0; j < SCAN_ITEMS; j++) {
            if (base + j < count) op.store(base + j, p, v[j]);
            p += v[j];
        }
        __syncthreads();
    }
    return true;
}

template <class Op>
__global__ void __launch_bounds__(SCAN_BLOCK) k_scan_lb(Op op, TileStatus *status, int32_t epoch,
                                                        long long spin_limit) {
    scan_lb_phase(op, status, epoch, spin_limit);
}

// ---------------------------------------------------------------------------
// launchers (host), defined in match.cu and contract.cu
// ---------------------------------------------------------------------------
struct LevelLaunch {
    DevState *st;
    Work w;
    int level;
    int rating;
    int matcher;
    int suitor_blocks;   // 3 or 4 (0: 3): the first proposal pass's register budget
    int32_t n_bound;     // upper bound of the level's node count (grid sizes)
    int64_t nnz_bound;   // upper bound of its entry count
    bool huge;           // rows of more than HUGE_ROW gathered entries are possible
    int32_t epoch_relabel, epoch_degscan;
};

kp_status launch_graph_ids(int32_t n0, int32_t num_graphs, const int32_t *goff, int32_t *gid, cudaStream_t s,
                           int32_t *launches);
kp_status launch_check_batch_edges(const kp_graph *g, const int32_t *gid, const int32_t *goff, int32_t *flag,
                                   cudaStream_t s);
kp_status launch_out_weight(DevState *st, int32_t n0, int64_t nnz0, const eoff *xadj, const int32_t *ewgt,
                            int32_t *outw, cudaStream_t s, int32_t *launches);
kp_status launch_matching(const LevelLaunch &L, cudaStream_t s, int32_t *launches);
kp_status launch_relabel(const LevelLaunch &L, cudaStream_t s, int32_t *launches);
kp_status launch_contract(const LevelLaunch &L, cudaStream_t s, int32_t *launches);
kp_status launch_csr(const LevelLaunch &L, cudaStream_t s, int32_t *launches);
// The persistent tail from level `first`: levels above cluster_nodes in one
// cooperative grid (block_nodes nodes per block), the later ones in one
// thread-block cluster with hardware barriers (cluster_nodes < 0: no
// cluster part; the grid part hands over through DevState::tail_resume).
struct TailLaunch {
    int first, last;
    int32_t n_bound;
    int32_t block_nodes;
    int32_t cluster_nodes;
    int32_t epoch0;
};
kp_status launch_tail(DevState *st, const Work &w, int rating, int matcher, const TailLaunch &t, cudaStream_t s,
                      int32_t *launches);

}  // namespace kp
