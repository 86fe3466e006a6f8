// Contraction phase host engine: the level loop of the multilevel scheme
// (Section 2) with its stop rule (Section 4: contract until the graph is small
// enough), driven through the device level table of engine.cuh.
//
// Per level the stream carries: level begin (+ Out at level 0 for
// innerOuter), matching (Section 3.3), relabel scan, contraction, degree scan
// and compaction (Section 2).  The stop rule is decided on the device, which
// also writes a small per-level record into mapped host memory; the host
// enqueues up to LOOKAHEAD levels beyond the last one it has seen finish and
// never waits per level.  Levels enqueued after the stop find themselves
// inactive and return at once.  If the arena runs out, the device stops at
// the level that did not fit; the host adds a larger arena and resumes there.
#include <algorithm>
#include <cstdio>
#include <atomic>
#include <cstring>

#include "engine.cuh"

namespace kp {

namespace {

constexpr int LOOKAHEAD = 2;
// Levels with at most this many nodes run in the persistent tail launch
// (default of kp_options.tail_nodes).
constexpr int32_t TAIL_NODES = 1 << 18;

std::atomic<int> g_coop_supported{-1};

struct Scratch {
    cudaStream_t s = nullptr;
    std::vector<void *> ptrs;
    template <class T>
    kp_status get(T **p, int64_t count) {
        KP_TRY(dev_alloc_n(p, count, s));
        ptrs.push_back(*p);
        return KP_OK;
    }
    ~Scratch() {
        for (void *p : ptrs) dev_free(p, s);
    }
};

// Host side of the device state, in pinned memory; the snapshots are mapped
// so the device can write them directly.
struct HostMirror {
    DevState *state = nullptr;
    LevelSnap *snap = nullptr;
    LevelSnap *snap_dev = nullptr;
    int32_t *deg0 = nullptr, *deg0_dev = nullptr;   // the input's largest degree + 1 (0: not yet)
    HostMirror() {
        if (cudaMallocHost((void **)&state, sizeof(DevState)) != cudaSuccess) state = nullptr;
        if (cudaHostAlloc((void **)&snap, sizeof(LevelSnap) * MAX_LEVELS, cudaHostAllocMapped) != cudaSuccess)
            snap = nullptr;
        if (snap && cudaHostGetDevicePointer((void **)&snap_dev, snap, 0) != cudaSuccess) snap_dev = nullptr;
        if (cudaHostAlloc((void **)&deg0, sizeof(int32_t), cudaHostAllocMapped) != cudaSuccess) deg0 = nullptr;
        if (deg0 && cudaHostGetDevicePointer((void **)&deg0_dev, deg0, 0) != cudaSuccess) deg0_dev = nullptr;
    }
    ~HostMirror() {
        if (state) cudaFreeHost(state);
        if (snap) cudaFreeHost(snap);
        if (deg0) cudaFreeHost(deg0);
    }
};

unsigned long long align256(unsigned long long b) { return (b + 255ull) & ~255ull; }

}  // namespace

// Device scratch of the level loop, sized for level 0 (every later level is
// smaller), and the device state.
kp_status alloc_work(Scratch &sc, Work &w, int32_t n0, eoff nnz0, const kp_options *o, const BatchSpec *batch,
                     int32_t *glevels_dev, DevState **dst) {
    std::memset(&w, 0, sizeof w);
    if (o->matcher == KP_MATCHER_SUITOR) {
        KP_TRY(sc.get(&w.offer, n0));
        // list1 holds rows longer than the middle pass's limit only
        w.cache_slots = (int32_t)std::min<int64_t>((int64_t)n0, (int64_t)nnz0 / SUITOR_WARP_ROW + 2);
        KP_TRY(sc.get(&w.wslot, n0));
        KP_TRY(sc.get(&w.cache, (int64_t)w.cache_slots * SUITOR_CACHE_K));
        KP_TRY(sc.get(&w.cache_hdr, w.cache_slots));
    } else {
        KP_TRY(sc.get(&w.match, n0));
        KP_TRY(sc.get(&w.cand, n0));
    }
    if (o->matcher == KP_MATCHER_GPA) {
        KP_TRY(sc.get(&w.gnb, 2 * (int64_t)n0));
        KP_TRY(sc.get(&w.grej, nnz0));
        KP_TRY(sc.get(&w.gclose, n0));
        KP_TRY(sc.get(&w.gtake, n0));
        KP_TRY(sc.get(&w.gpend, n0));
        KP_TRY(sc.get(&w.gdec, n0));
        KP_TRY(sc.get(&w.ghub, (int64_t)nnz0 / 2048 + 1));   // rows longer than GPA_HUB_ROW = 2048
    }
    KP_TRY(sc.get(&w.list0, n0));
    KP_TRY(sc.get(&w.list1, n0));
    KP_TRY(sc.get(&w.first, n0));
    KP_TRY(sc.get(&w.second, n0));
    KP_TRY(sc.get(&w.off, (int64_t)n0 + 1));
    KP_TRY(sc.get(&w.degp, n0));
    KP_TRY(sc.get(&w.tmp_adj, nnz0));
    KP_TRY(sc.get(&w.tmp_w, nnz0));
    KP_TRY(sc.get(&w.big_adj, nnz0));
    KP_TRY(sc.get(&w.big_w, nnz0));
    for (int c = 1; c <= 4; c++) KP_TRY(sc.get(&w.lists[c], n0));
    KP_TRY(sc.get(&w.lists[6], n0));
    KP_TRY(sc.get(&w.lists[5], (int64_t)nnz0 / HUGE_ROW + 2));   // each such row holds more than HUGE_ROW entries
    KP_TRY(sc.get(&w.status, scan_tiles(n0) + 1));
    KP_TRY(sc.get(dst, 1));
    w.seed = o->seed;
    w.spin_limit = o->spin_limit;
    if (batch) {
        w.batch = 1;
        w.num_graphs = batch->num_graphs;
        w.seeds = batch->seeds;
        w.stops = batch->stop_sizes;
        w.glevels = glevels_dev;
        KP_TRY(sc.get(&w.gactive, batch->num_graphs));
    }
    return KP_OK;
}

// Levels with at most this many nodes run in one thread-block cluster
// (-1: never).
int32_t cluster_nodes_of(const kp_options *o) { return o->cluster_nodes == 0 ? 8192 : o->cluster_nodes; }

unsigned long long initial_arena(const kp_options *o, int32_t n0, eoff nnz0) {
    unsigned long long cap =
        o->arena_bytes > 0
            ? align256((unsigned long long)o->arena_bytes)
            : align256((60ull + sizeof(eoff)) * (unsigned long long)n0 + 32ull * (unsigned long long)nnz0 + (1ull << 20));
    if (o->rating == KP_RATING_INNER_OUTER)   // Out of the input lives at the arena's start
        cap = std::max<unsigned long long>(cap, align256(4ull * (unsigned long long)n0) + 4096);
    return cap;
}

// Host image of the device state before level 0: the input as level 0, the
// arena, the options the kernels read.
void init_state(DevState *hs, const kp_graph *g, const kp_options *o, const BatchSpec *batch, int32_t *gid0,
                char *arena, unsigned long long arena_cap, LevelSnap *snap_dev) {
    const bool inner_outer = o->rating == KP_RATING_INNER_OUTER;
    std::memset(hs, 0, sizeof(DevState));
    DevLevel &L0 = hs->lv[0];
    L0.n = g->n;
    L0.nnz = g->nnz;
    L0.U = g->nnz;
    // one graph is contracted at all only above the stop size; the graphs of
    // a batch decide for themselves at the level start
    const bool active0 = batch ? true : (g->n > o->stop_size && o->max_levels > 0);
    L0.flags = LV_BUILT | (active0 ? LV_ACTIVE : 0);
    L0.xadj = const_cast<eoff *>(g->xadj);
    L0.adjncy = const_cast<int32_t *>(g->adjncy);
    L0.ewgt = const_cast<int32_t *>(g->ewgt);
    L0.vwgt = const_cast<int32_t *>(g->vwgt);
    if (batch) {
        L0.gid = gid0;
        L0.goff = const_cast<int32_t *>(batch->node_offsets);
    }
    hs->arena = arena;
    hs->arena_cap = arena_cap;
    hs->arena_used = 0;
    if (inner_outer) {
        L0.outw = (int32_t *)arena;
        hs->arena_used = align256(4ull * (unsigned long long)g->n);
    }
    hs->stop_size = o->stop_size;
    hs->max_levels = o->max_levels;
    hs->min_shrink_permille = o->min_shrink_permille;
    hs->inner_outer = inner_outer ? 1 : 0;
    hs->suitor_lanes = o->suitor_lanes;
    // built in: rows above 256 gathered entries take the radix passes, which
    // measured faster there than the shared-memory and register networks
    // (power-law graphs; grids have few such rows)
    hs->sort_shared_max = o->sort_shared_max ? o->sort_shared_max : SORT_SHARED_DEFAULT;
    hs->radix_bits = o->radix_bits ? o->radix_bits : 8;
    hs->tail_resume = -1;
    hs->snap = snap_dev;
}

// The coarse levels, maps, batch offsets and per-level counters from the
// device state read back after the loop (h holds level 0 already).
kp_status assemble_hierarchy(kp_hierarchy *h, const DevState *hs, bool suitor, int32_t G,
                             const int32_t *level_launches, cudaStream_t s) {
    int last = 0;
    while (last + 1 < MAX_LEVELS && (hs->lv[last + 1].flags & LV_BUILT)) last++;
    for (int l = 1; l <= last; l++) {
        const DevLevel &D = hs->lv[l];
        kp_level kl;
        kl.n = D.n;
        kl.nnz = D.nnz;
        kl.xadj = D.xadj;
        kl.adjncy = D.adjncy;
        kl.ewgt = D.ewgt;
        kl.vwgt = D.vwgt;
        kl.owned = true;
        h->levels.push_back(kl);
    }
    for (int l = 0; l < last; l++) h->levels[(size_t)l].map = hs->lv[l].map;
    h->levels[(size_t)last].map = nullptr;
    if (G > 0) {
        for (int l = 1; l <= last; l++) h->levels[(size_t)l].goff = hs->lv[l].goff;
        h->glevels.resize((size_t)G);
        KP_CUDA(cudaMemcpyAsync(h->glevels.data(), h->glevels_dev, sizeof(int32_t) * (size_t)G,
                                cudaMemcpyDeviceToHost, s));
        KP_CUDA(cudaStreamSynchronize(s));
    }
    h->per_level.assign((size_t)last, kp_level_profile{});
    int32_t total_rounds = 0;
    int64_t total_matched = 0;
    for (int l = 0; l < last; l++) {
        kp_level_profile &P = h->per_level[(size_t)l];
        const Counters &C = hs->ctr[l];
        P.n = hs->lv[l].n;
        P.nnz = hs->lv[l].nnz;
        P.rounds = suitor ? 1 : C.rounds;
        P.searches = (int64_t)C.searches;
        P.failed_cas = (int64_t)C.failed_cas;
        P.launches = level_launches ? level_launches[l] : 0;
        total_rounds += P.rounds;
        total_matched += (int64_t)hs->lv[l].n - hs->lv[l + 1].n;
    }
    h->total_rounds = total_rounds;
    h->total_matched = total_matched;
    return KP_OK;
}

kp_status validate_graph(const kp_graph *g, cudaStream_t s, int64_t spin_limit);

// Sizes and arrays of an input graph, checked on the host whether or not
// the graph itself is checked.  nnz = 2|E| and omega >= 1 with the sum of
// omega below 2^31 bound nnz below 2^32, which the coarse row bounds of the
// relabel scan rely on (their sum is kept in 32 bits).
kp_status check_graph_sizes(const kp_graph *g) {
    if (g->n < 0 || g->nnz < 0) return set_error(KP_ERR_INVALID, "negative graph size");
    if ((int64_t)g->nnz >= NNZ_LIMIT) return set_error(KP_ERR_OVERFLOW, "nnz >= 2^32: the edge weights sum to 2^31 or more");
    if (g->n > 0 && (!g->xadj || !g->vwgt || (g->nnz > 0 && (!g->adjncy || !g->ewgt))))
        return set_error(KP_ERR_INVALID, "null graph array");
    return KP_OK;
}

kp_status coarsen_impl(const kp_graph *g, const kp_options *o, cudaStream_t s, kp_hierarchy **out,
                       const BatchSpec *batch) {
    const int rating = o->rating;
    if (rating < 0 || rating > 4) return set_error(KP_ERR_UNSUPPORTED, "unknown rating");
    if (o->matcher != KP_MATCHER_SUITOR && o->matcher != KP_MATCHER_HANDSHAKE && o->matcher != KP_MATCHER_GPA)
        return set_error(KP_ERR_UNSUPPORTED, "unknown matcher");
    KP_TRY(check_graph_sizes(g));
    if (o->max_levels < 0 || o->max_levels > MAX_LEVELS - 8 || o->min_shrink_permille < 0 ||
        o->min_shrink_permille > 1000 || o->spin_limit <= 0 || o->arena_bytes < 0 || o->tail_nodes < -1)
        return set_error(KP_ERR_INVALID, "bad option value");
    if (!(o->suitor_lanes == 0 || o->suitor_lanes == 1 || o->suitor_lanes == 2 || o->suitor_lanes == 4 ||
          o->suitor_lanes == 8 || o->suitor_lanes == 32) ||
        (o->tail_block_nodes != 0 && (o->tail_block_nodes < 256 || o->tail_block_nodes > 16384)) ||
        (o->sort_shared_max != 0 && (o->sort_shared_max < 128 || o->sort_shared_max > MID_MAX)) ||
        (o->radix_bits != 0 && (o->radix_bits < 4 || o->radix_bits > 8)) || o->cluster_nodes < -1 ||
        !(o->suitor_blocks == 0 || o->suitor_blocks == 3 || o->suitor_blocks == 4))
        return set_error(KP_ERR_INVALID, "bad tuning knob");
    if (o->matcher == KP_MATCHER_HANDSHAKE || o->matcher == KP_MATCHER_GPA) {
        if (g_coop_supported < 0) {
            int dev = 0, v = 0;
            KP_CUDA(cudaGetDevice(&dev));
            KP_CUDA(cudaDeviceGetAttribute(&v, cudaDevAttrCooperativeLaunch, dev));
            g_coop_supported = v;
        }
        if (!g_coop_supported) return set_error(KP_ERR_UNSUPPORTED, "device lacks cooperative launch");
    }
    const int32_t G = batch ? batch->num_graphs : 0;
    std::vector<int32_t> host_off;
    if (batch) {   // the node ranges of the graphs must tile [0, n)
        if (G < 1 || !batch->node_offsets) return set_error(KP_ERR_INVALID, "batch needs num_graphs >= 1 and offsets");
        host_off.resize((size_t)G + 1);
        KP_CUDA(cudaMemcpyAsync(host_off.data(), batch->node_offsets, sizeof(int32_t) * ((size_t)G + 1),
                                cudaMemcpyDeviceToHost, s));
        KP_CUDA(cudaStreamSynchronize(s));
        if (host_off[0] != 0 || host_off[(size_t)G] != g->n) return set_error(KP_ERR_INVALID, "batch offsets must run from 0 to n");
        for (int32_t i = 0; i < G; i++)
            if (host_off[(size_t)i + 1] < host_off[(size_t)i])
                return set_error(KP_ERR_INVALID, "batch offsets must not decrease");
    }
    PhaseTimer timer(o->profile != 0, s);
    int32_t launches = 0;
    if (o->validate && g->n > 0) {
        timer.mark(KP_PHASE_VALIDATE);
        KP_TRY(validate_graph(g, s, o->spin_limit));
        timer.mark(-1);
        launches += 1;
    }

    kp_hierarchy *h = new kp_hierarchy();
    h->stream = s;
    h->num_graphs = G;
    KP_CUDA(cudaGetDevice(&h->device));
    kp_level l0;
    l0.n = g->n;
    l0.nnz = g->nnz;
    l0.xadj = const_cast<eoff *>(g->xadj);
    l0.adjncy = const_cast<int32_t *>(g->adjncy);
    l0.ewgt = const_cast<int32_t *>(g->ewgt);
    l0.vwgt = const_cast<int32_t *>(g->vwgt);
    l0.owned = false;
    h->levels.push_back(l0);
    auto fail = [&](kp_status st) {
        kp_hierarchy_free(h);
        return st;
    };
    const int32_t n0 = g->n;
    const eoff nnz0 = g->nnz;
    const bool suitor = o->matcher == KP_MATCHER_SUITOR;
    const bool inner_outer = rating == KP_RATING_INNER_OUTER;
    const bool active0 = batch ? true : (n0 > o->stop_size && o->max_levels > 0);
    h->levels[0].goff = batch ? const_cast<int32_t *>(batch->node_offsets) : nullptr;
    if (batch) {   // per-graph level counts (1 until a graph is contracted)
        h->glevels.assign((size_t)G, 1);
        kp_status st0 = dev_alloc_n(&h->glevels_dev, G, s);
        if (st0 != KP_OK) return fail(st0);
        h->allocations.push_back(h->glevels_dev);
        st0 = dev_alloc_n(&h->gid0, n0, s);
        if (st0 != KP_OK) return fail(st0);
        h->allocations.push_back(h->gid0);
        if (cudaMemcpyAsync(h->glevels_dev, h->glevels.data(), sizeof(int32_t) * (size_t)G, cudaMemcpyHostToDevice,
                            s) != cudaSuccess)
            return fail(cuda_error(cudaGetLastError(), "upload graph levels"));
        if (n0 > 0) {
            st0 = launch_graph_ids(n0, G, batch->node_offsets, h->gid0, s, &launches);
            if (st0 != KP_OK) return fail(st0);
        }
        if (o->validate && n0 > 0) {   // every edge stays inside its graph
            int32_t *flag = nullptr;
            st0 = dev_alloc_n(&flag, 1, s);
            if (st0 != KP_OK) return fail(st0);
            int32_t hflag = 0;
            cudaMemsetAsync(flag, 0, sizeof(int32_t), s);
            st0 = launch_check_batch_edges(g, h->gid0, batch->node_offsets, flag, s);
            if (st0 == KP_OK && (cudaMemcpyAsync(&hflag, flag, sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                                 cudaStreamSynchronize(s) != cudaSuccess))
                st0 = cuda_error(cudaGetLastError(), "batch edge check");
            dev_free(flag, s);
            if (st0 != KP_OK) return fail(st0);
            if (hflag) return fail(set_error(KP_ERR_INVALID, "a batch edge joins two different graphs"));
        }
    }
    if (n0 == 0 || !active0) {
        h->total.n = n0;
        h->total.nnz = nnz0;
        h->total.launches = launches;
        if (cudaStreamSynchronize(s) != cudaSuccess) return fail(cuda_error(cudaGetLastError(), "sync"));
        timer.accumulate(&h->total, h->per_level);
        *out = h;
        return KP_OK;
    }

    // scratch sized for level 0
    Scratch sc;
    sc.s = s;
    Work w;
    DevState *dst = nullptr;
    kp_status st = alloc_work(sc, w, n0, nnz0, o, batch, h->glevels_dev, &dst);
    if (st != KP_OK) return fail(st);
    if (cudaMemsetAsync(w.status, 0, sizeof(TileStatus) * (size_t)(scan_tiles(n0) + 1), s) != cudaSuccess)
        return fail(cuda_error(cudaGetLastError(), "clear scan status"));

    thread_local HostMirror mirror;
    if (!mirror.state || !mirror.snap || !mirror.snap_dev || !mirror.deg0_dev)
        return fail(set_error(KP_ERR_OOM, "pinned host state"));
    *(volatile int32_t *)mirror.deg0 = 0;
    w.deg0_host = mirror.deg0_dev;
    DevState *hs = mirror.state;
    LevelSnap *snap = mirror.snap;

    // the arena for all coarse levels (grown on overflow)
    unsigned long long arena_cap = initial_arena(o, n0, nnz0);
    char *arena = nullptr;
    st = dev_alloc((void **)&arena, arena_cap, s);
    if (st != KP_OK) return fail(st);
    h->allocations.push_back(arena);
    std::memset(snap, 0, sizeof(LevelSnap) * MAX_LEVELS);
    init_state(hs, g, o, batch, h->gid0, arena, arena_cap, mirror.snap_dev);
    DevLevel &L0 = hs->lv[0];
    if (cudaMemcpyAsync(dst, hs, sizeof(DevState), cudaMemcpyHostToDevice, s) != cudaSuccess)
        return fail(cuda_error(cudaGetLastError(), "upload state"));
    if (inner_outer) {
        timer.mark(KP_PHASE_OUT);
        st = launch_out_weight(dst, n0, nnz0, g->xadj, g->ewgt, L0.outw, s, &launches);
        if (st != KP_OK) return fail(st);
    }

    // -1: never (the Global Path Algorithm runs every level on its own)
    const int32_t tail_nodes = o->matcher == KP_MATCHER_GPA ? -1 : o->tail_nodes == 0 ? TAIL_NODES : o->tail_nodes;
    int32_t epoch = 0;
    int start = 0;
    int32_t spares = 0;   // spare arena chunks supplied
    int deg_level = -1;   // level whose largest degree is known (deg_max), -1: none yet
    int64_t deg_max = 0;
    std::vector<int32_t> level_launches(MAX_LEVELS, 0);
    cudaEvent_t ring[LOOKAHEAD + 1];
    for (auto &e : ring)
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess)
            return fail(cuda_error(cudaGetLastError(), "event"));
    auto bail = [&](kp_status e) {
        for (auto &ev : ring) cudaEventDestroy(ev);
        return fail(e);
    };
    for (;;) {   // one pass per arena size
        int32_t n_bound = start == 0 ? n0 : hs->lv[start].n;
        int64_t nnz_bound = start == 0 ? (int64_t)nnz0 : std::max<int64_t>(hs->lv[start].nnz, 1);
        // a batch runs one more level: graphs stopping at the level cap are
        // only recorded at the level after it
        const int level_end = o->max_levels + (batch ? 1 : 0);
        for (int level = start; level < level_end; level++) {
            char trace_name[32];
            snprintf(trace_name, sizeof trace_name, "level %d", level);
            TraceRange trace(trace_name);
            // the rest in one persistent launch once the level is small (dense
            // small levels, as in power-law graphs, stay with the wide grids)
            if (n_bound <= tail_nodes && nnz_bound <= 8ll * tail_nodes) {
                timer.mark(KP_PHASE_TAIL, level);
                const int32_t before = launches;
                TailLaunch t;
                t.first = level;
                t.last = level_end;
                t.n_bound = n_bound;
                t.block_nodes = o->tail_block_nodes ? o->tail_block_nodes : 2048;
                t.cluster_nodes = cluster_nodes_of(o);
                t.epoch0 = epoch;
                st = launch_tail(dst, w, rating, o->matcher, t, s, &launches);
                timer.mark(-1, level);
                if (st != KP_OK) return bail(st);
                level_launches[(size_t)level] += launches - before;
                epoch += 2 * (level_end - level) + 2;
                break;
            }
            LevelLaunch LL;
            LL.st = dst;
            LL.w = w;
            LL.level = level;
            LL.rating = rating;
            LL.matcher = o->matcher;
            LL.suitor_blocks = o->suitor_blocks;
            LL.n_bound = n_bound;
            LL.nnz_bound = nnz_bound;
            // a coarse degree is at most twice the largest of the level
            // before, and a gathered row holds the degrees of two nodes; the
            // input's largest degree arrives from level 0's start (read
            // without waiting: until then the kernel is launched)
            if (deg_level < 0) {
                const int32_t d0 = *(volatile int32_t *)mirror.deg0;
                if (d0 > 0) {
                    deg_level = 0;
                    deg_max = d0 - 1;
                }
            }
            LL.huge = deg_level < 0 || level - deg_level > 20 ||
                      2 * (deg_max << (level - deg_level)) > (int64_t)HUGE_ROW;
            LL.epoch_relabel = ++epoch;
            LL.epoch_degscan = ++epoch;
            const int32_t before = launches;
            timer.mark(KP_PHASE_MATCH, level);
            st = launch_matching(LL, s, &launches);
            if (st == KP_OK) {
                timer.mark(KP_PHASE_RELABEL, level);
                st = launch_relabel(LL, s, &launches);
            }
            if (st == KP_OK) {
                timer.mark(KP_PHASE_CONTRACT, level);
                st = launch_contract(LL, s, &launches);
            }
            if (st == KP_OK) {
                timer.mark(KP_PHASE_CSR, level);
                st = launch_csr(LL, s, &launches);
            }
            timer.mark(-1, level);
            if (st != KP_OK) return bail(st);
            level_launches[(size_t)level] += launches - before;
            if (cudaEventRecord(ring[level % (LOOKAHEAD + 1)], s) != cudaSuccess)
                return bail(cuda_error(cudaGetLastError(), "event record"));
            // wait for the level LOOKAHEAD behind; stop enqueuing once it ended the loop
            const int seen = level - LOOKAHEAD;
            if (seen >= start) {
                if (cudaEventSynchronize(ring[seen % (LOOKAHEAD + 1)]) != cudaSuccess)
                    return bail(cuda_error(cudaGetLastError(), "event sync"));
                const volatile LevelSnap *sn = snap + seen;
                if (sn->stop) break;
                if (sn->done && sn->cn > 0) {   // a tighter bound for the grids
                    n_bound = sn->cn;
                    nnz_bound = std::max<int64_t>((int64_t)sn->nnz, 1);
                    deg_level = seen + 1;   // its largest degree (below 1024 when not recorded)
                    deg_max = std::max<int64_t>(sn->maxdeg, 1023);
                }
                // a spare arena chunk before the levels already enqueued and
                // the next ones could run out (graphs that shrink slowly, as
                // power-law ones do): no restart, no round trip.  A level
                // after `seen` reserves at most 24 bytes per coarse node of
                // `seen` and 8 per coarse entry (maps, weights, CSR); the
                // device moves to the spare when a level's reservation does
                // not fit the rest of the current chunk.
                if (sn->done && sn->arena_gen == spares) {
                    const unsigned long long per_level = 24ull * (unsigned long long)sn->cn +
                                                         8ull * (unsigned long long)sn->nnz +
                                                         4ull * (unsigned long long)(G + 1) + 8192ull;
                    if (sn->room < (LOOKAHEAD + 2) * per_level) {
                        // room for a few more levels of this size (each one
                        // reservation fits it, so no level restarts for it)
                        const unsigned long long cap =
                            align256(std::max<unsigned long long>(arena_cap, (LOOKAHEAD + 4) * per_level));
                        char *chunk = nullptr;
                        st = dev_alloc((void **)&chunk, cap, s);
                        if (st != KP_OK) return bail(st);
                        h->allocations.push_back(chunk);
                        report_arena_growth((int64_t)cap);
                        hs->arena_next = chunk;
                        hs->arena_next_cap = cap;
                        if (cudaMemcpyAsync(&dst->arena_next, &hs->arena_next, sizeof(char *) + sizeof(unsigned long long),
                                            cudaMemcpyHostToDevice, s) != cudaSuccess)
                            return bail(cuda_error(cudaGetLastError(), "spare arena"));
                        spares++;
                    }
                }
            }
        }
        if (cudaStreamSynchronize(s) != cudaSuccess) return bail(cuda_error(cudaGetLastError(), "sync"));
        if (cudaMemcpy(hs, dst, sizeof(DevState), cudaMemcpyDeviceToHost) != cudaSuccess)
            return bail(cuda_error(cudaGetLastError(), "read state"));
        if (hs->err & ERR_TIMEOUT)
            return bail(set_error(KP_ERR_TIMEOUT, suitor ? "a bounded wait gave up (proposal chain or scan look-back)"
                                                         : "a bounded wait gave up (grid barrier or scan look-back)"));
        if (!hs->overflow) break;
        // the arena was too small: resume at the level that did not fit
        const int lo = hs->overflow - 1;
        arena_cap = align256(std::max<unsigned long long>(arena_cap * 2, 2 * hs->arena_used + 4096));
        arena = nullptr;
        st = dev_alloc((void **)&arena, arena_cap, s);
        if (st != KP_OK) return bail(st);
        h->allocations.push_back(arena);
        report_arena_growth((int64_t)arena_cap);
        hs->arena = arena;
        hs->arena_cap = arena_cap;
        hs->arena_used = 0;
        hs->overflow = 0;
        hs->stop = 0;
        hs->tail_resume = -1;
        hs->lv[lo].flags = LV_BUILT | LV_ACTIVE;
        std::memset(&hs->ctr[lo], 0, sizeof(Counters));
        for (int l = lo; l < MAX_LEVELS; l++) {
            snap[l].stop = 0;
            snap[l].done = 0;
        }
        if (cudaMemcpyAsync(dst, hs, sizeof(DevState), cudaMemcpyHostToDevice, s) != cudaSuccess)
            return bail(cuda_error(cudaGetLastError(), "upload state"));
        start = lo;
    }
    for (auto &ev : ring) cudaEventDestroy(ev);

    st = assemble_hierarchy(h, hs, suitor, G, level_launches.data(), s);
    if (st != KP_OK) return fail(st);
    timer.accumulate(&h->total, h->per_level);
    h->total.launches = launches;
    h->total.rounds = h->total_rounds;
    h->total.n = n0;
    h->total.nnz = nnz0;
    for (const auto &lp : h->per_level) {
        h->total.searches += lp.searches;
        h->total.failed_cas += lp.failed_cas;
    }
    *out = h;
    return KP_OK;
}

}  // namespace kp

// ---------------------------------------------------------------------------
// captured plans: the whole hierarchy in one persistent launch, recorded
// once into a CUDA graph and replayed
// ---------------------------------------------------------------------------
struct kp_plan {
    kp_graph g{};
    kp_options o{};
    kp::BatchSpec b{};
    bool batch = false;
    int32_t G = 0;
    int device = 0;
    cudaStream_t s0 = nullptr;   // allocations are stream-ordered on it
    cudaStream_t cap = nullptr;  // capture stream (the default stream cannot capture)
    kp::Scratch sc;
    kp::Work w{};
    kp::DevState *dst = nullptr;
    int32_t *glevels_dev = nullptr, *gid0 = nullptr;
    char *arena = nullptr;
    unsigned long long arena_cap = 0;
    kp::DevState *hs_init = nullptr, *hs_read = nullptr;   // pinned
    kp::LevelSnap *snap = nullptr, *snap_dev = nullptr;    // mapped
    int32_t *glevels_init = nullptr;                       // pinned ones
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int32_t launches = 0;
    int32_t block_nodes = 2048;
    std::vector<std::pair<int32_t, int64_t>> sizes;   // (n, nnz) per level of the checking run
    ~kp_plan() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        kp::dev_free(arena, s0);
        kp::dev_free(glevels_dev, s0);
        kp::dev_free(gid0, s0);
        if (hs_init) cudaFreeHost(hs_init);
        if (hs_read) cudaFreeHost(hs_read);
        if (snap) cudaFreeHost(snap);
        if (glevels_init) cudaFreeHost(glevels_init);
        if (cap) cudaStreamDestroy(cap);
    }
};

namespace kp {

kp_status plan_capture(kp_plan *p) {
    cudaStream_t s = p->cap;
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    p->exec = nullptr;
    p->graph = nullptr;
    p->launches = 0;
    KP_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed));
    kp_status st = KP_OK;
    const int32_t n0 = p->g.n;
    if (cudaMemsetAsync(p->w.status, 0, sizeof(TileStatus) * (size_t)(scan_tiles(n0) + 1), s) != cudaSuccess ||
        cudaMemcpyAsync(p->dst, p->hs_init, sizeof(DevState), cudaMemcpyHostToDevice, s) != cudaSuccess)
        st = cuda_error(cudaGetLastError(), "capture: state");
    if (st == KP_OK && p->batch) {
        if (cudaMemcpyAsync(p->glevels_dev, p->glevels_init, sizeof(int32_t) * (size_t)p->G, cudaMemcpyHostToDevice,
                            s) != cudaSuccess)
            st = cuda_error(cudaGetLastError(), "capture: graph levels");
        if (st == KP_OK) st = launch_graph_ids(n0, p->G, p->b.node_offsets, p->gid0, s, &p->launches);
    }
    if (st == KP_OK && p->o.rating == KP_RATING_INNER_OUTER)
        st = launch_out_weight(p->dst, n0, p->g.nnz, p->g.xadj, p->g.ewgt, p->hs_init->lv[0].outw, s, &p->launches);
    // the levels the checking run found above the tail threshold as separate
    // launches (grids sized by that run's sizes; every kernel covers any
    // size), the rest in one persistent launch
    const int level_end = p->o.max_levels + (p->batch ? 1 : 0);
    const int64_t tail_nodes = p->o.tail_nodes == 0 ? TAIL_NODES : p->o.tail_nodes;
    int K = 0;
    if (p->o.matcher == KP_MATCHER_GPA)   // every level on its own (a replay may run deeper)
        K = level_end;
    else if (tail_nodes >= 0)
        while (K + 1 < (int)p->sizes.size() && K < level_end &&
               !(p->sizes[(size_t)K].first <= tail_nodes && p->sizes[(size_t)K].second <= 8 * tail_nodes))
            K++;
    else
        K = std::min<int>((int)p->sizes.size() - 1, level_end);
    int32_t epoch = 0;
    for (int level = 0; level < K && st == KP_OK; level++) {
        LevelLaunch LL;
        LL.st = p->dst;
        LL.w = p->w;
        LL.level = level;
        LL.rating = p->o.rating;
        LL.matcher = p->o.matcher;
        LL.suitor_blocks = p->o.suitor_blocks;
        const size_t sl = std::min<size_t>((size_t)level, p->sizes.size() - 1);
        LL.n_bound = std::max(p->sizes[sl].first, 1);
        LL.nnz_bound = std::max<int64_t>(p->sizes[sl].second, 1);
        LL.huge = true;   // a replay may meet other degrees than the checking run
        LL.epoch_relabel = ++epoch;
        LL.epoch_degscan = ++epoch;
        st = launch_matching(LL, s, &p->launches);
        if (st == KP_OK) st = launch_relabel(LL, s, &p->launches);
        if (st == KP_OK) st = launch_contract(LL, s, &p->launches);
        if (st == KP_OK) st = launch_csr(LL, s, &p->launches);
    }
    if (st == KP_OK && K < level_end)
    {
        TailLaunch t;
        t.first = K;
        t.last = level_end;
        t.n_bound = std::max(1, p->sizes[(size_t)std::min<int>(K, (int)p->sizes.size() - 1)].first);
        t.block_nodes = p->block_nodes;
        t.cluster_nodes = cluster_nodes_of(&p->o);
        t.epoch0 = epoch;
        st = launch_tail(p->dst, p->w, p->o.rating, p->o.matcher, t, s, &p->launches);
    }
    cudaGraph_t graph = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(s, &graph);
    if (st != KP_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    if (ce != cudaSuccess) return cuda_error(ce, "end capture");
    p->graph = graph;
    KP_CUDA(cudaGraphInstantiate(&p->exec, graph, 0));
    return KP_OK;
}

kp_status plan_create_impl(const kp_graph *g, int32_t num_graphs, const int32_t *node_offsets, const uint64_t *seeds,
                           const int32_t *stop_sizes, const kp_options *o, cudaStream_t s, kp_plan **out) {
    if (g->n <= 0) return set_error(KP_ERR_INVALID, "a plan needs a non-empty graph");
    if (num_graphs < 0) return set_error(KP_ERR_INVALID, "negative num_graphs");
    BatchSpec b;
    b.num_graphs = num_graphs;
    b.node_offsets = node_offsets;
    b.seeds = seeds;
    b.stop_sizes = stop_sizes;
    // checks the options, the batch offsets and (with o->validate) the input
    // once, by an ordinary coarsening; its level sizes size the recorded grids
    kp_options first = *o;
    first.profile = 0;
    kp_hierarchy *h0 = nullptr;
    KP_TRY(coarsen_impl(g, &first, s, &h0, num_graphs > 0 ? &b : nullptr));
    std::vector<std::pair<int32_t, int64_t>> sizes;
    for (const kp_level &l : h0->levels) sizes.emplace_back(l.n, (int64_t)l.nnz);
    kp_hierarchy_free(h0);

    kp_plan *p = new kp_plan();
    p->g = *g;
    p->o = first;
    p->o.validate = 0;
    p->b = b;
    p->batch = num_graphs > 0;
    p->G = num_graphs;
    p->s0 = s;
    p->sc.s = s;
    p->block_nodes = o->tail_block_nodes ? o->tail_block_nodes : 2048;
    p->sizes = sizes;
    auto fail = [&](kp_status st) {
        delete p;
        return st;
    };
    if (cudaGetDevice(&p->device) != cudaSuccess) return fail(cuda_error(cudaGetLastError(), "device"));
    if (cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking) != cudaSuccess)
        return fail(cuda_error(cudaGetLastError(), "capture stream"));
    if (p->batch) {
        kp_status st = dev_alloc_n(&p->glevels_dev, num_graphs, s);
        if (st == KP_OK) st = dev_alloc_n(&p->gid0, g->n, s);
        if (st != KP_OK) return fail(st);
        if (cudaMallocHost((void **)&p->glevels_init, sizeof(int32_t) * (size_t)num_graphs) != cudaSuccess)
            return fail(set_error(KP_ERR_OOM, "pinned graph levels"));
        for (int32_t i = 0; i < num_graphs; i++) p->glevels_init[i] = 1;
    }
    kp_status st = alloc_work(p->sc, p->w, g->n, g->nnz, &p->o, p->batch ? &p->b : nullptr, p->glevels_dev, &p->dst);
    if (st != KP_OK) return fail(st);
    if (cudaMallocHost((void **)&p->hs_init, sizeof(DevState)) != cudaSuccess ||
        cudaMallocHost((void **)&p->hs_read, sizeof(DevState)) != cudaSuccess ||
        cudaHostAlloc((void **)&p->snap, sizeof(LevelSnap) * MAX_LEVELS, cudaHostAllocMapped) != cudaSuccess ||
        cudaHostGetDevicePointer((void **)&p->snap_dev, p->snap, 0) != cudaSuccess)
        return fail(set_error(KP_ERR_OOM, "pinned plan state"));
    p->arena_cap = initial_arena(&p->o, g->n, g->nnz);
    st = dev_alloc((void **)&p->arena, p->arena_cap, s);
    if (st != KP_OK) return fail(st);
    init_state(p->hs_init, g, &p->o, p->batch ? &p->b : nullptr, p->gid0, p->arena, p->arena_cap, p->snap_dev);
    if (cudaStreamSynchronize(s) != cudaSuccess) return fail(cuda_error(cudaGetLastError(), "sync"));
    st = plan_capture(p);
    if (st != KP_OK) return fail(st);
    *out = p;
    return KP_OK;
}

kp_status plan_run_impl(kp_plan *p, cudaStream_t s, kp_hierarchy **out) {
    TraceRange trace("kp_plan_run");
    for (int attempt = 0;; attempt++) {
        std::memset(p->snap, 0, sizeof(LevelSnap) * MAX_LEVELS);
        KP_CUDA(cudaGraphLaunch(p->exec, s));
        KP_CUDA(cudaMemcpyAsync(p->hs_read, p->dst, sizeof(DevState), cudaMemcpyDeviceToHost, s));
        KP_CUDA(cudaStreamSynchronize(s));
        if (p->hs_read->err & ERR_TIMEOUT) return set_error(KP_ERR_TIMEOUT, "a bounded wait gave up");
        if (!p->hs_read->overflow) break;
        if (attempt >= 8) return set_error(KP_ERR_OOM, "the plan's arena kept overflowing");
        // the arena was too small: a larger one, the captured state upload
        // reads the new image, and the run starts over
        const unsigned long long cap =
            align256(std::max<unsigned long long>(p->arena_cap * 2, 2 * p->hs_read->arena_used + 4096));
        char *arena = nullptr;
        KP_TRY(dev_alloc((void **)&arena, cap, s));
        dev_free(p->arena, s);
        p->arena = arena;
        p->arena_cap = cap;
        init_state(p->hs_init, &p->g, &p->o, p->batch ? &p->b : nullptr, p->gid0, p->arena, p->arena_cap,
                   p->snap_dev);
        if (p->o.rating == KP_RATING_INNER_OUTER) {   // Out lives at the arena start: record again
            KP_CUDA(cudaStreamSynchronize(s));
            KP_TRY(plan_capture(p));
        }
    }
    kp_hierarchy *h = new kp_hierarchy();
    h->stream = s;
    h->device = p->device;
    h->num_graphs = p->G;
    h->glevels_dev = p->glevels_dev;
    h->gid0 = p->gid0;
    kp_level l0;
    l0.n = p->g.n;
    l0.nnz = p->g.nnz;
    l0.xadj = const_cast<eoff *>(p->g.xadj);
    l0.adjncy = const_cast<int32_t *>(p->g.adjncy);
    l0.ewgt = const_cast<int32_t *>(p->g.ewgt);
    l0.vwgt = const_cast<int32_t *>(p->g.vwgt);
    l0.owned = false;
    l0.goff = p->batch ? const_cast<int32_t *>(p->b.node_offsets) : nullptr;
    h->levels.push_back(l0);
    const kp_status st = assemble_hierarchy(h, p->hs_read, p->o.matcher == KP_MATCHER_SUITOR, p->G, nullptr, s);
    if (st != KP_OK) {
        delete h;
        return st;
    }
    h->total.launches = p->launches;
    h->total.rounds = h->total_rounds;
    h->total.n = p->g.n;
    h->total.nnz = p->g.nnz;
    for (const auto &lp : h->per_level) {
        h->total.searches += lp.searches;
        h->total.failed_cas += lp.failed_cas;
    }
    *out = h;
    return KP_OK;
}

}  // namespace kp

extern "C" {

kp_status kp_plan_create(const kp_graph *g, int32_t num_graphs, const int32_t *node_offsets, const uint64_t *seeds,
                         const int32_t *stop_sizes, const kp_options *o, kp_stream s, kp_plan **out) {
    if (!g || !out) return kp::set_error(KP_ERR_INVALID, "null argument");
    *out = nullptr;
    kp_options def;
    kp_options_default(&def);
    try {
        return kp::plan_create_impl(g, num_graphs, node_offsets, seeds, stop_sizes, o ? o : &def, (cudaStream_t)s,
                                    out);
    } catch (const std::bad_alloc &) {
        return kp::set_error(KP_ERR_OOM, "host allocation failed");
    }
}

kp_status kp_plan_run(kp_plan *p, kp_stream s, kp_hierarchy **out) {
    if (!p || !out) return kp::set_error(KP_ERR_INVALID, "null argument");
    *out = nullptr;
    try {
        return kp::plan_run_impl(p, (cudaStream_t)s, out);
    } catch (const std::bad_alloc &) {
        return kp::set_error(KP_ERR_OOM, "host allocation failed");
    }
}

void kp_plan_destroy(kp_plan *p) {
    if (!p) return;
    cudaStreamSynchronize(p->s0);
    delete p;
}

}  // extern "C"
