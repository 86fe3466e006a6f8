// The tail of the level loop in one cooperative launch.  Once levels are
// small, per-level kernel launches and host round trips cost more than the
// work, so one persistent grid runs every remaining level: the same phases
// as the per-phase kernels (match.cuh, contract.cuh), separated by a bounded
// grid barrier instead of kernel boundaries.  The grid is sized for the first
// tail level; the loop ends when a level is no longer active (stop rule,
// arena full, or a bounded wait that gave up).
#include <algorithm>

#ifndef KP_COHERENT_LOADS
#error "tail.cu must be compiled with -DKP_COHERENT_LOADS and -Xptxas -dlcm=cg"
#endif
#include "contract.cuh"
#include "match.cuh"

namespace kp {

// mode: TAIL_GRID runs every remaining level; TAIL_HANDOFF stops at the
// first level with at most `handoff` nodes and records it in tail_resume;
// TAIL_CLUSTER_AFTER continues from tail_resume (nothing if unset);
// TAIL_CLUSTER runs every remaining level.  The cluster modes are launched
// as one thread-block cluster, whose barrier is the hardware one.
enum { TAIL_GRID = 0, TAIL_HANDOFF = 1, TAIL_CLUSTER_AFTER = 2, TAIL_CLUSTER = 3 };

// three resident blocks per SM (at most 80 registers): the tail is latency
// bound, and its grid is sized from the occupancy
template <int R, bool SUITOR>
__global__ void __launch_bounds__(MATCH_BLOCK, 3) k_tail(DevState *st, int first, int last, Work w, int32_t epoch0,
                                                      int32_t handoff, int mode) {
    __shared__ OverflowSmem sm;
    GridBarrier *bar = &st->tail_bar;
    int32_t *err = &st->err;
    const long long lim = w.spin_limit;
    const bool in_cluster = mode >= TAIL_CLUSTER_AFTER;
    int start = first;
    // a level's start (carving its map and coarse weights, clearing its
    // offers) runs in the compaction phase of the level before, which reads
    // none of what it writes: one barrier less per level.  The cluster part
    // continues from a level the grid part has started, unless the grid
    // part handed over at its own first level (it started none).
    bool begun = false;
    if (mode == TAIL_CLUSTER_AFTER) {
        start = ld_relaxed_i32(&st->tail_resume);   // written by the previous launch
        if (start < first) return;   // the grid part finished the hierarchy
        begun = start > first;
    }
    for (int level = start; level < last; level++) {
        // in a cluster every block must take the same decision: the level's
        // flags are read where no block runs a phase (a block that left
        // early would leave the others at the next hardware barrier)
        const int32_t flags =
            in_cluster ? cluster_uniform_read(&st->lv[level].flags) : ld_relaxed_i32(&st->lv[level].flags);
        if (!(flags & LV_ACTIVE)) break;
        if (mode == TAIL_HANDOFF && ld_relaxed_i32(&st->lv[level].n) <= handoff) {
            if (blockIdx.x == 0 && threadIdx.x == 0) st->tail_resume = level;
            break;
        }
        if (!begun) {
            phase_level_begin<R, SUITOR>(st, level, w);
            if (!grid_sync(bar, err, lim)) return;
        }
        begun = false;
        if (SUITOR) {
            phase_suitor<R, SUITOR_FIRST>(st, level, w);
            if (!grid_sync(bar, err, lim)) return;
            // the wide pass only when some node was parked (a uniform
            // decision: that pass does not write the size it reads)
            if (ld_relaxed_i32(&st->ctr[level].list_size[0]) > 0) {
                phase_suitor<R, SUITOR_WIDE_TAIL>(st, level, w);
                if (!grid_sync(bar, err, lim)) return;
            }
        } else {
            if (!phase_handshake<R>(st, level, w)) return;
            if (!grid_sync(bar, err, lim)) return;
        }
        {
            RelabelOp<SUITOR> op;
            op.st = st;
            op.level = level;
            op.w = w;
            // a look-back wait that gave up has set the error flag: the
            // barrier below then ends every block together
            scan_lb_phase(op, w.status, epoch0 + 2 * (level - first) + 1, lim);
        }
        if (!grid_sync(bar, err, lim)) return;
        // no cluster or warp-sort kernel here: those rows stay in classes 4 and 3
        phase_contract_small(st, level, w, 0, 0);
        if (!grid_sync(bar, err, lim)) return;
        phase_contract_overflow<true, true, 2>(st, level, w, sm);
        if (!grid_sync(bar, err, lim)) return;
        {
            DegScanOp op;
            op.st = st;
            op.level = level;
            op.w = w;
            scan_lb_phase(op, w.status, epoch0 + 2 * (level - first) + 2, lim);
        }
        if (!grid_sync(bar, err, lim)) return;
        phase_compact(st, level, w);
        if (level + 1 < last) {
            // level+1's flags were decided by the degree scan (before the
            // barrier above); the start returns at once if it is not active
            phase_level_begin<R, SUITOR>(st, level + 1, w);
            begun = true;
        }
        if (!grid_sync(bar, err, lim)) return;
    }
}

namespace {

template <int R, bool SUITOR>
kp_status launch_tail_rs(DevState *st, const Work &w, const TailLaunch &t, cudaStream_t s, int32_t *launches) {
    static const int occ = [] {
        int o = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_tail<R, SUITOR>, MATCH_BLOCK, 0) != cudaSuccess)
            o = 1;
        return o > 0 ? o : 1;
    }();
    // the largest cluster (16, else 8) that the device can place
    static const int cluster = [] {
        if (cudaFuncSetAttribute(k_tail<R, SUITOR>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
            cudaSuccess)
            cudaGetLastError();
        for (int c : {16, 8}) {
            cudaLaunchConfig_t cfg = {};
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeClusterDimension;
            attr[0].val.clusterDim.x = c;
            attr[0].val.clusterDim.y = 1;
            attr[0].val.clusterDim.z = 1;
            cfg.gridDim = dim3(c);
            cfg.blockDim = dim3(MATCH_BLOCK);
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            int n = 0;
            if (cudaOccupancyMaxActiveClusters(&n, k_tail<R, SUITOR>, &cfg) == cudaSuccess && n > 0) return c;
            cudaGetLastError();
        }
        return 0;
    }();
    DevState *a0 = st;
    int a1 = t.first, a2 = t.last;
    Work a3 = w;
    int32_t a4 = t.epoch0;
    int32_t a5 = t.cluster_nodes;
    const bool use_cluster = t.cluster_nodes >= 0 && cluster > 0;
    const bool grid_part = !use_cluster || t.n_bound > t.cluster_nodes;
    if (grid_part) {
        int a6 = use_cluster ? TAIL_HANDOFF : TAIL_GRID;
        void *args[] = {&a0, &a1, &a2, &a3, &a4, &a5, &a6};
        const int64_t want = ((int64_t)std::max<int32_t>(t.n_bound, 1) + t.block_nodes - 1) / t.block_nodes;
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)occ * num_sms()));
        KP_CUDA(cudaLaunchCooperativeKernel((const void *)k_tail<R, SUITOR>, dim3(grid), dim3(MATCH_BLOCK), args, 0,
                                            s));
        *launches += 1;
    }
    if (use_cluster) {
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = cluster;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(cluster);
        cfg.blockDim = dim3(MATCH_BLOCK);
        cfg.stream = s;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        const int mode = grid_part ? TAIL_CLUSTER_AFTER : TAIL_CLUSTER;
        KP_CUDA(cudaLaunchKernelEx(&cfg, k_tail<R, SUITOR>, a0, a1, a2, a3, a4, a5, mode));
        *launches += 1;
    }
    return KP_OK;
}

template <int R>
kp_status launch_tail_r(DevState *st, const Work &w, int matcher, const TailLaunch &t, cudaStream_t s,
                        int32_t *launches) {
    if (matcher == KP_MATCHER_SUITOR) return launch_tail_rs<R, true>(st, w, t, s, launches);
    return launch_tail_rs<R, false>(st, w, t, s, launches);
}

}  // namespace

kp_status launch_tail(DevState *st, const Work &w, int rating, int matcher, const TailLaunch &t, cudaStream_t s,
                      int32_t *launches) {
    switch (rating) {
    case KP_RATING_EXPANSION_STAR2: return launch_tail_r<KP_RATING_EXPANSION_STAR2>(st, w, matcher, t, s, launches);
    case KP_RATING_INNER_OUTER: return launch_tail_r<KP_RATING_INNER_OUTER>(st, w, matcher, t, s, launches);
    case KP_RATING_WEIGHT: return launch_tail_r<KP_RATING_WEIGHT>(st, w, matcher, t, s, launches);
    case KP_RATING_EXPANSION: return launch_tail_r<KP_RATING_EXPANSION>(st, w, matcher, t, s, launches);
    case KP_RATING_EXPANSION_STAR: return launch_tail_r<KP_RATING_EXPANSION_STAR>(st, w, matcher, t, s, launches);
    default: return set_error(KP_ERR_UNSUPPORTED, "unknown rating");
    }
}

}  // namespace kp
