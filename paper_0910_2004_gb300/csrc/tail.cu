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

template <int R, bool SUITOR>
__global__ void __launch_bounds__(MATCH_BLOCK) k_tail(DevState *st, int first, int last, Work w, int32_t epoch0) {
    __shared__ OverflowSmem sm;
    GridBarrier *bar = &st->tail_bar;
    int32_t *err = &st->err;
    const long long lim = w.spin_limit;
    for (int level = first; level < last; level++) {
        if (!(ld_relaxed_i32(&st->lv[level].flags) & LV_ACTIVE)) break;
        phase_level_begin<R, SUITOR>(st, level, w);
        if (!grid_sync(bar, err, lim)) return;
        if (SUITOR) {
            phase_suitor<R, false>(st, level, w);
            if (!grid_sync(bar, err, lim)) return;
            // the wide pass only when some node was parked (uniform decision)
            if (ld_relaxed_i32(&st->ctr[level].list_size[0]) > 0) {
                phase_suitor<R, true>(st, level, w);
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
            if (!scan_lb_phase(op, w.status, epoch0 + 2 * (level - first) + 1, lim)) return;
        }
        if (!grid_sync(bar, err, lim)) return;
        phase_contract_small(st, level, w);
        if (!grid_sync(bar, err, lim)) return;
        phase_contract_overflow<true, true, 2>(st, level, w, sm);
        if (!grid_sync(bar, err, lim)) return;
        {
            DegScanOp op;
            op.st = st;
            op.level = level;
            op.w = w;
            if (!scan_lb_phase(op, w.status, epoch0 + 2 * (level - first) + 2, lim)) return;
        }
        if (!grid_sync(bar, err, lim)) return;
        phase_compact(st, level, w);
        if (!grid_sync(bar, err, lim)) return;
    }
}

namespace {

template <int R, bool SUITOR>
kp_status launch_tail_rs(DevState *st, const Work &w, int first, int last, int32_t n_bound, int32_t block_nodes, int32_t epoch0,
                         cudaStream_t s) {
    static const int occ = [] {
        int o = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_tail<R, SUITOR>, MATCH_BLOCK, 0) != cudaSuccess)
            o = 1;
        return o > 0 ? o : 1;
    }();
    const int64_t want = ((int64_t)std::max<int32_t>(n_bound, 1) + block_nodes - 1) / block_nodes;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)occ * num_sms()));
    DevState *a0 = st;
    int a1 = first, a2 = last;
    Work a3 = w;
    int32_t a4 = epoch0;
    void *args[] = {&a0, &a1, &a2, &a3, &a4};
    KP_CUDA(cudaLaunchCooperativeKernel((const void *)k_tail<R, SUITOR>, dim3(grid), dim3(MATCH_BLOCK), args, 0, s));
    return KP_OK;
}

template <int R>
kp_status launch_tail_r(DevState *st, const Work &w, int matcher, int first, int last, int32_t n_bound,
                        int32_t block_nodes, int32_t epoch0, cudaStream_t s) {
    if (matcher == KP_MATCHER_SUITOR) return launch_tail_rs<R, true>(st, w, first, last, n_bound, block_nodes, epoch0, s);
    return launch_tail_rs<R, false>(st, w, first, last, n_bound, block_nodes, epoch0, s);
}

}  // namespace

kp_status launch_tail(DevState *st, const Work &w, int rating, int matcher, int first, int last, int32_t n_bound,
                      int32_t block_nodes, int32_t epoch0, cudaStream_t s, int32_t *launches) {
    kp_status r;
    switch (rating) {
    case KP_RATING_EXPANSION_STAR2:
        r = launch_tail_r<KP_RATING_EXPANSION_STAR2>(st, w, matcher, first, last, n_bound, block_nodes, epoch0, s);
        break;
    case KP_RATING_INNER_OUTER:
        r = launch_tail_r<KP_RATING_INNER_OUTER>(st, w, matcher, first, last, n_bound, block_nodes, epoch0, s);
        break;
    case KP_RATING_WEIGHT: r = launch_tail_r<KP_RATING_WEIGHT>(st, w, matcher, first, last, n_bound, block_nodes, epoch0, s); break;
    case KP_RATING_EXPANSION:
        r = launch_tail_r<KP_RATING_EXPANSION>(st, w, matcher, first, last, n_bound, block_nodes, epoch0, s);
        break;
    case KP_RATING_EXPANSION_STAR:
        r = launch_tail_r<KP_RATING_EXPANSION_STAR>(st, w, matcher, first, last, n_bound, block_nodes, epoch0, s);
        break;
    default: return set_error(KP_ERR_UNSUPPORTED, "unknown rating");
    }
    if (r == KP_OK) *launches += 1;
    return r;
}

}  // namespace kp
