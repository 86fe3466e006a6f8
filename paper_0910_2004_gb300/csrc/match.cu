// Matching of locally heaviest edges (Section 3.3): launchers of the
// per-phase kernels defined in match.cuh, and Out(v) of the input level.
#include <algorithm>

#include "gpa.cuh"

namespace kp {

// Out(v) = sum of the weights of v's edges (Section 3.1), input level: G
// lanes per node (G = 1 for sparse graphs: a thread sums its short row with
// independent loads, so many rows are in flight), grid-stride over nodes.
template <int G>
__global__ void k_out_weight(int32_t n, const eoff *__restrict__ xadj, const int32_t *__restrict__ ewgt,
                             int32_t *__restrict__ outw) {
    const int gl = threadIdx.x & (G - 1);
    const unsigned gmask = group_mask<G>();
    const int64_t groups = ((int64_t)gridDim.x * blockDim.x) / G;
    // the loop bound is the same for the G lanes of a group (shuffles below)
    for (int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G; v < n; v += groups) {
        int64_t s = 0;
        const eoff beg = xadj[v], end = xadj[v + 1];
#pragma unroll 4
        for (eoff e = beg + gl; e < end; e += G) s += ewgt[e];
#pragma unroll
        for (int off = G / 2; off > 0; off >>= 1) s += __shfl_xor_sync(gmask, s, off);
        if (gl == 0) outw[v] = (int32_t)s;
    }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
namespace {

template <class K>
int occupancy_of(K kernel, int block) {
    int o = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kernel, block, 0) != cudaSuccess || o < 1) o = 1;
    return o;
}

template <int R>
kp_status launch_matching_r(const LevelLaunch &L, cudaStream_t s, int32_t *launches) {
    const int sms = num_sms();
    const int64_t nb = std::max<int64_t>(1, L.n_bound);
    const int grid1 = (int)std::max<int64_t>(1, std::min<int64_t>((nb + 255) / 256, (int64_t)sms * 8));
    if (L.matcher == KP_MATCHER_SUITOR) {
        static const int occ3 = occupancy_of(k_suitor<R, SUITOR_FIRST, 3>, MATCH_BLOCK);
        static const int occ4 = occupancy_of(k_suitor<R, SUITOR_FIRST, 4>, MATCH_BLOCK);
        static const int occ_warp = occupancy_of(k_suitor<R, SUITOR_WARP>, MATCH_BLOCK);
        static const int occ_wide = occupancy_of(k_suitor<R, SUITOR_WIDE>, MATCH_BLOCK);
        const bool four = L.suitor_blocks == 4;
        // at least 32 start nodes per warp, at most the blocks that fit at once
        const int64_t want = (nb + 32 * (MATCH_BLOCK / 32) - 1) / (32 * (MATCH_BLOCK / 32));
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want * 4, (int64_t)(four ? occ4 : occ3) * sms));
        k_level_begin<R, true><<<grid1, 256, 0, s>>>(L.st, L.level, L.w);
        if (four) k_suitor<R, SUITOR_FIRST, 4><<<grid, MATCH_BLOCK, 0, s>>>(L.st, L.level, L.w);
        else k_suitor<R, SUITOR_FIRST, 3><<<grid, MATCH_BLOCK, 0, s>>>(L.st, L.level, L.w);
        // the passes over parked nodes (they return at once when nothing is
        // parked); ordinary launches, so other streams' kernels run beside them
        k_suitor<R, SUITOR_WARP><<<occ_warp * sms, MATCH_BLOCK, 0, s>>>(L.st, L.level, L.w);
        k_suitor<R, SUITOR_WIDE><<<occ_wide * sms, MATCH_BLOCK, 0, s>>>(L.st, L.level, L.w);
        *launches += 4;
    } else if (L.matcher == KP_MATCHER_GPA) {
        static const int occ = occupancy_of(k_gpa<R>, MATCH_BLOCK);
        const int64_t want = (nb * 8 + MATCH_BLOCK - 1) / MATCH_BLOCK;
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)occ * sms));
        k_level_begin<R, false><<<grid1, 256, 0, s>>>(L.st, L.level, L.w);
        DevState *st = L.st;
        int level = L.level;
        Work w = L.w;
        void *args[] = {&st, &level, &w};
        KP_CUDA(cudaLaunchCooperativeKernel((const void *)k_gpa<R>, dim3(grid), dim3(MATCH_BLOCK), args, 0, s));
        *launches += 2;
    } else {
        static const int occ = occupancy_of(k_match<R>, MATCH_BLOCK);
        const int64_t want = (nb * 8 + MATCH_BLOCK - 1) / MATCH_BLOCK;
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)occ * sms));
        k_level_begin<R, false><<<grid1, 256, 0, s>>>(L.st, L.level, L.w);
        DevState *st = L.st;
        int level = L.level;
        Work w = L.w;
        void *args[] = {&st, &level, &w};
        KP_CUDA(cudaLaunchCooperativeKernel((const void *)k_match<R>, dim3(grid), dim3(MATCH_BLOCK), args, 0, s));
        *launches += 2;
    }
    KP_CUDA(cudaGetLastError());
    return KP_OK;
}

}  // namespace

kp_status launch_matching(const LevelLaunch &L, cudaStream_t s, int32_t *launches) {
    switch (L.rating) {
    case KP_RATING_EXPANSION_STAR2: return launch_matching_r<KP_RATING_EXPANSION_STAR2>(L, s, launches);
    case KP_RATING_INNER_OUTER: return launch_matching_r<KP_RATING_INNER_OUTER>(L, s, launches);
    case KP_RATING_WEIGHT: return launch_matching_r<KP_RATING_WEIGHT>(L, s, launches);
    case KP_RATING_EXPANSION: return launch_matching_r<KP_RATING_EXPANSION>(L, s, launches);
    case KP_RATING_EXPANSION_STAR: return launch_matching_r<KP_RATING_EXPANSION_STAR>(L, s, launches);
    default: return set_error(KP_ERR_UNSUPPORTED, "unknown rating");
    }
}

// Graph of every input node of a batch: the last graph whose first node is
// at or before it.
__global__ void k_graph_ids(int32_t n0, int32_t num_graphs, const int32_t *__restrict__ goff,
                            int32_t *__restrict__ gid) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n0; v += stride) {
        int32_t lo = 0, hi = num_graphs - 1;
        while (lo < hi) {
            const int32_t mid = lo + (hi - lo + 1) / 2;
            if (goff[mid] <= v) lo = mid;
            else hi = mid - 1;
        }
        gid[v] = lo;
    }
}

// Every edge of a batch stays inside its graph.
__global__ void k_check_batch_edges(int32_t n, const eoff *__restrict__ xadj, const int32_t *__restrict__ adjncy,
                                    const int32_t *__restrict__ gid, const int32_t *__restrict__ goff,
                                    int32_t *flag) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const int32_t g = gid[v];
        const int32_t lo = goff[g], hi = goff[g + 1];
        for (eoff e = xadj[v]; e < xadj[v + 1]; e++) {
            const int32_t u = adjncy[e];
            if (u < lo || u >= hi) {
                atomicOr(flag, 1);
                break;
            }
        }
    }
}

kp_status launch_graph_ids(int32_t n0, int32_t num_graphs, const int32_t *goff, int32_t *gid, cudaStream_t s,
                           int32_t *launches) {
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(((int64_t)n0 + 255) / 256, (int64_t)num_sms() * 8));
    k_graph_ids<<<grid, 256, 0, s>>>(n0, num_graphs, goff, gid);
    *launches += 1;
    KP_CUDA(cudaGetLastError());
    return KP_OK;
}

kp_status launch_check_batch_edges(const kp_graph *g, const int32_t *gid, const int32_t *goff, int32_t *flag,
                                   cudaStream_t s) {
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(((int64_t)g->n + 255) / 256, (int64_t)num_sms() * 8));
    k_check_batch_edges<<<grid, 256, 0, s>>>(g->n, g->xadj, g->adjncy, gid, goff, flag);
    KP_CUDA(cudaGetLastError());
    return KP_OK;
}

kp_status launch_out_weight(DevState *, int32_t n0, int64_t nnz0, const eoff *xadj, const int32_t *ewgt,
                            int32_t *outw, cudaStream_t s, int32_t *launches) {
    const bool sparse = nnz0 <= 16ll * n0;
    const int64_t threads = (int64_t)n0 * (sparse ? 1 : 8);
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((threads + 255) / 256, (int64_t)num_sms() * 32));
    if (sparse) k_out_weight<1><<<grid, 256, 0, s>>>(n0, xadj, ewgt, outw);
    else k_out_weight<8><<<grid, 256, 0, s>>>(n0, xadj, ewgt, outw);
    *launches += 1;
    KP_CUDA(cudaGetLastError());
    return KP_OK;
}

}  // namespace kp
