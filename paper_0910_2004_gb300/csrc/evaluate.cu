// Projection of a coarse partition (uncontraction, Section 2) and evaluation
// of a partition: cut and block weights (Section 2), balance bound L_max
// (Section 2), imbalance and per-node FM gains (Section 5.2).
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>

#include "kp_internal.cuh"

namespace kp {

constexpr int PROJECT_MAX_LEVELS = 128;

struct ProjectParams {
    int32_t n0;
    int32_t L;
    const int32_t *coarse_part;
    int32_t *fine_part;
    const int32_t *maps[PROJECT_MAX_LEVELS];
};

// p_0(v) = p_L(map_{L-1}(...map_0(v))): every level of the uncontraction in
// one pass, a chain of gathers per input node.
__global__ void k_project(const __grid_constant__ ProjectParams p) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < p.n0; v += stride) {
        int32_t x = (int32_t)v;
        for (int l = 0; l < p.L; l++) x = p.maps[l][x];
        p.fine_part[v] = p.coarse_part[x];
    }
}

// Device accumulators of one evaluation.
struct EvalAcc {
    unsigned long long ext_sum;   // sum over v of omega(v, other blocks) = 2 * cut
    unsigned long long total_c;
    long long max_c;
    long long max_bw;
    int32_t err;
    int32_t long_count;   // rows left to the group kernel by the thread kernel
    int32_t pad[2];
};

constexpr int EVAL_BLOCK = 256;
constexpr int BW_SMEM = 2048;   // block weights kept in shared memory up to this k
constexpr int HIST_K = 256;     // warp groups sum a long row's connections in shared memory up to this k
constexpr int HUB_ROW = 4096;   // longer rows (k <= HUB_K) go to a block each (k_cut_gain_hubs)
constexpr int HUB_BLOCK = 512;
constexpr int HUB_K = 4096;     // the hub kernel's k connection sums in shared memory (32 KB)

struct CutGainParams {
    int32_t n;
    int32_t k;
    int32_t id_base;   // neighbour ids minus this are the graph's node ids (0 for a whole graph)
    const eoff *__restrict__ xadj;
    const int32_t *__restrict__ adjncy;
    const int32_t *__restrict__ ewgt;
    const int32_t *__restrict__ vwgt;
    const int32_t *__restrict__ part;
    unsigned long long *block_w;
    int64_t *gain;
    int32_t *target;
    EvalAcc *acc;
    // G = 32 kernels with k <= HUB_K: leave rows of more than hub_min
    // entries to k_cut_gain_hubs (the list kernel skips them in its list,
    // the per-node kernel appends them to hub_list).  hub_min is HUB_ROW
    // when a warp can sum a row in its shared-memory bins (k <= HIST_K),
    // else 32: above that a warp would pass over the row once per adjacent
    // block
    int32_t hub_defer = 0;
    int32_t hub_min = HUB_ROW;
    int32_t *hub_list = nullptr;
};

// One G-lane group per node.  The adjacent blocks of v are visited in
// increasing id order (each step finds the smallest block id above the last
// one and sums the weight towards it), so the first block reaching the
// largest connection is the smallest such id.  A whole warp (G = 32) with
// k <= HIST_K instead sums a row longer than the warp into a per-warp
// shared-memory array of k connections in one pass and takes the largest
// (smallest id on ties): one pass instead of one per adjacent block, which
// matters for the hubs of power-law graphs.  FROM_LIST: only the rows of
// `rows` (count in acc->long_count), without the node weights (the thread
// kernel has added those for every node).
template <int G, bool FROM_LIST = false>
__global__ void __launch_bounds__(EVAL_BLOCK) k_cut_gain(CutGainParams p, const int32_t *rows = nullptr) {
    __shared__ unsigned long long s_bw[BW_SMEM];
    __shared__ unsigned long long s_red[EVAL_BLOCK / 32];
    __shared__ long long s_max[EVAL_BLOCK / 32];
    constexpr bool HIST = G == 32;
    __shared__ unsigned long long s_conn[HIST ? EVAL_BLOCK / 32 : 1][HIST ? HIST_K : 1];
    const bool use_hist = HIST && p.k <= HIST_K;
    const bool smem_bw = p.k <= BW_SMEM;
    if (smem_bw)
        for (int i = threadIdx.x; i < p.k; i += blockDim.x) s_bw[i] = 0;
    __syncthreads();
    const unsigned gmask = group_mask<G>();
    const int lane = threadIdx.x & 31;
    const int gl = lane & (G - 1);
    const int64_t gid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
    const int64_t ngroups = (int64_t)gridDim.x * blockDim.x / G;
    unsigned long long ext_acc = 0, c_acc = 0;
    long long cmax = 0;
    int32_t bad = 0;
    const int64_t count = FROM_LIST ? (int64_t)*(volatile int32_t *)&p.acc->long_count : (int64_t)p.n;
    for (int64_t i = gid; i < count; i += ngroups) {
        const int64_t v = FROM_LIST ? (int64_t)rows[i] : i;
        const int32_t pv = p.part[v];
        const bool pv_ok = pv >= 0 && pv < p.k;
        const eoff beg = p.xadj[v], end = p.xadj[v + 1];
        const int32_t deg = (int32_t)(end - beg);
        // entries held in registers when the row fits the group
        int32_t rb = -1, rw = 0;
        if (deg <= G && gl < deg) {
            rb = p.part[p.adjncy[beg + gl] - p.id_base];
            rw = p.ewgt[beg + gl];
            if (rb < 0 || rb >= p.k) {
                bad = 1;
                rb = -1;
            }
        }
        long long inw = 0, tot = 0;
        int32_t best = -1;
        long long best_conn = 0;
        // a hub left to the block kernel (its node weight is still added below)
        const bool defer = HIST && p.hub_defer && deg > p.hub_min;
        if (defer) {
            if (!FROM_LIST && gl == 0) p.hub_list[atomicAdd(&p.acc->long_count, 1)] = (int32_t)v;
        } else if (use_hist && deg > G) {
            // one pass: connection to every block in this warp's bins
            unsigned long long *conn = s_conn[HIST ? threadIdx.x >> 5 : 0];
            for (int32_t b = lane; b < p.k; b += 32) conn[b] = 0;
            __syncwarp();
#pragma unroll 4
            for (eoff e = beg + lane; e < end; e += 32) {
                const int32_t b = p.part[p.adjncy[e] - p.id_base];
                const int32_t w = p.ewgt[e];
                if (b < 0 || b >= p.k) {
                    bad = 1;
                    continue;
                }
                tot += w;
                if (b == pv) inw += w;
                else atomicAdd(&conn[b], (unsigned long long)(long long)w);
            }
            __syncwarp();
            for (int32_t b = lane; b < p.k; b += 32) {   // increasing ids: ties keep the smaller
                const long long c = (long long)conn[b];
                if (c > best_conn) {
                    best_conn = c;
                    best = b;
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                inw += __shfl_xor_sync(0xffffffffu, inw, o);
                tot += __shfl_xor_sync(0xffffffffu, tot, o);
                const long long oc = __shfl_xor_sync(0xffffffffu, best_conn, o);
                const int32_t ob = __shfl_xor_sync(0xffffffffu, best, o);
                if (oc > best_conn || (oc == best_conn && oc > 0 && ob < best)) {
                    best_conn = oc;
                    best = ob;
                }
            }
            __syncwarp();   // every lane has read the bins before the next row clears them
        } else {
            // pass over the row: internal weight, total weight, smallest other block
            int32_t nextb = 0x7fffffff;
            if (deg <= G) {
                if (rb >= 0) {
                    tot = rw;
                    if (rb == pv) inw = rw;
                    else nextb = rb;
                }
            } else {
                for (eoff e = beg + gl; e < end; e += G) {
                    const int32_t b = p.part[p.adjncy[e] - p.id_base];
                    const int32_t w = p.ewgt[e];
                    if (b < 0 || b >= p.k) {
                        bad = 1;
                        continue;
                    }
                    tot += w;
                    if (b == pv) inw += w;
                    else nextb = min(nextb, b);
                }
            }
#pragma unroll
            for (int o = G / 2; o > 0; o >>= 1) {
                inw += __shfl_xor_sync(gmask, inw, o);
                tot += __shfl_xor_sync(gmask, tot, o);
                nextb = min(nextb, __shfl_xor_sync(gmask, nextb, o));
            }
            while (nextb != 0x7fffffff) {
                const int32_t cur = nextb;
                long long conn = 0;
                nextb = 0x7fffffff;
                if (deg <= G) {
                    if (rb == cur) conn = rw;
                    else if (rb > cur && rb != pv) nextb = rb;
                } else {
                    for (eoff e = beg + gl; e < end; e += G) {
                        const int32_t b = p.part[p.adjncy[e] - p.id_base];
                        if (b < 0 || b >= p.k) continue;
                        if (b == cur) conn += p.ewgt[e];
                        else if (b > cur && b != pv) nextb = min(nextb, b);
                    }
                }
#pragma unroll
                for (int o = G / 2; o > 0; o >>= 1) {
                    conn += __shfl_xor_sync(gmask, conn, o);
                    nextb = min(nextb, __shfl_xor_sync(gmask, nextb, o));
                }
                if (conn > best_conn) {
                    best_conn = conn;
                    best = cur;
                }
            }
        }
        if (gl == 0 && !defer) {
            p.gain[v] = (best >= 0 ? best_conn : 0) - inw;
            p.target[v] = best;
            ext_acc += (unsigned long long)(tot - inw);
        }
        if (gl == 0 && !FROM_LIST) {
            const int32_t c = p.vwgt[v];
            c_acc += (unsigned long long)(long long)c;
            cmax = max(cmax, (long long)c);
            if (!pv_ok) {
                bad = 1;
            } else if (smem_bw) {
                atomicAdd(&s_bw[pv], (unsigned long long)(long long)c);
            } else {
                atomicAdd(&p.block_w[pv], (unsigned long long)(long long)c);
            }
        }
    }
    // block reductions, then one atomic per block
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ext_acc += __shfl_xor_sync(0xffffffffu, ext_acc, o);
        c_acc += __shfl_xor_sync(0xffffffffu, c_acc, o);
        cmax = max(cmax, __shfl_xor_sync(0xffffffffu, cmax, o));
    }
    const int warp = threadIdx.x >> 5;
    if (lane == 0) {
        s_red[warp] = ext_acc;
        s_max[warp] = cmax;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long e = 0;
        long long m = 0;
        for (int w = 0; w < EVAL_BLOCK / 32; w++) {
            e += s_red[w];
            m = max(m, s_max[w]);
        }
        atomicAdd(&p.acc->ext_sum, e);
        atomicMax(&p.acc->max_c, m);
    }
    __syncthreads();
    if (lane == 0) s_red[warp] = c_acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long c = 0;
        for (int w = 0; w < EVAL_BLOCK / 32; w++) c += s_red[w];
        atomicAdd(&p.acc->total_c, c);
    }
    if (bad) atomicOr(&p.acc->err, ERR_BAD_PART);
    if (smem_bw)
        for (int i = threadIdx.x; i < p.k; i += blockDim.x)
            if (s_bw[i]) atomicAdd(&p.block_w[i], s_bw[i]);
}

// Rows of more than p.hub_min entries (hubs of power-law graphs; with
// k > HIST_K every row longer than a warp), one block each, k <= HUB_K: all
// threads sum the row's connection to every block in shared memory in one
// pass and the largest is taken (smallest block id on ties).  The G = 32
// kernels leave these rows to it (their node weights stay there); the rows
// are those of `rows` [0, acc->long_count) with more than p.hub_min entries.
__global__ void __launch_bounds__(HUB_BLOCK) k_cut_gain_hubs(CutGainParams p, const int32_t *rows) {
    constexpr int NW = HUB_BLOCK / 32;
    extern __shared__ unsigned long long conn[];   // p.k sums (launched with 8k bytes)
    __shared__ long long s_in[NW], s_tot[NW], s_bc[NW];
    __shared__ int32_t s_bb[NW];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int32_t count = *(volatile int32_t *)&p.acc->long_count;
    unsigned long long ext = 0;
    int32_t bad = 0;
    for (int32_t li = blockIdx.x; li < count; li += gridDim.x) {
        const int32_t v = rows[li];
        const eoff beg = p.xadj[v], end = p.xadj[v + 1];
        if (end - beg <= p.hub_min) continue;   // the same for the whole block
        const int32_t pv = p.part[v];
        for (int32_t b = threadIdx.x; b < p.k; b += HUB_BLOCK) conn[b] = 0;
        __syncthreads();
        long long inw = 0, tot = 0;
#pragma unroll 4
        for (eoff e = beg + (eoff)threadIdx.x; e < end; e += HUB_BLOCK) {
            const int32_t b = p.part[p.adjncy[e] - p.id_base];
            const int32_t w = p.ewgt[e];
            if (b < 0 || b >= p.k) {
                bad = 1;
                continue;
            }
            tot += w;
            if (b == pv) inw += w;
            else atomicAdd(&conn[b], (unsigned long long)(long long)w);
        }
        __syncthreads();
        long long bc = 0;
        int32_t bb = -1;
        for (int32_t b = threadIdx.x; b < p.k; b += HUB_BLOCK) {   // increasing ids: ties keep the smaller
            const long long c = (long long)conn[b];
            if (c > bc) {
                bc = c;
                bb = b;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            inw += __shfl_xor_sync(0xffffffffu, inw, o);
            tot += __shfl_xor_sync(0xffffffffu, tot, o);
            const long long oc = __shfl_xor_sync(0xffffffffu, bc, o);
            const int32_t ob = __shfl_xor_sync(0xffffffffu, bb, o);
            if (oc > bc || (oc == bc && oc > 0 && ob < bb)) {
                bc = oc;
                bb = ob;
            }
        }
        if (lane == 0) {
            s_in[warp] = inw;
            s_tot[warp] = tot;
            s_bc[warp] = bc;
            s_bb[warp] = bb;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            long long in_all = 0, tot_all = 0, c = 0;
            int32_t t = -1;
            for (int i = 0; i < NW; i++) {
                in_all += s_in[i];
                tot_all += s_tot[i];
                if (s_bc[i] > c || (s_bc[i] == c && c > 0 && s_bb[i] < t)) {
                    c = s_bc[i];
                    t = s_bb[i];
                }
            }
            p.gain[v] = (t >= 0 ? c : 0) - in_all;
            p.target[v] = t;
            ext += (unsigned long long)(tot_all - in_all);
        }
        __syncthreads();   // the bins and partial sums are read before the next row
    }
    if (threadIdx.x == 0 && ext) atomicAdd(&p.acc->ext_sum, ext);
    if (bad) atomicOr(&p.acc->err, ERR_BAD_PART);
}

// One thread per node for rows of at most EVAL_TROW entries (the row is read
// into registers with independent loads; the connection to every adjacent
// block is summed over the row, the largest wins, ties to the smaller block
// id, as in the group kernel); longer rows are listed for the group kernel.
// Node weights, their sum and maximum and the block weights are added here
// for every node; with k above BW_SMEM the block weights of a warp's nodes
// are combined per block before the global atomic.
constexpr int EVAL_TROW = 16;

template <bool SMEM_BW>
__global__ void __launch_bounds__(EVAL_BLOCK) k_cut_gain_rows(CutGainParams p, int32_t *long_rows) {
    __shared__ unsigned long long s_bw[SMEM_BW ? BW_SMEM : 1];
    __shared__ unsigned long long s_red[EVAL_BLOCK / 32];
    __shared__ long long s_max[EVAL_BLOCK / 32];
    if (SMEM_BW)
        for (int i = threadIdx.x; i < p.k; i += blockDim.x) s_bw[i] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    unsigned long long ext_acc = 0, c_acc = 0;
    long long cmax = 0;
    int32_t bad = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v0 = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); v0 < p.n; v0 += stride) {
        const int64_t v = v0 + lane;
        const bool live = v < p.n;
        int32_t pv = -1, c = 0, d = 0;
        eoff beg = 0;
        if (live) {
            pv = p.part[v];
            c = p.vwgt[v];
            beg = p.xadj[v];
            d = (int32_t)(p.xadj[v + 1] - beg);
        }
        const bool pv_ok = pv >= 0 && pv < p.k;
        if (live) {
            c_acc += (unsigned long long)(long long)c;
            cmax = max(cmax, (long long)c);
            if (!pv_ok) bad = 1;
        }
        if (SMEM_BW) {
            if (live && pv_ok) atomicAdd(&s_bw[pv], (unsigned long long)(long long)c);
        } else {
            const int key = (live && pv_ok) ? pv : -1 - lane;   // unique for lanes without a block
            const unsigned peers = __match_any_sync(0xffffffffu, key);
            long long sum = 0;
#pragma unroll
            for (int j = 0; j < 32; j++) {
                const long long cj = __shfl_sync(0xffffffffu, (long long)c, j);
                if ((peers >> j) & 1u) sum += cj;
            }
            if (live && pv_ok && (peers & ((1u << lane) - 1u)) == 0)
                atomicAdd(&p.block_w[pv], (unsigned long long)sum);
        }
        if (!live) continue;
        if (d > EVAL_TROW) {
            long_rows[atomicAdd(&p.acc->long_count, 1)] = (int32_t)v;
            continue;
        }
        int32_t b[EVAL_TROW], w[EVAL_TROW];
#pragma unroll
        for (int i = 0; i < EVAL_TROW; i++) {
            if (i >= d) break;
            b[i] = p.adjncy[beg + i];
        }
#pragma unroll
        for (int i = 0; i < EVAL_TROW; i++) {
            if (i >= d) break;
            w[i] = p.ewgt[beg + i];
        }
#pragma unroll
        for (int i = 0; i < EVAL_TROW; i++) {
            if (i >= d) break;
            const int32_t bb = p.part[b[i] - p.id_base];
            if (bb < 0 || bb >= p.k) {
                bad = 1;
                b[i] = -1;
            } else {
                b[i] = bb;
            }
        }
        long long inw = 0, tot = 0;
        bool boundary = false;
#pragma unroll
        for (int i = 0; i < EVAL_TROW; i++) {
            if (i >= d) break;
            if (b[i] >= 0) {
                tot += w[i];
                if (b[i] == pv) inw += w[i];
                else boundary = true;
            }
        }
        int32_t best = -1;
        long long best_conn = 0;
        if (boundary) {   // interior nodes (every neighbour in pv) skip the search
#pragma unroll
            for (int i = 0; i < EVAL_TROW; i++) {
                if (i >= d) break;
                if (b[i] >= 0 && b[i] != pv) {
                    long long conn = 0;
#pragma unroll
                    for (int j = 0; j < EVAL_TROW; j++) {
                        if (j >= d) break;
                        if (b[j] == b[i]) conn += w[j];
                    }
                    if (conn > best_conn || (conn == best_conn && best >= 0 && b[i] < best)) {
                        best_conn = conn;
                        best = b[i];
                    }
                }
            }
        }
        p.gain[v] = (best >= 0 ? best_conn : 0) - inw;
        p.target[v] = best;
        ext_acc += (unsigned long long)(tot - inw);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ext_acc += __shfl_xor_sync(0xffffffffu, ext_acc, o);
        c_acc += __shfl_xor_sync(0xffffffffu, c_acc, o);
        cmax = max(cmax, __shfl_xor_sync(0xffffffffu, cmax, o));
    }
    const int warp = threadIdx.x >> 5;
    if (lane == 0) {
        s_red[warp] = ext_acc;
        s_max[warp] = cmax;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long e = 0;
        long long m = 0;
        for (int w2 = 0; w2 < EVAL_BLOCK / 32; w2++) {
            e += s_red[w2];
            m = max(m, s_max[w2]);
        }
        atomicAdd(&p.acc->ext_sum, e);
        atomicMax(&p.acc->max_c, m);
    }
    __syncthreads();
    if (lane == 0) s_red[warp] = c_acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int w2 = 0; w2 < EVAL_BLOCK / 32; w2++) t += s_red[w2];
        atomicAdd(&p.acc->total_c, t);
    }
    if (bad) atomicOr(&p.acc->err, ERR_BAD_PART);
    if (SMEM_BW)
        for (int i = threadIdx.x; i < p.k; i += blockDim.x)
            if (s_bw[i]) atomicAdd(&p.block_w[i], s_bw[i]);
}

__global__ void k_max_block(int32_t k, const long long *block_w, EvalAcc *acc) {
    long long m = 0;
    for (int i = threadIdx.x; i < k; i += blockDim.x) m = max(m, block_w[i]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(&acc->max_bw, m);
}

// floor((1+eps) c(V)/k + max c) with eps read as round(eps * 10^6) ppm.
int64_t l_max_of(int64_t total_c, int64_t max_c, int32_t k, double eps) {
    const long long eps_ppm = llround(eps * 1e6);
    const __int128 num = (__int128)(1000000 + eps_ppm) * total_c + (__int128)k * 1000000 * max_c;
    const __int128 den = (__int128)k * 1000000;
    return (int64_t)(num / den);
}

namespace {

kp_status check_eval_args(const kp_graph *g, const int32_t *part, int32_t k, double eps,
                          const kp_cut_gain_out *out) {
    if (!g || !out) return set_error(KP_ERR_INVALID, "null argument");
    if (k < 1) return set_error(KP_ERR_INVALID, "k must be >= 1");
    if (!(eps >= 0.0) || eps > 1000.0) return set_error(KP_ERR_INVALID, "eps must be in [0, 1000]");
    if (g->n < 0 || g->nnz < 0) return set_error(KP_ERR_INVALID, "negative graph size");
    if ((int64_t)g->nnz >= NNZ_LIMIT) return set_error(KP_ERR_OVERFLOW, "nnz >= 2^32: the edge weights sum to 2^31 or more");
    if (g->n > 0 && (!part || !g->xadj || !g->vwgt || !out->gain || !out->target ||
                     (g->nnz > 0 && (!g->adjncy || !g->ewgt))))
        return set_error(KP_ERR_INVALID, "null array");
    if (!out->block_w) return set_error(KP_ERR_INVALID, "null block_w");
    return KP_OK;
}

}  // namespace

// Evaluation with the accumulators in caller-provided device memory `acc`.
kp_status cut_gain_with(const kp_graph *g, const int32_t *part, int32_t k, double eps, kp_cut_gain_out *out,
                        cudaStream_t s, EvalAcc *acc, EvalAcc *host_acc, int32_t id_base = 0,
                        int32_t *long_rows = nullptr) {
    KP_TRY(check_eval_args(g, part, k, eps, out));
    KP_CUDA(cudaMemsetAsync(acc, 0, sizeof(EvalAcc), s));
    KP_CUDA(cudaMemsetAsync(out->block_w, 0, sizeof(int64_t) * (size_t)k, s));
    if (g->n > 0) {
        CutGainParams p;
        p.n = g->n;
        p.k = k;
        p.id_base = id_base;
        p.xadj = g->xadj;
        p.adjncy = g->adjncy;
        p.ewgt = g->ewgt;
        p.vwgt = g->vwgt;
        p.part = part;
        p.block_w = reinterpret_cast<unsigned long long *>(out->block_w);
        p.gain = out->gain;
        p.target = out->target;
        p.acc = acc;
        const double avg = (double)g->nnz / (double)g->n;
        const int grid_cap = num_sms() * 8;
        auto grid_for = [&](int G) {
            const int64_t want = ((int64_t)g->n * G + EVAL_BLOCK - 1) / EVAL_BLOCK;
            return (int)std::max<int64_t>(1, std::min<int64_t>(want, grid_cap));
        };
        // hub rows by a block each when a row list is at hand (the G = 32
        // kernels below leave them to k_cut_gain_hubs)
        const bool hubs = long_rows && k <= HUB_K && (avg <= 12.0 || avg > 20.0);
        p.hub_defer = hubs ? 1 : 0;
        p.hub_min = k <= HIST_K ? HUB_ROW : 32;
        p.hub_list = long_rows;
        if (long_rows && (avg <= 12.0 || avg > 20.0)) {
            // rows of up to 16 entries one thread each, the longer ones listed
            // for one warp each
            if (k <= BW_SMEM) k_cut_gain_rows<true><<<grid_for(1), EVAL_BLOCK, 0, s>>>(p, long_rows);
            else k_cut_gain_rows<false><<<grid_for(1), EVAL_BLOCK, 0, s>>>(p, long_rows);
            KP_CUDA(cudaGetLastError());
            k_cut_gain<32, true><<<grid_cap, EVAL_BLOCK, 0, s>>>(p, long_rows);
        } else if (avg <= 5.0) {
            k_cut_gain<4><<<grid_for(4), EVAL_BLOCK, 0, s>>>(p);
        } else if (avg <= 10.0) {
            k_cut_gain<8><<<grid_for(8), EVAL_BLOCK, 0, s>>>(p);
        } else if (avg <= 20.0) {
            k_cut_gain<16><<<grid_for(16), EVAL_BLOCK, 0, s>>>(p);
        } else {
            k_cut_gain<32><<<grid_for(32), EVAL_BLOCK, 0, s>>>(p);
        }
        KP_CUDA(cudaGetLastError());
        if (hubs)
            k_cut_gain_hubs<<<num_sms() * 2, HUB_BLOCK, sizeof(unsigned long long) * (size_t)k, s>>>(p, long_rows);
        k_max_block<<<1, 1024, 0, s>>>(k, reinterpret_cast<const long long *>(out->block_w), acc);
        KP_CUDA(cudaGetLastError());
    }
    KP_CUDA(cudaMemcpyAsync(host_acc, acc, sizeof(EvalAcc), cudaMemcpyDeviceToHost, s));
    KP_CUDA(cudaStreamSynchronize(s));
    if (host_acc->err & ERR_BAD_PART) return set_error(KP_ERR_INVALID, "block id outside [0,k)");
    out->cut = (int64_t)(host_acc->ext_sum / 2);
    out->total_c = (int64_t)host_acc->total_c;
    out->max_c = (int64_t)host_acc->max_c;
    out->l_max = l_max_of(out->total_c, out->max_c, k, eps);
    out->imbalance = std::max<int64_t>(0, (int64_t)host_acc->max_bw - out->l_max);
    return KP_OK;
}

// ---------------------------------------------------------------------------
// evaluation without any allocation
// ---------------------------------------------------------------------------
// Scratch of kp_cut_gain_noalloc: words [0, 8) hold the accumulators
// (EvalAcc), words [8, 8 + KP_CUT_GAIN_NOALLOC_MAX_K) one partial weight per
// block.  Every device that loads the library holds it until the process
// exits; all calls share it.
constexpr int NOALLOC_HEADER_WORDS = 8;
static_assert(sizeof(EvalAcc) <= NOALLOC_HEADER_WORDS * sizeof(unsigned long long), "accumulator header");
static __device__ __align__(256) unsigned long long
    g_noalloc_scratch[NOALLOC_HEADER_WORDS + KP_CUT_GAIN_NOALLOC_MAX_K];

// Copies the block weights to the caller's buffer and reduces their maximum.
__global__ void k_noalloc_finish(int32_t k, const unsigned long long *bw, long long *block_w_out, EvalAcc *acc) {
    long long m = 0;
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
        const long long v = (long long)bw[i];
        block_w_out[i] = v;
        m = max(m, v);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(&acc->max_bw, m);
}

namespace {
std::mutex g_noalloc_mu;
unsigned long long *g_noalloc_ptr[64] = {nullptr};

// Device address of the static scratch on the current device, looked up once
// per device with that device current.
kp_status noalloc_scratch(unsigned long long **out) {
    int dev = 0;
    KP_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return set_error(KP_ERR_UNSUPPORTED, "device ordinal above 63");
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(static scratch)");
        g_noalloc_ptr[dev] = static_cast<unsigned long long *>(p);
    }
    *out = g_noalloc_ptr[dev];
    return KP_OK;
}
}  // namespace

kp_status cut_gain_noalloc_impl(const kp_graph *g, const int32_t *part, int32_t k, double eps,
                                kp_cut_gain_out *out, cudaStream_t s) {
    KP_TRY(check_eval_args(g, part, k, eps, out));
    if (k > KP_CUT_GAIN_NOALLOC_MAX_K)
        return set_error(KP_ERR_UNSUPPORTED, "kp_cut_gain_noalloc: k exceeds KP_CUT_GAIN_NOALLOC_MAX_K (16384)");
    unsigned long long *scratch = nullptr;
    KP_TRY(noalloc_scratch(&scratch));
    EvalAcc *acc = reinterpret_cast<EvalAcc *>(scratch);
    unsigned long long *bw = scratch + NOALLOC_HEADER_WORDS;
    // the accumulators and the k partial block weights start at zero
    KP_CUDA(cudaMemsetAsync(scratch, 0, sizeof(unsigned long long) * (size_t)(NOALLOC_HEADER_WORDS + k), s));
    if (g->n > 0) {
        CutGainParams p;
        p.n = g->n;
        p.k = k;
        p.id_base = 0;
        p.xadj = g->xadj;
        p.adjncy = g->adjncy;
        p.ewgt = g->ewgt;
        p.vwgt = g->vwgt;
        p.part = part;
        p.block_w = bw;
        p.gain = out->gain;
        p.target = out->target;
        p.acc = acc;
        const double avg = (double)g->nnz / (double)g->n;
        const int grid_cap = num_sms() * 8;
        auto grid_for = [&](int G) {
            const int64_t want = ((int64_t)g->n * G + EVAL_BLOCK - 1) / EVAL_BLOCK;
            return (int)std::max<int64_t>(1, std::min<int64_t>(want, grid_cap));
        };
        if (avg <= 5.0) k_cut_gain<4><<<grid_for(4), EVAL_BLOCK, 0, s>>>(p);
        else if (avg <= 10.0) k_cut_gain<8><<<grid_for(8), EVAL_BLOCK, 0, s>>>(p);
        else if (avg <= 20.0) k_cut_gain<16><<<grid_for(16), EVAL_BLOCK, 0, s>>>(p);
        else k_cut_gain<32><<<grid_for(32), EVAL_BLOCK, 0, s>>>(p);
        KP_CUDA(cudaGetLastError());
    }
    k_noalloc_finish<<<1, 1024, 0, s>>>(k, bw, reinterpret_cast<long long *>(out->block_w), acc);
    KP_CUDA(cudaGetLastError());
    EvalAcc host_acc;   // pageable: no pinned allocation
    KP_CUDA(cudaMemcpyAsync(&host_acc, acc, sizeof(EvalAcc), cudaMemcpyDeviceToHost, s));
    KP_CUDA(cudaStreamSynchronize(s));
    if (host_acc.err & ERR_BAD_PART) return set_error(KP_ERR_INVALID, "block id outside [0,k)");
    out->cut = (int64_t)(host_acc.ext_sum / 2);
    out->total_c = (int64_t)host_acc.total_c;
    out->max_c = (int64_t)host_acc.max_c;
    out->l_max = l_max_of(out->total_c, out->max_c, k, eps);
    out->imbalance = std::max<int64_t>(0, (int64_t)host_acc.max_bw - out->l_max);
    return KP_OK;
}

// Cut/gain of one graph of a batch union: `view` is the graph's slice (its
// xadj and vwgt start at the graph's first node, adjncy and ewgt are the
// union's arrays), neighbour ids are id_base higher than the graph's ids.
kp_status cut_gain_slice(const kp_graph *view, int32_t id_base, const int32_t *part, int32_t k, double eps,
                         kp_cut_gain_out *out, cudaStream_t s) {
    KP_TRY(check_eval_args(view, part, k, eps, out));
    EvalAcc *acc = nullptr;
    KP_TRY(dev_alloc_n(&acc, 1, s));
    thread_local EvalAcc *host_acc = nullptr;
    if (!host_acc && cudaMallocHost((void **)&host_acc, sizeof(EvalAcc)) != cudaSuccess) {
        host_acc = nullptr;
        dev_free(acc, s);
        return set_error(KP_ERR_OOM, "pinned host accumulator");
    }
    int32_t *rows = nullptr;
    kp_status st = dev_alloc_n(&rows, view->n, s);
    if (st == KP_OK) st = cut_gain_with(view, part, k, eps, out, s, acc, host_acc, id_base, rows);
    dev_free(rows, s);
    dev_free(acc, s);
    return st;
}

kp_status cut_gain_impl(const kp_graph *g, const int32_t *part, int32_t k, double eps, kp_cut_gain_out *out,
                        cudaStream_t s) {
    KP_TRY(check_eval_args(g, part, k, eps, out));
    EvalAcc *acc = nullptr;
    KP_TRY(dev_alloc_n(&acc, 1, s));
    thread_local EvalAcc *host_acc = nullptr;
    if (!host_acc && cudaMallocHost((void **)&host_acc, sizeof(EvalAcc)) != cudaSuccess) {
        host_acc = nullptr;
        dev_free(acc, s);
        return set_error(KP_ERR_OOM, "pinned host accumulator");
    }
    int32_t *rows = nullptr;
    kp_status st = dev_alloc_n(&rows, g->n, s);
    if (st == KP_OK) st = cut_gain_with(g, part, k, eps, out, s, acc, host_acc, 0, rows);
    dev_free(rows, s);
    dev_free(acc, s);
    return st;
}

struct ProjectBatchParams {
    int32_t n0;
    const int32_t *gid0;
    const int32_t *glevels;
    const int32_t *coarse_part;
    const int32_t *coarse_offsets;
    int32_t *fine_part;
    const int32_t *maps[PROJECT_MAX_LEVELS];
    const int32_t *goffs[PROJECT_MAX_LEVELS];
};

// Batches: every graph from its own coarsest level, whose partition sits at
// coarse_part[coarse_offsets[g] + local id].
__global__ void k_project_batch(const __grid_constant__ ProjectBatchParams p) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < p.n0; v += stride) {
        const int32_t g = p.gid0[v];
        const int32_t L = p.glevels[g] - 1;
        int32_t x = (int32_t)v;
        for (int l = 0; l < L; l++) x = p.maps[l][x];
        p.fine_part[v] = p.coarse_part[p.coarse_offsets[g] + (x - p.goffs[L][g])];
    }
}

struct CoarsestParams {
    int32_t num_graphs;
    const int32_t *glevels;
    int32_t *sizes;
    const int32_t *goffs[PROJECT_MAX_LEVELS];
};

__global__ void k_batch_coarsest(const __grid_constant__ CoarsestParams p) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < p.num_graphs; g += stride) {
        const int32_t L = p.glevels[g] - 1;
        p.sizes[g] = p.goffs[L][g + 1] - p.goffs[L][g];
    }
}

kp_status batch_coarsest_impl(const kp_hierarchy *h, int32_t *sizes, cudaStream_t s) {
    if (!h || !sizes) return set_error(KP_ERR_INVALID, "null argument");
    if (h->num_graphs == 0) return set_error(KP_ERR_INVALID, "not a batch hierarchy");
    const int32_t L = (int32_t)h->levels.size();
    if (L > PROJECT_MAX_LEVELS) return set_error(KP_ERR_UNSUPPORTED, "too many levels");
    CoarsestParams p;
    std::memset(&p, 0, sizeof p);
    p.num_graphs = h->num_graphs;
    p.glevels = h->glevels_dev;
    for (int l = 0; l < L; l++) p.goffs[l] = h->levels[(size_t)l].goff;
    int32_t *d = nullptr;
    KP_TRY(dev_alloc_n(&d, h->num_graphs, s));
    p.sizes = d;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(((int64_t)h->num_graphs + 255) / 256, 1024));
    k_batch_coarsest<<<grid, 256, 0, s>>>(p);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(sizes, d, sizeof(int32_t) * (size_t)h->num_graphs, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    dev_free(d, s);
    if (e != cudaSuccess) return cuda_error(e, "batch coarsest sizes");
    return KP_OK;
}

kp_status project_batch_impl(const kp_hierarchy *h, const int32_t *coarse_part, const int32_t *coarse_offsets,
                             int32_t *fine_part, cudaStream_t s) {
    if (!h) return set_error(KP_ERR_INVALID, "null argument");
    if (h->num_graphs == 0) return set_error(KP_ERR_INVALID, "not a batch hierarchy");
    const int32_t n0 = h->levels[0].n;
    if (n0 == 0) return KP_OK;
    if (!coarse_part || !coarse_offsets || !fine_part) return set_error(KP_ERR_INVALID, "null argument");
    const int32_t L = (int32_t)h->levels.size();
    if (L > PROJECT_MAX_LEVELS) return set_error(KP_ERR_UNSUPPORTED, "too many levels");
    ProjectBatchParams p;
    std::memset(&p, 0, sizeof p);
    p.n0 = n0;
    p.gid0 = h->gid0;
    p.glevels = h->glevels_dev;
    p.coarse_part = coarse_part;
    p.coarse_offsets = coarse_offsets;
    p.fine_part = fine_part;
    for (int l = 0; l < L; l++) {
        p.maps[l] = h->levels[(size_t)l].map;
        p.goffs[l] = h->levels[(size_t)l].goff;
    }
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(((int64_t)n0 + 255) / 256, (int64_t)num_sms() * 16));
    k_project_batch<<<grid, 256, 0, s>>>(p);
    KP_CUDA(cudaGetLastError());
    return KP_OK;
}

kp_status project_impl(const kp_hierarchy *h, const int32_t *coarse_part, int32_t *fine_part, cudaStream_t s) {
    if (!h || (h->levels[0].n > 0 && (!coarse_part || !fine_part))) return set_error(KP_ERR_INVALID, "null argument");
    const int32_t L = (int32_t)h->levels.size() - 1;
    if (L >= PROJECT_MAX_LEVELS) return set_error(KP_ERR_UNSUPPORTED, "too many levels");
    const int32_t n0 = h->levels[0].n;
    if (n0 == 0) return KP_OK;
    ProjectParams p;
    p.n0 = n0;
    p.L = L;
    p.coarse_part = coarse_part;
    p.fine_part = fine_part;
    for (int l = 0; l < L; l++) p.maps[l] = h->levels[l].map;
    const int64_t want = ((int64_t)n0 + 255) / 256;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)num_sms() * 16));
    k_project<<<grid, 256, 0, s>>>(p);
    KP_CUDA(cudaGetLastError());
    return KP_OK;
}


kp_status pipeline_host_impl(const kp_graph *hg, const kp_options *o, int32_t k, double eps,
                             kp_initial_partition_fn ip, void *user, int32_t *fine_part, int64_t *gain,
                             int32_t *target, int64_t *block_w, kp_cut_gain_out *out, int32_t *num_levels,
                             cudaStream_t s) {
    if (!hg || !o || !ip || !out) return set_error(KP_ERR_INVALID, "null argument");
    if (hg->n < 0 || hg->nnz < 0) return set_error(KP_ERR_INVALID, "negative size");
    if (k < 1) return set_error(KP_ERR_INVALID, "k must be >= 1");
    const int32_t n = hg->n;
    const eoff nnz = hg->nnz;
    eoff *d_xadj = nullptr;
    int32_t *d_adj = nullptr, *d_w = nullptr, *d_c = nullptr;
    int32_t *d_cpart = nullptr, *d_fpart = nullptr, *d_target = nullptr;
    int64_t *d_gain = nullptr, *d_bw = nullptr;
    kp_hierarchy *h = nullptr;
    std::vector<int32_t> cw, cpart;
    kp_status st = KP_OK;
    auto cleanup = [&]() {
        if (h) kp_hierarchy_free(h);
        void *ptrs[] = {d_xadj, d_adj, d_w, d_c, d_cpart, d_fpart, d_target, d_gain, d_bw};
        for (void *q : ptrs)
            if (q) dev_free(q, s);
    };
#define PH(call)                  \
    do {                          \
        st = (call);              \
        if (st != KP_OK) {        \
            cleanup();            \
            return st;            \
        }                         \
    } while (0)
#define PH_CUDA(call) PH(((call) == cudaSuccess) ? KP_OK : cuda_error(cudaGetLastError(), #call))
    PH(dev_alloc_n(&d_xadj, (int64_t)n + 1, s));
    PH(dev_alloc_n(&d_adj, nnz, s));
    PH(dev_alloc_n(&d_w, nnz, s));
    PH(dev_alloc_n(&d_c, n, s));
    PH(dev_alloc_n(&d_fpart, n, s));
    PH(dev_alloc_n(&d_target, n, s));
    PH(dev_alloc_n(&d_gain, n, s));
    PH(dev_alloc_n(&d_bw, k, s));
    PH_CUDA(cudaMemcpyAsync(d_xadj, hg->xadj, sizeof(eoff) * ((size_t)n + 1), cudaMemcpyHostToDevice, s));
    if (nnz > 0) {
        PH_CUDA(cudaMemcpyAsync(d_adj, hg->adjncy, sizeof(int32_t) * (size_t)nnz, cudaMemcpyHostToDevice, s));
        PH_CUDA(cudaMemcpyAsync(d_w, hg->ewgt, sizeof(int32_t) * (size_t)nnz, cudaMemcpyHostToDevice, s));
    }
    if (n > 0) PH_CUDA(cudaMemcpyAsync(d_c, hg->vwgt, sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice, s));
    kp_graph dg = {n, nnz, d_xadj, d_adj, d_w, d_c};
    PH(coarsen_impl(&dg, o, s, &h));
    const kp_level &top = h->levels.back();
    cw.resize((size_t)std::max(top.n, 1));
    cpart.resize((size_t)std::max(top.n, 1));
    if (top.n > 0)
        PH_CUDA(cudaMemcpyAsync(cw.data(), top.vwgt, sizeof(int32_t) * (size_t)top.n, cudaMemcpyDeviceToHost, s));
    PH_CUDA(cudaStreamSynchronize(s));
    if (ip(top.n, cw.data(), k, cpart.data(), user) != 0) PH(set_error(KP_ERR_INVALID, "initial partition callback failed"));
    PH(dev_alloc_n(&d_cpart, top.n, s));
    if (top.n > 0)
        PH_CUDA(cudaMemcpyAsync(d_cpart, cpart.data(), sizeof(int32_t) * (size_t)top.n, cudaMemcpyHostToDevice, s));
    PH(project_impl(h, d_cpart, d_fpart, s));
    kp_cut_gain_out o2;
    o2.block_w = d_bw;
    o2.gain = d_gain;
    o2.target = d_target;
    PH(cut_gain_impl(&dg, d_fpart, k, eps, &o2, s));
    if (n > 0) {
        if (fine_part) PH_CUDA(cudaMemcpyAsync(fine_part, d_fpart, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToHost, s));
        if (gain) PH_CUDA(cudaMemcpyAsync(gain, d_gain, sizeof(int64_t) * (size_t)n, cudaMemcpyDeviceToHost, s));
        if (target) PH_CUDA(cudaMemcpyAsync(target, d_target, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToHost, s));
    }
    if (block_w) PH_CUDA(cudaMemcpyAsync(block_w, d_bw, sizeof(int64_t) * (size_t)k, cudaMemcpyDeviceToHost, s));
    PH_CUDA(cudaStreamSynchronize(s));
    out->cut = o2.cut;
    out->total_c = o2.total_c;
    out->max_c = o2.max_c;
    out->l_max = o2.l_max;
    out->imbalance = o2.imbalance;
    if (num_levels) *num_levels = (int32_t)h->levels.size();
#undef PH_CUDA
#undef PH
    cleanup();
    return cudaStreamSynchronize(s) == cudaSuccess ? KP_OK : cuda_error(cudaGetLastError(), "final sync");
}

}  // namespace kp
