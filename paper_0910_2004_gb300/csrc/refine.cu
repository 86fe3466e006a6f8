// The data-parallel steps that prepare refinement (Section 5): the quotient
// graph of a partition (which pairs of blocks are adjacent, and how heavily)
// and the bounded breadth-first search from the block boundaries that
// limits local search to a band around the cut.
#include <algorithm>

#include "kp_internal.cuh"

namespace kp {

constexpr int REFINE_BLOCK = 256;
constexpr int32_t QUOTIENT_MAX_K = 4096;   // dense k x k accumulator

// ---------------------------------------------------------------------------
// quotient graph
// ---------------------------------------------------------------------------
// Every directed cut entry adds its weight to cell (p(u), p(v)) of a dense
// k x k matrix.  Rows of at most QROW entries: one thread each, the weight
// towards each other block summed in registers, one atomic per (row, block);
// longer rows: the whole warp, 32 entries at a time, warp-combined atomics.
// With k*k <= QSMEM_CELLS the cells are kept per block in shared memory and
// added to the matrix at the end.  Block ids outside [0,k) set the error flag.
constexpr int QROW = 16;
constexpr int QSMEM_CELLS = 4096;
constexpr int32_t QHUB_ROW = 2048;   // longer rows: a block each (k_quotient_hubs)
constexpr int QHUB_BLOCK = 512;

__device__ __forceinline__ void quotient_row_warp(int32_t u, int32_t pu, eoff beg, eoff end,
                                                  const int32_t *__restrict__ adjncy,
                                                  const int32_t *__restrict__ ewgt,
                                                  const int32_t *__restrict__ part, int32_t k,
                                                  unsigned long long *cells, int32_t *err) {
    const int lane = threadIdx.x & 31;
    (void)u;
    {
        for (eoff e0 = beg; e0 < end; e0 += 32) {   // the same bounds for the whole warp
            const eoff e = e0 + lane;
            int32_t pv = -1;
            int32_t w = 0;
            if (e < end) {
                pv = part[adjncy[e]];
                w = ewgt[e];
                if (pv < 0 || pv >= k) {
                    atomicOr(err, 1);
                    pv = -1;
                }
            }
            const bool cut = pv >= 0 && pv != pu;
            const int key = cut ? pv : -1 - lane;   // lanes without a cut entry: unique keys
            const unsigned peers = __match_any_sync(0xffffffffu, key);
            long long sum = 0;
#pragma unroll
            for (int j = 0; j < 32; j++) {
                const long long wj = __shfl_sync(0xffffffffu, (long long)w, j);
                if ((peers >> j) & 1u) sum += wj;
            }
            if (cut && (peers & ((1u << lane) - 1u)) == 0)
                atomicAdd(&cells[(int64_t)pu * k + pv], (unsigned long long)sum);
        }
    }
}

// Rows longer than QHUB_ROW are listed (hubs, hub_count) for k_quotient_hubs,
// the other rows longer than QROW (mids, mid_count) for k_quotient_mid, whose
// warps take them one at a time: a warp here would walk the long rows of its
// 32 nodes one after the other, and the warps holding several long rows of a
// power-law graph would set the kernel's time.
template <bool SMEM>
__global__ void __launch_bounds__(REFINE_BLOCK) k_quotient_acc(int32_t n, const eoff *__restrict__ xadj,
                                                               const int32_t *__restrict__ adjncy,
                                                               const int32_t *__restrict__ ewgt,
                                                               const int32_t *__restrict__ part, int32_t k,
                                                               unsigned long long *gcells, int32_t *err,
                                                               int32_t *hubs, int32_t *hub_count, int32_t *mids,
                                                               int32_t *mid_count) {
    __shared__ unsigned long long s_cells[SMEM ? QSMEM_CELLS : 1];
    const int64_t kk = (int64_t)k * k;
    if (SMEM) {
        for (int64_t i = threadIdx.x; i < kk; i += blockDim.x) s_cells[i] = 0;
        __syncthreads();
    }
    unsigned long long *cells = SMEM ? s_cells : gcells;
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v0 = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); v0 < n; v0 += stride) {
        const int64_t u = v0 + lane;
        int32_t pu = -1, d = 0;
        eoff beg = 0;
        if (u < n) {
            pu = part[u];
            beg = xadj[u];
            d = (int32_t)(xadj[u + 1] - beg);
            if (pu < 0 || pu >= k) {
                atomicOr(err, 1);
                pu = -1;
            }
        }
        if (pu >= 0 && d <= QROW) {
            int32_t b[QROW], w[QROW];
#pragma unroll
            for (int i = 0; i < QROW; i++) {
                if (i >= d) break;
                b[i] = adjncy[beg + i];
            }
#pragma unroll
            for (int i = 0; i < QROW; i++) {
                if (i >= d) break;
                w[i] = ewgt[beg + i];
            }
            bool any_cut = false;
#pragma unroll
            for (int i = 0; i < QROW; i++) {
                if (i >= d) break;
                const int32_t pb = part[b[i]];
                if (pb < 0 || pb >= k) {
                    atomicOr(err, 1);
                    b[i] = pu;   // skipped below
                } else {
                    b[i] = pb;
                    any_cut |= pb != pu;
                }
            }
            if (any_cut) {
#pragma unroll
                for (int i = 0; i < QROW; i++) {
                    if (i >= d) break;
                    if (b[i] == pu) continue;
                    bool first = true;
                    long long sum = 0;
#pragma unroll
                    for (int j = 0; j < QROW; j++) {
                        if (j >= d) break;
                        if (b[j] == b[i]) {
                            if (j < i) first = false;
                            sum += w[j];
                        }
                    }
                    if (first) atomicAdd(&cells[(int64_t)pu * k + b[i]], (unsigned long long)sum);
                }
            }
        }
        // the long rows of this warp's 32 nodes go to their lists
        // (warp-aggregated appends)
        const bool hub = pu >= 0 && d > QHUB_ROW, mid = pu >= 0 && d > QROW && !hub;
        unsigned m = __ballot_sync(0xffffffffu, hub);
        if (m) {
            int32_t base = 0;
            if (lane == 0) base = atomicAdd(hub_count, __popc(m));
            base = __shfl_sync(0xffffffffu, base, 0);
            if (hub) hubs[base + __popc(m & ((1u << lane) - 1u))] = (int32_t)u;
        }
        m = __ballot_sync(0xffffffffu, mid);
        if (m) {
            int32_t base = 0;
            if (lane == 0) base = atomicAdd(mid_count, __popc(m));
            base = __shfl_sync(0xffffffffu, base, 0);
            if (mid) mids[base + __popc(m & ((1u << lane) - 1u))] = (int32_t)u;
        }
    }
    if (SMEM) {
        __syncthreads();
        for (int64_t i = threadIdx.x; i < kk; i += blockDim.x)
            if (s_cells[i]) atomicAdd(&gcells[i], s_cells[i]);
    }
}

// The listed hub rows, one block each: the weight towards every block is
// summed in shared memory in one pass over the row (k 64-bit sums), then
// each nonzero sum is added to its cell of the dense matrix.
__global__ void __launch_bounds__(QHUB_BLOCK) k_quotient_hubs(const eoff *__restrict__ xadj,
                                                              const int32_t *__restrict__ adjncy,
                                                              const int32_t *__restrict__ ewgt,
                                                              const int32_t *__restrict__ part, int32_t k,
                                                              const int32_t *__restrict__ hubs,
                                                              const int32_t *hub_count, unsigned long long *gcells,
                                                              int32_t *err) {
    extern __shared__ unsigned long long s_bins[];
    const int32_t count = *hub_count;
    for (int32_t i = blockIdx.x; i < count; i += gridDim.x) {
        const int32_t u = hubs[i];
        const int32_t pu = part[u];   // checked by the row kernel
        for (int32_t b = threadIdx.x; b < k; b += blockDim.x) s_bins[b] = 0;
        __syncthreads();
        const eoff beg = xadj[u], end = xadj[u + 1];
        for (eoff e = beg + threadIdx.x; e < end; e += blockDim.x) {
            const int32_t pv = part[adjncy[e]];
            if (pv < 0 || pv >= k) {
                atomicOr(err, 1);
                continue;
            }
            if (pv != pu) atomicAdd(&s_bins[pv], (unsigned long long)ewgt[e]);
        }
        __syncthreads();
        for (int32_t b = threadIdx.x; b < k; b += blockDim.x)
            if (s_bins[b]) atomicAdd(&gcells[(int64_t)pu * k + b], s_bins[b]);
        __syncthreads();
    }
}

// The listed long rows (QROW < d <= QHUB_ROW), one warp per row taken from a
// counter (cells per block in shared memory when k*k <= QSMEM_CELLS).
template <bool SMEM>
__global__ void __launch_bounds__(REFINE_BLOCK) k_quotient_mid(const eoff *__restrict__ xadj,
                                                               const int32_t *__restrict__ adjncy,
                                                               const int32_t *__restrict__ ewgt,
                                                               const int32_t *__restrict__ part, int32_t k,
                                                               const int32_t *__restrict__ mids,
                                                               const int32_t *mid_count, int32_t *next,
                                                               unsigned long long *gcells, int32_t *err) {
    __shared__ unsigned long long s_cells[SMEM ? QSMEM_CELLS : 1];
    const int64_t kk = (int64_t)k * k;
    if (SMEM) {
        for (int64_t i = threadIdx.x; i < kk; i += blockDim.x) s_cells[i] = 0;
        __syncthreads();
    }
    unsigned long long *cells = SMEM ? s_cells : gcells;
    const int lane = threadIdx.x & 31;
    const int32_t count = *mid_count;
    for (;;) {
        int32_t i = 0;
        if (lane == 0) i = atomicAdd(next, 1);
        i = __shfl_sync(0xffffffffu, i, 0);
        if (i >= count) break;
        const int32_t u = mids[i];
        const eoff beg = xadj[u], end = xadj[u + 1];
        quotient_row_warp(u, part[u], beg, end, adjncy, ewgt, part, k, cells, err);
    }
    if (SMEM) {
        __syncthreads();
        for (int64_t i = threadIdx.x; i < kk; i += blockDim.x)
            if (s_cells[i]) atomicAdd(&gcells[i], s_cells[i]);
    }
}

// Nonzero cells per row (one warp per block row).
__global__ void k_quotient_count(int32_t k, const unsigned long long *__restrict__ cells, int32_t *q_xadj) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t a = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; a < k; a += warps) {
        int32_t c = 0;
        for (int32_t b = lane; b < k; b += 32) c += cells[a * k + b] != 0ull;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
        if (lane == 0) q_xadj[a + 1] = c;
    }
}

// Exclusive scan of the k row counts in one block (k <= QUOTIENT_MAX_K).
__global__ void k_quotient_scan(int32_t k, int32_t *q_xadj, long long *nnz_out) {
    __shared__ int32_t s[QUOTIENT_MAX_K + 1];
    for (int32_t i = threadIdx.x; i < k; i += blockDim.x) s[i] = q_xadj[i + 1];
    __syncthreads();
    if (threadIdx.x == 0) {
        int32_t run = 0;
        for (int32_t i = 0; i < k; i++) {
            const int32_t c = s[i];
            s[i] = run;
            run += c;
        }
        s[k] = run;
        *nnz_out = run;
    }
    __syncthreads();
    for (int32_t i = threadIdx.x; i <= k; i += blockDim.x) q_xadj[i] = s[i];
}

// Row a of the quotient CSR: the nonzero cells in ascending b (one warp per
// row, ballot ranks keep the order).
__global__ void k_quotient_write(int32_t k, const unsigned long long *__restrict__ cells,
                                 const int32_t *__restrict__ q_xadj, int64_t capacity, int32_t *q_adjncy,
                                 int64_t *q_ewgt) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t a = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; a < k; a += warps) {
        int32_t pos = q_xadj[a];
        if ((int64_t)q_xadj[k] > capacity) continue;   // the caller's buffers are too small
        for (int32_t b0 = 0; b0 < k; b0 += 32) {
            const int32_t b = b0 + lane;
            const unsigned long long c = b < k ? cells[a * k + b] : 0ull;
            const unsigned m = __ballot_sync(0xffffffffu, c != 0ull);
            if (c != 0ull) {
                const int32_t r = pos + __popc(m & ((1u << lane) - 1u));
                q_adjncy[r] = b;
                q_ewgt[r] = (int64_t)c;
            }
            pos += __popc(m);
        }
    }
}

// ---------------------------------------------------------------------------
// bounded breadth-first search from the boundary
// ---------------------------------------------------------------------------
// Distance 0 for boundary nodes (a neighbour in another block; with a pair,
// a node of one pair block with a neighbour in the other), -1 for the other
// nodes that take part, -2 for nodes outside the pair.  Boundary nodes form
// the first frontier (warp-aggregated appends).
__global__ void __launch_bounds__(REFINE_BLOCK) k_band_init(int32_t n, const eoff *__restrict__ xadj,
                                                            const int32_t *__restrict__ adjncy,
                                                            const int32_t *__restrict__ part, int32_t k,
                                                            int32_t pa, int32_t pb, int32_t *dist,
                                                            int32_t *frontier, int32_t *count, int32_t *err) {
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v0 = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); v0 < n; v0 += stride) {
        const int64_t v = v0 + lane;
        bool src = false;
        if (v < n) {
            const int32_t pv = part[v];
            if (pv < 0 || pv >= k) {
                atomicOr(err, 1);
                dist[v] = -2;
            } else if (pa >= 0 && pv != pa && pv != pb) {
                dist[v] = -2;
            } else {
                const int32_t want = pa < 0 ? -1 : (pv == pa ? pb : pa);   // -1: any other block
                for (eoff e = xadj[v]; e < xadj[v + 1]; e++) {
                    const int32_t pu = part[adjncy[e]];
                    if (pu < 0 || pu >= k) {
                        atomicOr(err, 1);
                        continue;
                    }
                    if (pu != pv && (want < 0 || pu == want)) {
                        src = true;
                        break;
                    }
                }
                dist[v] = src ? 0 : -1;
            }
        }
        const unsigned m = __ballot_sync(0xffffffffu, src);
        int32_t base = 0;
        if (lane == 0 && m) base = atomicAdd(count, __popc(m));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (src) frontier[base + __popc(m & ((1u << lane) - 1u))] = (int32_t)v;
    }
}

// One breadth-first step.  Push (small frontier): every frontier node claims
// its unvisited neighbours of the same block (the first claim wins; the
// distance is the same whoever claims).  Pull (frontier above n/16): every
// unvisited node looks for a same-block neighbour at distance depth-1 and
// takes depth itself, no atomics on dist.  The choice is made on the device
// from the frontier size, the same for every block.  New nodes are appended
// to the next frontier either way.
__global__ void __launch_bounds__(REFINE_BLOCK) k_band_step(int32_t n, const eoff *__restrict__ xadj,
                                                            const int32_t *__restrict__ adjncy,
                                                            const int32_t *__restrict__ part, int32_t *dist,
                                                            const int32_t *frontier, const int32_t *count,
                                                            int32_t *next, int32_t *next_count, int32_t depth) {
    const int lane = threadIdx.x & 31;
    const int64_t cnt = *count;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    if (cnt * 16 > n) {
        for (int64_t v0 = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); v0 < n; v0 += stride) {
            const int64_t v = v0 + lane;
            bool found = false;
            if (v < n && dist[v] == -1) {
                const int32_t pv = part[v];
                for (eoff e = xadj[v]; e < xadj[v + 1]; e++) {
                    const int32_t u = adjncy[e];
                    if (dist[u] == depth - 1 && part[u] == pv) {
                        found = true;
                        break;
                    }
                }
            }
            // this step writes only the value `depth` and the test above looks
            // for depth-1 (set by the previous step), so what other threads
            // write meanwhile cannot change any decision
            const unsigned m = __ballot_sync(0xffffffffu, found);
            int32_t base = 0;
            if (lane == 0 && m) base = atomicAdd(next_count, __popc(m));
            base = __shfl_sync(0xffffffffu, base, 0);
            if (found) {
                dist[v] = depth;
                next[base + __popc(m & ((1u << lane) - 1u))] = (int32_t)v;
            }
        }
        return;
    }
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); i0 < cnt; i0 += stride) {
        const int64_t i = i0 + lane;
        int32_t u = -1, pu = -1;
        eoff beg = 0, end = 0;
        if (i < cnt) {
            u = frontier[i];
            beg = xadj[u];
            end = xadj[u + 1];
            pu = part[u];
        }
        // a warp walks its frontier nodes' rows together, one entry per lane
        // per step, so long rows do not serialise behind short ones
        for (int32_t j = 0;; j++) {
            const bool live = u >= 0 && beg + j < end;
            if (!__any_sync(0xffffffffu, live)) break;
            bool claimed = false;
            int32_t v = -1;
            if (live) {
                v = adjncy[beg + j];
                if (part[v] == pu && dist[v] == -1) claimed = atomicCAS(&dist[v], -1, depth) == -1;
            }
            const unsigned m = __ballot_sync(0xffffffffu, claimed);
            int32_t base = 0;
            if (lane == 0 && m) base = atomicAdd(next_count, __popc(m));
            base = __shfl_sync(0xffffffffu, base, 0);
            if (claimed) next[base + __popc(m & ((1u << lane) - 1u))] = v;
        }
    }
}

namespace {

kp_status check_refine_args(const kp_graph *g, const int32_t *part, int32_t k) {
    if (!g) return set_error(KP_ERR_INVALID, "null argument");
    if (k < 1) return set_error(KP_ERR_INVALID, "k must be >= 1");
    if (g->n < 0 || g->nnz < 0) return set_error(KP_ERR_INVALID, "negative graph size");
    if ((int64_t)g->nnz >= NNZ_LIMIT) return set_error(KP_ERR_OVERFLOW, "nnz >= 2^32: the edge weights sum to 2^31 or more");
    if (g->n > 0 && (!part || !g->xadj || (g->nnz > 0 && (!g->adjncy || !g->ewgt))))
        return set_error(KP_ERR_INVALID, "null array");
    return KP_OK;
}

int grid_for(int64_t threads) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((threads + REFINE_BLOCK - 1) / REFINE_BLOCK,
                                                       (int64_t)num_sms() * 8));
}

}  // namespace

kp_status quotient_graph_impl(const kp_graph *g, const int32_t *part, int32_t k, int32_t *q_xadj,
                              int32_t *q_adjncy, int64_t *q_ewgt, int64_t capacity, int64_t *q_nnz,
                              cudaStream_t s) {
    KP_TRY(check_refine_args(g, part, k));
    if (!q_xadj || !q_nnz || capacity < 0 || (capacity > 0 && (!q_adjncy || !q_ewgt)))
        return set_error(KP_ERR_INVALID, "null output");
    if (k > QUOTIENT_MAX_K) return set_error(KP_ERR_UNSUPPORTED, "quotient graph: k above 4096");
    unsigned long long *cells = nullptr;
    int32_t *err = nullptr;   // [0] block id error, [1] hub rows, [2] long rows, [3] long rows taken
    int32_t *hubs = nullptr, *mids = nullptr;
    long long *nnz_dev = nullptr;
    const bool smem = (int64_t)k * k <= QSMEM_CELLS;
    KP_TRY(dev_alloc_n(&cells, (int64_t)k * k, s));
    kp_status st = dev_alloc_n(&err, 4, s);
    if (st == KP_OK) st = dev_alloc_n(&nnz_dev, 1, s);
    if (st == KP_OK) st = dev_alloc_n(&hubs, (int64_t)g->nnz / QHUB_ROW + 1, s);
    if (st == KP_OK) st = dev_alloc_n(&mids, (int64_t)g->nnz / (QROW + 1) + 1, s);
    auto done = [&](kp_status r) {
        dev_free(cells, s);
        dev_free(err, s);
        dev_free(nnz_dev, s);
        dev_free(hubs, s);
        dev_free(mids, s);
        return r;
    };
    if (st != KP_OK) return done(st);
    if (cudaMemsetAsync(cells, 0, sizeof(unsigned long long) * (size_t)k * k, s) != cudaSuccess ||
        cudaMemsetAsync(err, 0, 4 * sizeof(int32_t), s) != cudaSuccess ||
        cudaMemsetAsync(q_xadj, 0, sizeof(int32_t), s) != cudaSuccess)
        return done(cuda_error(cudaGetLastError(), "clear"));
    if (g->n > 0) {
        if (smem)
            k_quotient_acc<true><<<grid_for(g->n), REFINE_BLOCK, 0, s>>>(g->n, g->xadj, g->adjncy, g->ewgt, part, k,
                                                                         cells, err, hubs, err + 1, mids, err + 2);
        else
            k_quotient_acc<false><<<grid_for(g->n), REFINE_BLOCK, 0, s>>>(g->n, g->xadj, g->adjncy, g->ewgt, part, k,
                                                                          cells, err, hubs, err + 1, mids, err + 2);
        if (g->nnz > QROW) {
            if (smem)
                k_quotient_mid<true><<<num_sms() * 4, REFINE_BLOCK, 0, s>>>(g->xadj, g->adjncy, g->ewgt, part, k, mids,
                                                                            err + 2, err + 3, cells, err);
            else
                k_quotient_mid<false><<<num_sms() * 8, REFINE_BLOCK, 0, s>>>(g->xadj, g->adjncy, g->ewgt, part, k, mids,
                                                                             err + 2, err + 3, cells, err);
        }
        if (g->nnz > QHUB_ROW)
            k_quotient_hubs<<<num_sms() * 2, QHUB_BLOCK, sizeof(unsigned long long) * (size_t)k, s>>>(
                g->xadj, g->adjncy, g->ewgt, part, k, hubs, err + 1, cells, err);
    }
    k_quotient_count<<<grid_for((int64_t)k * 32), REFINE_BLOCK, 0, s>>>(k, cells, q_xadj);
    k_quotient_scan<<<1, 1024, 0, s>>>(k, q_xadj, nnz_dev);
    k_quotient_write<<<grid_for((int64_t)k * 32), REFINE_BLOCK, 0, s>>>(k, cells, q_xadj, capacity, q_adjncy,
                                                                        q_ewgt);
    if (cudaGetLastError() != cudaSuccess) return done(cuda_error(cudaGetLastError(), "quotient kernels"));
    int32_t herr = 0;
    long long hnnz = 0;
    if (cudaMemcpyAsync(&herr, err, sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(&hnnz, nnz_dev, sizeof(long long), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return done(cuda_error(cudaGetLastError(), "quotient readback"));
    *q_nnz = hnnz;
    if (herr) return done(set_error(KP_ERR_INVALID, "block id outside [0,k)"));
    if (hnnz > capacity) return done(set_error(KP_ERR_OVERFLOW, "quotient graph larger than the capacity"));
    return done(KP_OK);
}

kp_status boundary_band_impl(const kp_graph *g, const int32_t *part, int32_t k, int32_t depth, int32_t pa,
                             int32_t pb, int32_t *dist, cudaStream_t s) {
    KP_TRY(check_refine_args(g, part, k));
    if (depth < 0) return set_error(KP_ERR_INVALID, "negative depth");
    if ((pa >= 0) != (pb >= 0) || pa >= k || pb >= k || (pa >= 0 && pa == pb))
        return set_error(KP_ERR_INVALID, "pair must be two different blocks in [0,k) or (-1,-1)");
    if (g->n > 0 && !dist) return set_error(KP_ERR_INVALID, "null dist");
    if (g->n == 0) return KP_OK;
    const int32_t n = g->n;
    int32_t *fa = nullptr, *fb = nullptr, *counts = nullptr, *err = nullptr;
    kp_status st = dev_alloc_n(&fa, n, s);
    if (st == KP_OK) st = dev_alloc_n(&fb, n, s);
    if (st == KP_OK) st = dev_alloc_n(&counts, (int64_t)depth + 1, s);
    if (st == KP_OK) st = dev_alloc_n(&err, 1, s);
    auto done = [&](kp_status r) {
        dev_free(fa, s);
        dev_free(fb, s);
        dev_free(counts, s);
        dev_free(err, s);
        return r;
    };
    if (st != KP_OK) return done(st);
    if (cudaMemsetAsync(counts, 0, sizeof(int32_t) * ((size_t)depth + 1), s) != cudaSuccess ||
        cudaMemsetAsync(err, 0, sizeof(int32_t), s) != cudaSuccess)
        return done(cuda_error(cudaGetLastError(), "clear"));
    k_band_init<<<grid_for(n), REFINE_BLOCK, 0, s>>>(n, g->xadj, g->adjncy, part, k, pa, pb, dist, fa, counts, err);
    // each step reads the frontier size on the device: no host round trip
    for (int32_t d = 1; d <= depth; d++) {
        int32_t *cur = (d & 1) ? fa : fb, *nxt = (d & 1) ? fb : fa;
        k_band_step<<<grid_for(n), REFINE_BLOCK, 0, s>>>(n, g->xadj, g->adjncy, part, dist, cur, counts + d - 1, nxt,
                                                        counts + d, d);
    }
    if (cudaGetLastError() != cudaSuccess) return done(cuda_error(cudaGetLastError(), "band kernels"));
    int32_t herr = 0;
    if (cudaMemcpyAsync(&herr, err, sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return done(cuda_error(cudaGetLastError(), "band readback"));
    if (herr) return done(set_error(KP_ERR_INVALID, "block id outside [0,k)"));
    return done(KP_OK);
}

}  // namespace kp

extern "C" {

kp_status kp_quotient_graph(const kp_graph *g, const int32_t *part, int32_t k, int32_t *q_xadj, int32_t *q_adjncy,
                            int64_t *q_ewgt, int64_t capacity, int64_t *q_nnz, kp_stream s) {
    return kp::quotient_graph_impl(g, part, k, q_xadj, q_adjncy, q_ewgt, capacity, q_nnz, (cudaStream_t)s);
}

kp_status kp_boundary_band(const kp_graph *g, const int32_t *part, int32_t k, int32_t depth, int32_t pair_a,
                           int32_t pair_b, int32_t *dist, kp_stream s) {
    return kp::boundary_band_impl(g, part, k, depth, pair_a, pair_b, dist, (cudaStream_t)s);
}

}  // extern "C"
