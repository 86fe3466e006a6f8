// Contraction of one level (Section 2): the per-phase kernels over the
// device functions of contract.cuh, and their launchers.
#include <algorithm>

#include "contract.cuh"

namespace kp {

// 4 resident blocks per SM (64 registers) measured best for the small rows
__global__ void __launch_bounds__(CONTRACT_BLOCK, 4) k_contract_small(DevState *st, int level, Work w,
                                                                       int32_t huge_row) {
    phase_contract_small(st, level, w, huge_row, WARP_ROW);
}

__global__ void __launch_bounds__(CONTRACT_BLOCK) k_contract_rows32(DevState *st, int level, Work w) {
    phase_contract_rows32(st, level, w);
}

__global__ void __launch_bounds__(CONTRACT_BLOCK) k_contract_overflow(DevState *st, int level, Work w) {
    __shared__ OverflowSmem sm;
    // 2 radix entries per thread and chunk keep the kernel at 48 registers,
    // so the many-warp classes run at full occupancy and the classes overlap
    phase_contract_overflow<true, true, 2, false>(st, level, w, sm);
}

// ---------------------------------------------------------------------------
// rows of more than HUGE_ROW gathered entries (hubs of power-law graphs):
// one thread-block cluster per row.  Every step of the radix path of
// contract_block_radix is split over the cluster's CTAs: each gathers,
// counts and scatters a contiguous share of the row.  The per-digit counts
// of all CTAs are combined through distributed shared memory, so that CTA r
// places its entries of digit d after those of CTAs 0..r-1 (the sort stays
// stable, hence exact), and the hardware cluster barrier separates the
// steps.  One block alone would walk such a row chunk after chunk while the
// rest of the level waits for it.
// ---------------------------------------------------------------------------
constexpr int HUGE_ITEMS = 4;                                 // entries per thread and chunk
constexpr int HUGE_CHUNK = CONTRACT_BLOCK * HUGE_ITEMS;

struct HugeSmem {
    int32_t hist[256];        // this CTA's digit counts of the current pass
    int32_t base[256];        // where this CTA's next entry of each digit goes
    int32_t chunk_tot[256];
    int32_t wcnt[CONTRACT_BLOCK / 32][256];
    int32_t wsum[CONTRACT_BLOCK / 32];
    int32_t s_red[CONTRACT_BLOCK / 32];
    int32_t kept;             // gather: entries this CTA kept; merge: its run heads
    int32_t carry;
    int32_t wtot;             // merge: this CTA's weight sum
};

__device__ __forceinline__ unsigned cluster_rank() {
    unsigned r;
    asm("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ unsigned cluster_index() {
    unsigned r;
    asm("mov.u32 %0, %%clusterid.x;" : "=r"(r));
    return r;
}

__device__ __forceinline__ unsigned cluster_count() {
    unsigned r;
    asm("mov.u32 %0, %%nclusterid.x;" : "=r"(r));
    return r;
}

// The word at `p` (a shared-memory variable) in the CTA of the cluster with
// the given rank.
__device__ __forceinline__ int32_t dsmem_ld(const int32_t *p, unsigned rank) {
    const uint32_t local = (uint32_t)__cvta_generic_to_shared(p);
    uint32_t remote;
    int32_t v;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(local), "r"(rank));
    asm volatile("ld.shared::cluster.s32 %0, [%1];" : "=r"(v) : "r"(remote) : "memory");
    return v;
}

// Sum over the cluster's CTAs of a shared word, and the part of CTAs below
// `rank`.
__device__ __forceinline__ void dsmem_sums(const int32_t *p, unsigned ctas, unsigned rank, int32_t &all,
                                           int32_t &below) {
    all = 0;
    below = 0;
    for (unsigned r = 0; r < ctas; r++) {
        const int32_t v = r == rank ? *p : dsmem_ld(p, r);
        all += v;
        if (r < rank) below += v;
    }
}

// Ranks and scatters the entries [lo, hi) of src (this CTA's share) by the
// digit at `shift`, chunk by chunk; sm.base holds where this CTA's entries
// of each digit start.  Within a chunk the entries keep their index order
// (warps in order, items in order, lanes in order).
__device__ __forceinline__ void huge_scatter(const int32_t *src_k, const int32_t *src_v, int32_t *dst_k,
                                             int32_t *dst_v, int32_t lo, int32_t hi, int shift, int32_t dmask,
                                             HugeSmem &sm) {
    constexpr int NW = CONTRACT_BLOCK / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt = lanemask_lt();
    for (int32_t c0 = lo; c0 < hi; c0 += HUGE_CHUNK) {
#pragma unroll
        for (int j = 0; j < 256 / 32; j++) sm.wcnt[warp][j * 32 + lane] = 0;
        __syncwarp();
        int32_t kk[HUGE_ITEMS], vv[HUGE_ITEMS], rk[HUGE_ITEMS];
#pragma unroll
        for (int j = 0; j < HUGE_ITEMS; j++) {
            const int32_t i = c0 + (warp * HUGE_ITEMS + j) * 32 + lane;
            kk[j] = i < hi ? __ldcg(src_k + i) : 0;
            vv[j] = i < hi ? __ldcg(src_v + i) : 0;
        }
#pragma unroll
        for (int j = 0; j < HUGE_ITEMS; j++) {
            const int32_t i = c0 + (warp * HUGE_ITEMS + j) * 32 + lane;
            const bool valid = i < hi;
            const int d = valid ? ((kk[j] >> shift) & dmask) : 256 + lane;   // invalid lanes: unique
            const unsigned peers = __match_any_sync(0xffffffffu, d);
            const int wr = __popc(peers & lt);
            rk[j] = valid ? sm.wcnt[warp][d] + wr : 0;
            __syncwarp();
            if (valid && wr == 0) sm.wcnt[warp][d] += __popc(peers);
            __syncwarp();
        }
        __syncthreads();
        {
            int32_t run = 0;
#pragma unroll
            for (int w2 = 0; w2 < NW; w2++) {
                const int32_t c = sm.wcnt[w2][threadIdx.x];
                sm.wcnt[w2][threadIdx.x] = run;
                run += c;
            }
            sm.chunk_tot[threadIdx.x] = run;
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < HUGE_ITEMS; j++) {
            const int32_t i = c0 + (warp * HUGE_ITEMS + j) * 32 + lane;
            if (i < hi) {
                const int d = (kk[j] >> shift) & dmask;
                const int32_t r = sm.base[d] + sm.wcnt[warp][d] + rk[j];
                dst_k[r] = kk[j];
                dst_v[r] = vv[j];
            }
        }
        __syncthreads();
        sm.base[threadIdx.x] += sm.chunk_tot[threadIdx.x];
        __syncthreads();
    }
}

// One huge row x by the whole cluster (every CTA calls it with the same x).
// Steps as contract_block_radix: gather, `passes` radix passes between tmp
// and big, merge of equal neighbours from big into tmp.  The row's slot
// holds only the kept entries (a pair's two entries of the contracted edge
// are dropped, wherever they fall), so the gather first counts each CTA's
// kept entries and then writes them packed after those of the CTAs below:
// every write stays inside [0, M) of the slot.  Pass 0 reads each CTA's
// packed entries, later passes and the merge equal shares of [0, M).
__device__ void contract_cluster_radix(const CView &p, int32_t x, int passes, HugeSmem &sm) {
    const unsigned ctas = cluster_ctas(), rank = cluster_rank();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int NW = CONTRACT_BLOCK / 32;
    const unsigned lt = lanemask_lt();
    eoff xa, xb;
    int32_t da, db;
    members(p, x, xa, da, xb, db);
    const int32_t L = da + db;
    const eoff o = p.off[x];
    int32_t *src_k = (passes & 1) ? p.tmp_adj + o : p.big_adj + o;
    int32_t *src_v = (passes & 1) ? p.tmp_w + o : p.big_w + o;
    int32_t *dst_k = (passes & 1) ? p.big_adj + o : p.tmp_adj + o;
    int32_t *dst_v = (passes & 1) ? p.big_w + o : p.tmp_w + o;
    const int rb = p.radix_bits;
    const int32_t dmask = (1 << rb) - 1;
    const int32_t per = (L + (int32_t)ctas - 1) / (int32_t)ctas;
    const int32_t lo = min(L, (int32_t)rank * per), hi = min(L, lo + per);

    // 1a. count the kept entries of this CTA's share and their pass-0 digits
    sm.hist[threadIdx.x] = 0;
    if (threadIdx.x == 0) {
        sm.kept = 0;
        sm.carry = 0;
    }
    __syncthreads();
    for (int32_t c0 = lo; c0 < hi; c0 += CONTRACT_BLOCK) {
        const int32_t i = c0 + (int32_t)threadIdx.x;
        int32_t t = x;
        if (i < hi) t = p.map[p.adjncy[i < da ? xa + i : xb + (i - da)]];
        const bool keep = i < hi && t != x;
        const unsigned m = __ballot_sync(0xffffffffu, keep);
        if (lane == 0 && m) atomicAdd(&sm.kept, __popc(m));
        if (keep) atomicAdd(&sm.hist[t & dmask], 1);
    }
    __syncthreads();
    cluster_barrier();   // every CTA's kept count and digit counts
    int32_t M, kept_below;
    dsmem_sums(&sm.kept, ctas, rank, M, kept_below);
    const int32_t kept = sm.kept;
    const int32_t perM = (M + (int32_t)ctas - 1) / (int32_t)ctas;
    const int32_t mlo = min(M, (int32_t)rank * perM), mhi = min(M, mlo + perM);
    // 1b. gather again, packed at [kept_below, kept_below + kept) (the order
    //     within it does not matter: the entries are sorted next)
    for (int32_t c0 = lo; c0 < hi; c0 += CONTRACT_BLOCK) {
        const int32_t i = c0 + (int32_t)threadIdx.x;
        int32_t t = x, wv = 0;
        if (i < hi) {
            const eoff e = i < da ? xa + i : xb + (i - da);
            t = p.map[p.adjncy[e]];
            wv = p.ewgt[e];
        }
        const bool keep = i < hi && t != x;
        const unsigned m = __ballot_sync(0xffffffffu, keep);
        int32_t at = 0;
        if (lane == 0 && m) at = atomicAdd(&sm.carry, __popc(m));
        at = __shfl_sync(0xffffffffu, at, 0);
        if (keep) {
            const int32_t r = kept_below + at + __popc(m & lt);
            src_k[r] = t;
            src_v[r] = wv;
        }
    }
    __syncthreads();   // pass 0 reads only this CTA's own entries

    // 2. radix passes
    for (int pass = 0; pass < passes; pass++) {
        const int shift = rb * pass;
        int32_t in_lo = kept_below, in_hi = kept_below + kept;
        if (pass > 0) {
            in_lo = mlo;
            in_hi = mhi;
            sm.hist[threadIdx.x] = 0;   // the others read this CTA's counts before the last barrier
            __syncthreads();
            for (int32_t i = in_lo + (int32_t)threadIdx.x; i < in_hi; i += CONTRACT_BLOCK)
                atomicAdd(&sm.hist[(__ldcg(src_k + i) >> shift) & dmask], 1);
            __syncthreads();
            cluster_barrier();
        }
        {
            int32_t all, below;
            dsmem_sums(&sm.hist[threadIdx.x], ctas, rank, all, below);
            uint64_t tot;
            const int32_t excl = (int32_t)block_exclusive_scan<CONTRACT_BLOCK>((uint64_t)all, &tot);
            sm.base[threadIdx.x] = excl + below;
        }
        __syncthreads();
        huge_scatter(src_k, src_v, dst_k, dst_v, in_lo, in_hi, shift, dmask, sm);
        cluster_barrier();   // the pass's output is complete; the counts have been read
        int32_t *tk = src_k, *tv = src_v;
        src_k = dst_k;
        src_v = dst_v;
        dst_k = tk;
        dst_v = tv;
    }

    // 3. merge equal neighbours from big (src) into tmp; run r of the row
    //    goes to tmp[o + r] (r is at most the run's first index)
    for (int32_t i = mlo + (int32_t)threadIdx.x; i < mhi; i += CONTRACT_BLOCK) p.tmp_w[o + i] = 0;
    {
        int32_t h = 0;
        for (int32_t i = mlo + (int32_t)threadIdx.x; i < mhi; i += CONTRACT_BLOCK)
            h += (i == 0 || __ldcg(src_k + i - 1) != __ldcg(src_k + i)) ? 1 : 0;
        for (int off2 = 16; off2 > 0; off2 >>= 1) h += __shfl_xor_sync(0xffffffffu, h, off2);
        if (lane == 0) sm.s_red[warp] = h;
        __syncthreads();
        if (threadIdx.x == 0) {
            int32_t t = 0;
            for (int w2 = 0; w2 < NW; w2++) t += sm.s_red[w2];
            sm.kept = t;   // every CTA read the kept counts before the first pass
            sm.carry = 0;
        }
        __syncthreads();
    }
    cluster_barrier();   // zeroed sums and every CTA's head count
    int32_t runs, runs_below;
    dsmem_sums(&sm.kept, ctas, rank, runs, runs_below);
    int32_t wsum = 0;
    for (int32_t c0 = mlo; c0 < mhi; c0 += CONTRACT_BLOCK) {
        const int32_t i = c0 + (int32_t)threadIdx.x;
        const bool valid = i < mhi;
        const int32_t k = valid ? __ldcg(src_k + i) : SENT;
        const bool head = valid && (i == 0 || __ldcg(src_k + i - 1) != k);
        const unsigned hm = __ballot_sync(0xffffffffu, head);
        if (lane == 0) sm.wsum[warp] = __popc(hm);
        __syncthreads();
        int32_t before = runs_below + sm.carry;
        for (int w2 = 0; w2 < warp; w2++) before += sm.wsum[w2];
        if (valid) {
            // run index: heads up to and including this entry, minus one
            const int32_t r = before + __popc(hm & (lt | (1u << lane))) - 1;
            const int32_t v = __ldcg(src_v + i);
            if (head) p.tmp_adj[o + r] = k;
            atomicAdd(&p.tmp_w[o + r], v);
            wsum += v;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int32_t t = sm.carry;
            for (int w2 = 0; w2 < NW; w2++) t += sm.wsum[w2];
            sm.carry = t;
        }
        __syncthreads();
    }
    for (int off2 = 16; off2 > 0; off2 >>= 1) wsum += __shfl_xor_sync(0xffffffffu, wsum, off2);
    if (lane == 0) sm.s_red[warp] = wsum;
    __syncthreads();
    if (threadIdx.x == 0) {
        int32_t t = 0;
        for (int w2 = 0; w2 < NW; w2++) t += sm.s_red[w2];
        sm.wtot = t;
    }
    cluster_barrier();   // every CTA's weight sum; the merged row is complete
    if (rank == 0 && threadIdx.x == 0) {
        int32_t wt, unused;
        dsmem_sums(&sm.wtot, ctas, rank, wt, unused);
        p.degp[x] = runs;
        if (runs >= 1024) atomicMax(&p.ctr->maxdeg, runs);
        if (p.outw) p.outw[x] = wt;
    }
    cluster_barrier();   // CTA 0 has read the others' sums before they move on
}

// The huge rows of the level (class 5), one cluster per row in turn.
__global__ void __launch_bounds__(CONTRACT_BLOCK) k_contract_huge(DevState *st, int level, Work w) {
    __shared__ HugeSmem sm;
    CView p;
    // the level's flags and counts were written by earlier launches: every
    // CTA of a cluster takes the same decisions and meets the same barriers
    if (!load_view(st, level, w, p)) return;
    const int32_t count = p.ctr->nclass[5];
    if (count == 0) return;
    int bits = 1;
    while (bits < 31 && ((int64_t)1 << bits) < (int64_t)p.cn) bits++;
    const int passes = (bits + p.radix_bits - 1) / p.radix_bits;
    for (int32_t li = (int32_t)cluster_index(); li < count; li += (int32_t)cluster_count())
        contract_cluster_radix(p, p.lists[5][li], passes, sm);
}

__global__ void k_compact(DevState *st, int level, Work w) { phase_compact(st, level, w); }

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
kp_status launch_relabel(const LevelLaunch &L, cudaStream_t s, int32_t *launches) {
    const int64_t tiles = scan_tiles(std::max<int64_t>(1, L.n_bound));
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)num_sms() * 4));
    if (L.matcher == KP_MATCHER_SUITOR) {
        RelabelOp<true> op;
        op.st = L.st;
        op.level = L.level;
        op.w = L.w;
        k_scan_lb<RelabelOp<true>><<<grid, SCAN_BLOCK, 0, s>>>(op, L.w.status, L.epoch_relabel, L.w.spin_limit);
    } else {
        RelabelOp<false> op;
        op.st = L.st;
        op.level = L.level;
        op.w = L.w;
        k_scan_lb<RelabelOp<false>><<<grid, SCAN_BLOCK, 0, s>>>(op, L.w.status, L.epoch_relabel, L.w.spin_limit);
    }
    *launches += 1;
    KP_CUDA(cudaGetLastError());
    return KP_OK;
}

namespace {

struct HugeLaunch {
    int cluster = 0;    // CTAs per cluster (16, else 8; 0: no cluster fits)
    int clusters = 0;   // clusters resident at once
};

// The largest cluster the device places for the huge-row kernel, and how
// many of them fit at once.
const HugeLaunch &huge_launch() {
    static const HugeLaunch h = [] {
        HugeLaunch r;
        if (cudaFuncSetAttribute(k_contract_huge, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
            cudaGetLastError();
        for (int c : {16, 8}) {
            cudaLaunchConfig_t cfg = {};
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeClusterDimension;
            attr[0].val.clusterDim.x = c;
            attr[0].val.clusterDim.y = 1;
            attr[0].val.clusterDim.z = 1;
            cfg.gridDim = dim3(c);
            cfg.blockDim = dim3(CONTRACT_BLOCK);
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            int n = 0;
            if (cudaOccupancyMaxActiveClusters(&n, k_contract_huge, &cfg) == cudaSuccess && n > 0) {
                r.cluster = c;
                r.clusters = n;
                return r;
            }
            cudaGetLastError();
        }
        return r;
    }();
    return h;
}

}  // namespace

kp_status launch_contract(const LevelLaunch &L, cudaStream_t s, int32_t *launches) {
    const int64_t want = ((int64_t)std::max<int32_t>(1, L.n_bound) + CONTRACT_BLOCK - 1) / CONTRACT_BLOCK;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)1 << 30));
    // rows of more than HUGE_ROW entries get their own class only when the
    // cluster kernel runs for this level (else they stay with the radix class)
    const HugeLaunch &hl = huge_launch();
    // a level of at most HUGE_ROW entries has no such row; else at most
    // nnz / HUGE_ROW of them, one cluster each
    const int64_t most = L.nnz_bound / HUGE_ROW;
    const bool huge = L.huge && hl.cluster > 0 && most > 0;
    k_contract_small<<<grid, CONTRACT_BLOCK, 0, s>>>(L.st, L.level, L.w, huge ? HUGE_ROW : 0);
    // rows of 17..32 entries: one thread each when there are many of them
    // (decided on the device from the class count), else a warp each
    k_contract_rows32<<<num_sms() * 8, CONTRACT_BLOCK, 0, s>>>(L.st, L.level, L.w);
    k_contract_overflow<<<num_sms() * 8, CONTRACT_BLOCK, 0, s>>>(L.st, L.level, L.w);
    *launches += 3;
    KP_CUDA(cudaGetLastError());
    if (huge) {
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = hl.cluster;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(hl.cluster * (int)std::min<int64_t>(hl.clusters, most));
        cfg.blockDim = dim3(CONTRACT_BLOCK);
        cfg.stream = s;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        KP_CUDA(cudaLaunchKernelEx(&cfg, k_contract_huge, L.st, L.level, L.w));
        *launches += 1;
    }
    return KP_OK;
}

kp_status launch_csr(const LevelLaunch &L, cudaStream_t s, int32_t *launches) {
    const int64_t tiles = scan_tiles(std::max<int64_t>(1, L.n_bound));
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)num_sms() * 4));
    DegScanOp op;
    op.st = L.st;
    op.level = L.level;
    op.w = L.w;
    k_scan_lb<DegScanOp><<<grid, SCAN_BLOCK, 0, s>>>(op, L.w.status, L.epoch_degscan, L.w.spin_limit);
    const int64_t threads = (int64_t)std::max<int32_t>(1, L.n_bound) * 8;
    const int cgrid = (int)std::max<int64_t>(1, std::min<int64_t>((threads + 255) / 256, (int64_t)num_sms() * 16));
    k_compact<<<cgrid, 256, 0, s>>>(L.st, L.level, L.w);
    *launches += 2;
    KP_CUDA(cudaGetLastError());
    return KP_OK;
}

}  // namespace kp
