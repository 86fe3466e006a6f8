// Contraction of one level (Section 2): matched pairs become one node with
// c = c(u)+c(v), parallel edges are merged with summed omega, the contracted
// edge disappears.  Everything is read from the device level table.
//
//   relabel      single-pass scan over (is representative, row bound): coarse
//                ids, map, c', members, row offsets; its last tile carves the
//                coarse level from the arena
//   small rows   one thread per coarse node (<= 16 gathered entries):
//                register bitonic network, run merge
//   overflow     one kernel, classes in turn: rows <= 32 one warp (shuffle
//                bitonic), <= 128 one warp (shared memory), <= MID_MAX one
//                block (shared memory), longer one block (radix through global)
//   degree scan  coarse xadj; its last tile records nnz' and decides the stop
//                rule for the next level
//   compaction   merged rows move to the final CSR
#pragma once

#include "engine.cuh"

namespace kp {

// ---------------------------------------------------------------------------
// relabel
// ---------------------------------------------------------------------------
template <bool SUITOR>
struct RelabelOp {
    DevState *st;
    int level;
    Work w;
    // loaded by prepare()
    int32_t n;
    const eoff *xadj;
    const int32_t *vwgt, *gid;
    int32_t *map, *cvwgt, *gidn;

    __device__ bool prepare() {
        const DevLevel L = st->lv[level];
        if (!(L.flags & LV_ACTIVE)) return false;
        n = L.n;
        xadj = L.xadj;
        vwgt = L.vwgt;
        map = L.map;
        gid = L.gid;
        cvwgt = st->lv[level + 1].vwgt;
        gidn = st->lv[level + 1].gid;
        return true;
    }
    __device__ int64_t count() const { return n; }
    __device__ int32_t *tile_counter() const { return &st->ctr[level].tile_counter[0]; }
    __device__ void fail() const { stop_at(st, level, ERR_TIMEOUT); }
    __device__ int32_t partner(int64_t v) const {
        if (SUITOR) {
            const int32_t s = w.offer[v].s;
            return (s >= 0 && w.offer[s].s == (int32_t)v) ? s : (int32_t)v;
        }
        const int32_t p = w.match[v];
        return p < 0 ? (int32_t)v : p;   // still free after a barrier gave up: single
    }
    __device__ uint64_t load(int64_t v) const {
        if (w.batch && !w.gactive[gid[v]]) {   // its graph has stopped: not carried on
            map[v] = -1;
            return 0;
        }
        const int32_t p = partner(v);
        if (p < v) return 0;   // not the representative of its pair
        // row bounds are below 2^32 in both widths: U <= nnz < 2^32 (the
        // weight range bounds |E| < 2^31), so the low half never carries
        eoff ub = xadj[v + 1] - xadj[v];
        if (p != v) ub += xadj[p + 1] - xadj[p] - 2;   // the pair's own edge is dropped
        return (1ull << 32) | (uint32_t)ub;
    }
    __device__ void store(int64_t v, uint64_t excl, uint64_t val) const {
        if (val == 0) return;
        const int32_t x = (int32_t)(excl >> 32);
        const int32_t p = partner(v);
        map[v] = x;
        w.first[x] = (int32_t)v;
        if (p != v) {
            map[p] = x;
            w.second[x] = p;
            cvwgt[x] = vwgt[v] + vwgt[p];
        } else {
            w.second[x] = -1;
            cvwgt[x] = vwgt[v];
        }
        w.off[x] = (eoff)(excl & 0xffffffffu);
        if (w.batch) gidn[x] = gid[v];
    }
    // One thread: the coarse sizes are known, carve the coarse level.
    __device__ void total(uint64_t t) const {
        const int32_t cn = (int32_t)(t >> 32);
        const eoff U = (eoff)(t & 0xffffffffu);
        Counters *c = &st->ctr[level];
        c->cn = cn;
        c->U = U;
        DevLevel *L = &st->lv[level];
        // one graph: nothing matched, the level is not kept; a batch: every
        // graph has stopped (graphs without a match are found at the next level)
        if (w.batch ? cn == 0 : cn == n) {
            atomicOr(&L->flags, LV_NOMATCH);
            stop_at(st, level, 0);
            return;
        }
        const unsigned long long need_x = sizeof(eoff) * ((unsigned long long)cn + 1);
        const unsigned long long need_e = 4ull * (unsigned long long)(U > 0 ? U : 1);
        char *px = arena_carve(st, need_x);
        char *pa = px ? arena_carve(st, need_e) : nullptr;
        char *pw = pa ? arena_carve(st, need_e) : nullptr;
        char *po = (pw && st->inner_outer) ? arena_carve(st, 4ull * (unsigned long long)cn) : pw;
        if (!po) {
            st->overflow = level + 1;
            stop_at(st, level, 0);
            return;
        }
        DevLevel *C = &st->lv[level + 1];
        C->n = cn;
        C->U = U;
        C->xadj = (eoff *)px;
        C->adjncy = (int32_t *)pa;
        C->ewgt = (int32_t *)pw;
        C->outw = st->inner_outer ? (int32_t *)po : nullptr;
        w.off[cn] = U;
    }
};

// ---------------------------------------------------------------------------
// contraction view of a level, loaded from the table at kernel start
// ---------------------------------------------------------------------------
struct CView {
    int32_t cn;
    const eoff *xadj;
    const int32_t *adjncy, *ewgt, *map;
    const int32_t *first, *second;
    const eoff *off;
    int32_t *tmp_adj, *tmp_w, *big_adj, *big_w, *degp, *outw;
    int32_t *const *lists;
    Counters *ctr;
    int32_t sort_shared_max;   // longest row sorted in shared memory (<= MID_MAX)
    int32_t radix_bits;        // bits per pass of the radix path
};

__device__ __forceinline__ bool load_view(DevState *st, int level, const Work &w, CView &v) {
    const DevLevel L = st->lv[level];
    if (!(L.flags & LV_ACTIVE)) return false;
    v.ctr = &st->ctr[level];
    v.cn = v.ctr->cn;
    v.sort_shared_max = st->sort_shared_max;
    v.radix_bits = st->radix_bits;
    v.xadj = L.xadj;
    v.adjncy = L.adjncy;
    v.ewgt = L.ewgt;
    v.map = L.map;
    v.first = w.first;
    v.second = w.second;
    v.off = w.off;
    v.tmp_adj = w.tmp_adj;
    v.tmp_w = w.tmp_w;
    v.big_adj = w.big_adj;
    v.big_w = w.big_w;
    v.degp = w.degp;
    v.outw = st->lv[level + 1].outw;
    v.lists = w.lists;
    return true;
}

__device__ __forceinline__ void members(const CView &p, int32_t x, eoff &xa, int32_t &da, eoff &xb, int32_t &db) {
    const int32_t a = p.first[x], b = p.second[x];
    xa = p.xadj[a];
    da = (int32_t)(p.xadj[a + 1] - xa);
    xb = b >= 0 ? p.xadj[b] : 0;
    db = b >= 0 ? (int32_t)(p.xadj[b + 1] - xb) : 0;
}

// Rows with at most 16 gathered entries: one thread.  (map(u), omega) packed
// as (key << 32 | omega) in 16 registers, sorted by a bitonic network
// (sentinels last), merged run by run.
constexpr int TNET = 16;

template <int TNET>
__device__ __forceinline__ void contract_thread(const CView &p, int32_t x, eoff xa, int32_t da, eoff xb, int32_t db) {
    constexpr uint64_t SENT64 = (uint64_t)SENT << 32;
    uint64_t r[TNET];
#pragma unroll
    for (int i = 0; i < TNET; i++) {
        uint64_t v = SENT64;
        if (i < da + db) {
            const eoff e = i < da ? xa + i : xb + (i - da);
            const int32_t t = p.map[p.adjncy[e]];
            if (t != x) v = ((uint64_t)(uint32_t)t << 32) | (uint32_t)p.ewgt[e];
        }
        r[i] = v;
    }
#pragma unroll
    for (int k = 2; k <= TNET; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
#pragma unroll
            for (int i = 0; i < TNET; i++) {
                const int l = i ^ j;
                if (l > i) {
                    const uint64_t a = r[i], b = r[l];
                    const bool sw = ((i & k) == 0) ? (a > b) : (a < b);
                    r[i] = sw ? b : a;
                    r[l] = sw ? a : b;
                }
            }
        }
    }
    const eoff o = p.off[x];
    int32_t cnt = 0, curk = -1, sum = 0, total = 0;
#pragma unroll
    for (int i = 0; i < TNET; i++) {
        const int32_t k = (int32_t)(r[i] >> 32);
        const int32_t wv = (int32_t)(uint32_t)r[i];
        if (k != SENT) {
            total += wv;
            if (k == curk) {
                sum += wv;
            } else {
                if (curk >= 0) {
                    p.tmp_adj[o + cnt] = curk;
                    p.tmp_w[o + cnt] = sum;
                    cnt++;
                }
                curk = k;
                sum = wv;
            }
        }
    }
    if (curk >= 0) {
        p.tmp_adj[o + cnt] = curk;
        p.tmp_w[o + cnt] = sum;
        cnt++;
    }
    p.degp[x] = cnt;
    if (p.outw) p.outw[x] = total;
}

// Contracts the rows of at most TNET gathered entries and sorts the others
// into class lists by length; rows of more than huge_row entries (0: none)
// form class 5, which the caller hands to the cluster kernel, rows of 129 to
// warp_row entries (0: none) class 6, for the warp register sort.
static __device__ void phase_contract_small(DevState *st, int level, const Work &w, int32_t huge_row,
                                            int32_t warp_row) {
    CView p;
    if (!load_view(st, level, w, p)) return;
    if (w.batch) {   // first coarse node of every graph (the coarse graph ids are sorted)
        const int32_t *gidn = st->lv[level + 1].gid;
        int32_t *goffn = st->lv[level + 1].goff;
        const int64_t gs = (int64_t)gridDim.x * blockDim.x;
        for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g <= w.num_graphs; g += gs) {
            int32_t lo = 0, hi = p.cn;
            while (lo < hi) {
                const int32_t mid = lo + (hi - lo) / 2;
                if (gidn[mid] < g) lo = mid + 1;
                else hi = mid;
            }
            goffn[g] = lo;
        }
    }
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t x0 = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); x0 < p.cn; x0 += stride) {
        const int64_t x = x0 + lane;
        int cls = -1;
        int32_t da = 0, db = 0;
        eoff xa = 0, xb = 0;
        if (x < p.cn) {
            members(p, (int32_t)x, xa, da, xb, db);
            const int32_t L = da + db;
            cls = L <= TNET ? 0 : L <= 32 ? 1 : L <= 128 ? 2 : L <= p.sort_shared_max ? 3 : 4;
            if (cls == 4 && huge_row > 0 && L > huge_row) cls = 5;
            if (cls == 3 && L <= warp_row) cls = 6;
        }
#pragma unroll
        for (int c = 1; c <= 6; c++) {
            const bool mine = cls == c;
            const unsigned m = __ballot_sync(0xffffffffu, mine);
            if (m) {
                int32_t pos = 0;
                const int first_lane = __ffs(m) - 1;
                if (lane == first_lane) pos = atomicAdd(&p.ctr->nclass[c], __popc(m));
                pos = __shfl_sync(0xffffffffu, pos, first_lane);
                if (mine) p.lists[c][pos + __popc(m & lanemask_lt())] = (int32_t)x;
            }
        }
        if (cls == 0) contract_thread<TNET>(p, (int32_t)x, xa, da, xb, db);
    }
}

// Rows of 17..32 gathered entries: one warp, bitonic sort over the lanes.
__device__ __forceinline__ void contract_warp32(const CView &p, int32_t x) {
    eoff xa, xb;
    int32_t da, db;
    members(p, x, xa, da, xb, db);
    const int gl = threadIdx.x & 31;
    const int32_t L = da + db;
    int32_t key = SENT, val = 0;
    if (gl < L) {
        const eoff e = gl < da ? xa + gl : xb + (gl - da);
        const int32_t t = p.map[p.adjncy[e]];
        if (t != x) {
            key = t;
            val = p.ewgt[e];
        }
    }
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            const int32_t ok = __shfl_xor_sync(0xffffffffu, key, j);
            const int32_t ov = __shfl_xor_sync(0xffffffffu, val, j);
            const bool up = (gl & k) == 0;
            const bool lower = (gl & j) == 0;
            const bool take = lower ? (up ? ok < key : ok > key) : (up ? ok > key : ok < key);
            if (take) {
                key = ok;
                val = ov;
            }
        }
    }
    const int32_t prev = __shfl_up_sync(0xffffffffu, key, 1);
    const int32_t next = __shfl_down_sync(0xffffffffu, key, 1);
    const bool valid = key != SENT;
    const bool head = valid && (gl == 0 || prev != key);
    const bool tail = valid && (gl == 31 || next != key);
    int32_t s = val;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int32_t y = __shfl_up_sync(0xffffffffu, s, d);
        if (gl >= d) s += y;
    }
    const unsigned heads = __ballot_sync(0xffffffffu, head);
    const unsigned tails = __ballot_sync(0xffffffffu, tail);
    const unsigned upto = (gl == 31) ? 0xffffffffu : ((2u << gl) - 1u);
    const unsigned hb = heads & upto;
    const int start = hb ? 31 - __clz(hb) : 0;
    const int32_t before = __shfl_sync(0xffffffffu, s, start > 0 ? start - 1 : 0);
    const int32_t run = s - (start > 0 ? before : 0);
    const int32_t total = __shfl_sync(0xffffffffu, s, 31);
    if (tail) {
        const int32_t idx = __popc(tails & ((1u << gl) - 1u));
        const eoff o = p.off[x];
        p.tmp_adj[o + idx] = key;
        p.tmp_w[o + idx] = run;
    }
    if (gl == 0) {
        p.degp[x] = __popc(tails);
        if (p.outw) p.outw[x] = total;
    }
}

// Rows of 33..128 gathered entries: one warp, bitonic sort of up to 128
// (key, omega) pairs in the warp's shared memory, run indices by a warp scan
// of the head flags, run sums by shared atomics.
constexpr int WSORT = 128;

__device__ __forceinline__ void contract_warp_smem(const CView &p, int32_t x, int32_t *K, int32_t *V, int32_t *S) {
    const int lane = threadIdx.x & 31;
    eoff xa, xb;
    int32_t da, db;
    members(p, x, xa, da, xb, db);
    const int32_t L = da + db;
    const int P = L <= 64 ? 64 : 128;
    for (int i = lane; i < P; i += 32) {
        int32_t key = SENT, val = 0;
        if (i < L) {
            const eoff e = i < da ? xa + i : xb + (i - da);
            const int32_t t = p.map[p.adjncy[e]];
            if (t != x) {
                key = t;
                val = p.ewgt[e];
            }
        }
        K[i] = key;
        V[i] = val;
        S[i] = 0;
    }
    __syncwarp();
    for (int k = 2; k <= P; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int t = lane; t < P / 2; t += 32) {
                const int i = 2 * j * (t / j) + (t % j);
                const int l = i + j;
                const int32_t ki = K[i], kl = K[l];
                const bool up = (i & k) == 0;
                if (up ? ki > kl : ki < kl) {
                    K[i] = kl;
                    K[l] = ki;
                    const int32_t tv = V[i];
                    V[i] = V[l];
                    V[l] = tv;
                }
            }
            __syncwarp();
        }
    }
    const int per = P / 32;
    const int base = lane * per;
    int heads = 0;
    for (int q = 0; q < per; q++) {
        const int i = base + q;
        heads += (K[i] != SENT && (i == 0 || K[i - 1] != K[i])) ? 1 : 0;
    }
    int incl = heads;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += y;
    }
    const int nruns = __shfl_sync(0xffffffffu, incl, 31);
    int r = incl - heads - 1;
    const eoff o = p.off[x];
    int32_t wsum = 0;
    for (int q = 0; q < per; q++) {
        const int i = base + q;
        const int32_t k = K[i];
        if (k == SENT) break;
        if (i == 0 || K[i - 1] != k) {
            r++;
            p.tmp_adj[o + r] = k;
        }
        atomicAdd(&S[r], V[i]);
        wsum += V[i];
    }
    __syncwarp();
    for (int i = lane; i < nruns; i += 32) p.tmp_w[o + i] = S[i];
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) wsum += __shfl_xor_sync(0xffffffffu, wsum, d);
    if (lane == 0) {
        p.degp[x] = nruns;
        if (p.outw) p.outw[x] = wsum;
    }
    __syncwarp();
}

// Rows of 129..MID_MAX gathered entries: one block, bitonic sort in shared
// memory, then run heads, run sums and the merged row.
static __device__ void contract_block_smem(const CView &p, int32_t x, int32_t *keys, int32_t *vals, int32_t *sums,
                                    int32_t *s_red) {
    constexpr int IPT = MID_MAX / CONTRACT_BLOCK;
    eoff xa, xb;
    int32_t da, db;
    members(p, x, xa, da, xb, db);
    const int32_t L = da + db;
    int32_t P = 64;
    while (P < L) P <<= 1;
    for (int32_t i = threadIdx.x; i < P; i += blockDim.x) {
        int32_t key = SENT, val = 0;
        if (i < L) {
            const eoff e = i < da ? xa + i : xb + (i - da);
            const int32_t t = p.map[p.adjncy[e]];
            if (t != x) {
                key = t;
                val = p.ewgt[e];
            }
        }
        keys[i] = key;
        vals[i] = val;
        sums[i] = 0;
    }
    __syncthreads();
    for (int32_t k = 2; k <= P; k <<= 1) {
        for (int32_t j = k >> 1; j > 0; j >>= 1) {
            for (int32_t i = threadIdx.x; i < P; i += blockDim.x) {
                const int32_t ixj = i ^ j;
                if (ixj > i) {
                    const bool up = (i & k) == 0;
                    const int32_t ki = keys[i], kj = keys[ixj];
                    if (up ? ki > kj : ki < kj) {
                        keys[i] = kj;
                        keys[ixj] = ki;
                        const int32_t t = vals[i];
                        vals[i] = vals[ixj];
                        vals[ixj] = t;
                    }
                }
            }
            __syncthreads();
        }
    }
    const int32_t base = threadIdx.x * IPT;
    int32_t h[IPT];
    int32_t cnt = 0;
#pragma unroll
    for (int j = 0; j < IPT; j++) {
        const int32_t i = base + j;
        h[j] = (i < P && keys[i] != SENT && (i == 0 || keys[i - 1] != keys[i])) ? 1 : 0;
        cnt += h[j];
    }
    uint64_t tot;
    int32_t r = (int32_t)block_exclusive_scan<CONTRACT_BLOCK>((uint64_t)cnt, &tot) - 1;
    const eoff o = p.off[x];
    int32_t wsum = 0;
#pragma unroll
    for (int j = 0; j < IPT; j++) {
        const int32_t i = base + j;
        r += h[j];
        if (i < P && keys[i] != SENT) {
            atomicAdd(&sums[r], vals[i]);
            wsum += vals[i];
            if (h[j]) p.tmp_adj[o + r] = keys[i];
        }
    }
    __syncthreads();
    for (int32_t i = threadIdx.x; i < (int32_t)tot; i += blockDim.x) p.tmp_w[o + i] = sums[i];
    for (int off2 = 16; off2 > 0; off2 >>= 1) wsum += __shfl_xor_sync(0xffffffffu, wsum, off2);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = wsum;
    __syncthreads();
    if (threadIdx.x == 0) {
        int32_t t = 0;
        for (int wi = 0; wi < CONTRACT_BLOCK / 32; wi++) t += s_red[wi];
        p.degp[x] = (int32_t)tot;
        if (tot >= 1024) atomicMax(&p.ctr->maxdeg, (int32_t)tot);
        if (p.outw) p.outw[x] = t;
    }
    __syncthreads();
}

// Rows longer than the shared-memory limit: one block, RADIX_ITEMS entries
// per thread and chunk.
// 1. gather (map(u), omega) without the contracted edge into the slot at
//    off[x] (tmp or big, chosen so that the last pass ends in big), counting
//    the digits of every radix pass on the way
// 2. stable LSD radix sort by coarse neighbour, radix_bits (4..8) bits per pass, ping-pong
//    between tmp and big; a chunk is ranked warp by warp (match masks, item
//    by item in index order) and the warps' digit counts are scanned
// 3. merge equal neighbours from big into tmp (run heads by ballots, run
//    sums by atomics)

struct BigSmem {
    int32_t hist[8][256];
    int32_t base[256];
    int32_t chunk_tot[256];
    int32_t wcnt[CONTRACT_BLOCK / 32][256];
    int32_t wsum[CONTRACT_BLOCK / 32];
    int32_t s_red[CONTRACT_BLOCK / 32];
    int32_t s_carry;
};

template <int RADIX_ITEMS>
static __device__ void contract_block_radix(const CView &p, int32_t x, int passes, BigSmem &sm) {
    constexpr int RADIX_CHUNK = CONTRACT_BLOCK * RADIX_ITEMS;
    static_assert(CONTRACT_BLOCK == 256, "one thread per digit");
    constexpr int NW = CONTRACT_BLOCK / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
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
    for (int i = threadIdx.x; i < 8 * 256; i += CONTRACT_BLOCK) (&sm.hist[0][0])[i] = 0;
    if (threadIdx.x == 0) sm.s_carry = 0;
    __syncthreads();
    // 1. gather (the order of the kept entries does not matter: they are
    //    sorted next and equal keys are summed)
    for (int32_t c0 = 0; c0 < L; c0 += RADIX_CHUNK) {
#pragma unroll
        for (int j = 0; j < RADIX_ITEMS; j++) {
            const int32_t i = c0 + (warp * RADIX_ITEMS + j) * 32 + lane;
            int32_t t = x, wv = 0;
            if (i < L) {
                const eoff e = i < da ? xa + i : xb + (i - da);
                t = p.map[p.adjncy[e]];
                wv = p.ewgt[e];
            }
            const bool keep = i < L && t != x;
            const unsigned m = __ballot_sync(0xffffffffu, keep);
            int32_t at = 0;
            if (lane == 0 && m) at = atomicAdd(&sm.s_carry, __popc(m));
            at = __shfl_sync(0xffffffffu, at, 0);
            if (keep) {
                const int32_t r = at + __popc(m & lt);
                src_k[r] = t;
                src_v[r] = wv;
                for (int ps = 0; ps < passes; ps++) atomicAdd(&sm.hist[ps][(t >> (rb * ps)) & dmask], 1);
            }
        }
    }
    __syncthreads();
    const int32_t M = sm.s_carry;   // == off[x+1] - off[x]
    // 2. radix passes
    for (int pass = 0; pass < passes; pass++) {
        const int shift = rb * pass;
        {
            uint64_t tot;
            sm.base[threadIdx.x] =
                (int32_t)block_exclusive_scan<CONTRACT_BLOCK>((uint64_t)sm.hist[pass][threadIdx.x], &tot);
        }
        for (int32_t c0 = 0; c0 < M; c0 += RADIX_CHUNK) {
#pragma unroll
            for (int j = 0; j < 256 / 32; j++) sm.wcnt[warp][j * 32 + lane] = 0;
            __syncwarp();
            int32_t kk[RADIX_ITEMS], vv[RADIX_ITEMS], rk[RADIX_ITEMS];
#pragma unroll
            for (int j = 0; j < RADIX_ITEMS; j++) {
                const int32_t i = c0 + (warp * RADIX_ITEMS + j) * 32 + lane;
                const bool valid = i < M;
                kk[j] = valid ? src_k[i] : 0;
                vv[j] = valid ? src_v[i] : 0;
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
            for (int j = 0; j < RADIX_ITEMS; j++) {
                const int32_t i = c0 + (warp * RADIX_ITEMS + j) * 32 + lane;
                if (i < M) {
                    const int d = (kk[j] >> shift) & dmask;
                    const int32_t r = sm.base[d] + sm.wcnt[warp][d] + rk[j];
                    dst_k[r] = kk[j];
                    dst_v[r] = vv[j];
                }
            }
            __syncthreads();
            sm.base[threadIdx.x] += sm.chunk_tot[threadIdx.x];
        }
        __syncthreads();
        int32_t *tk = src_k, *tv = src_v;
        src_k = dst_k;
        src_v = dst_v;
        dst_k = tk;
        dst_v = tv;
    }
    // src == big now; 3. merge into tmp
    for (int32_t i = threadIdx.x; i < M; i += CONTRACT_BLOCK) p.tmp_w[o + i] = 0;
    if (threadIdx.x == 0) sm.s_carry = 0;
    __syncthreads();
    int32_t wsum = 0;
    for (int32_t c0 = 0; c0 < M; c0 += RADIX_CHUNK) {
        int32_t hk[RADIX_ITEMS];
        unsigned hm[RADIX_ITEMS];
        int32_t wrun = 0;
#pragma unroll
        for (int j = 0; j < RADIX_ITEMS; j++) {
            const int32_t i = c0 + (warp * RADIX_ITEMS + j) * 32 + lane;
            const bool valid = i < M;
            hk[j] = valid ? src_k[i] : SENT;
            const bool head = valid && (i == 0 || src_k[i - 1] != hk[j]);
            hm[j] = __ballot_sync(0xffffffffu, head);
            wrun += __popc(hm[j]);
        }
        if (lane == 0) sm.wsum[warp] = wrun;
        __syncthreads();
        int32_t before = sm.s_carry;
        for (int w2 = 0; w2 < warp; w2++) before += sm.wsum[w2];
#pragma unroll
        for (int j = 0; j < RADIX_ITEMS; j++) {
            const int32_t i = c0 + (warp * RADIX_ITEMS + j) * 32 + lane;
            // run index: heads up to and including this entry, minus one
            const int32_t r = before + __popc(hm[j] & (lt | (1u << lane))) - 1;
            before += __popc(hm[j]);
            if (i < M) {
                const int32_t v = src_v[i];
                if ((hm[j] >> lane) & 1u) p.tmp_adj[o + r] = hk[j];
                atomicAdd(&p.tmp_w[o + r], v);
                wsum += v;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int32_t t = sm.s_carry;
            for (int w2 = 0; w2 < NW; w2++) t += sm.wsum[w2];
            sm.s_carry = t;
        }
        __syncthreads();
    }
    for (int off2 = 16; off2 > 0; off2 >>= 1) wsum += __shfl_xor_sync(0xffffffffu, wsum, off2);
    if (lane == 0) sm.s_red[warp] = wsum;
    __syncthreads();
    if (threadIdx.x == 0) {
        int32_t t = 0;
        for (int w2 = 0; w2 < NW; w2++) t += sm.s_red[w2];
        p.degp[x] = sm.s_carry;
        if (sm.s_carry >= 1024) atomicMax(&p.ctr->maxdeg, sm.s_carry);
        if (p.outw) p.outw[x] = t;
    }
    __syncthreads();
}

// All overflow classes in one launch: blocks take roles by index.
union OverflowSmem {
    struct {
        int32_t K[CONTRACT_BLOCK / 32][WSORT];
        int32_t V[CONTRACT_BLOCK / 32][WSORT];
        int32_t S[CONTRACT_BLOCK / 32][WSORT];
    } warp;
    struct {
        int32_t keys[MID_MAX];
        int32_t vals[MID_MAX];
        int32_t sums[MID_MAX];
        int32_t s_red[CONTRACT_BLOCK / 32];
    } mid;
    BigSmem big;
};

// Rows of 129..WARP_ROW gathered entries (class 6, levels launched one
// kernel per phase): one warp, WARP_ROW / 32 entries per lane packed as
// (map(u) << 32 | omega) in registers, sorted by a bitonic network over the
// warp (element q = lane * N + i; partners in other lanes by shuffles, no
// block barrier), then run heads by a warp scan and run sums written by the
// run's first lane (lanes that continue a run add theirs after a warp
// barrier).
constexpr int32_t WARP_ROW = 512;

__device__ __forceinline__ uint64_t shfl_xor_u64(uint64_t v, int m) {
    const uint32_t lo = __shfl_xor_sync(0xffffffffu, (uint32_t)v, m);
    const uint32_t hi = __shfl_xor_sync(0xffffffffu, (uint32_t)(v >> 32), m);
    return ((uint64_t)hi << 32) | lo;
}

__device__ __forceinline__ void contract_warp_reg(const CView &p, int32_t x) {
    constexpr int N = WARP_ROW / 32;
    constexpr uint64_t SENT64 = (uint64_t)SENT << 32;
    const int lane = threadIdx.x & 31;
    eoff xa, xb;
    int32_t da, db;
    members(p, x, xa, da, xb, db);
    const int32_t L = da + db;
    uint64_t r[N];
    // any placement works before a sort: element i of a lane is entry
    // i * 32 + lane, so the loads are coalesced
#pragma unroll
    for (int i = 0; i < N; i++) {
        const int32_t q = i * 32 + lane;
        uint64_t v = SENT64;
        if (q < L) {
            const eoff e = q < da ? xa + q : xb + (q - da);
            const int32_t t = p.map[p.adjncy[e]];
            if (t != x) v = ((uint64_t)(uint32_t)t << 32) | (uint32_t)p.ewgt[e];
        }
        r[i] = v;
    }
#pragma unroll
    for (int k = 2; k <= WARP_ROW; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j >= N) {
                // partner: the same i in lane ^ (j / N)
                const bool lower = (lane & (j / N)) == 0;
                const bool up = ((lane * N) & k) == 0;
#pragma unroll
                for (int i = 0; i < N; i++) {
                    const uint64_t o = shfl_xor_u64(r[i], j / N);
                    const uint64_t mn = r[i] < o ? r[i] : o, mx = r[i] < o ? o : r[i];
                    r[i] = (lower == up) ? mn : mx;
                }
            } else {
#pragma unroll
                for (int i = 0; i < N; i++) {
                    const int l = i ^ j;
                    if (l > i) {
                        const bool up = ((lane * N + i) & k) == 0;
                        const uint64_t a = r[i], b = r[l];
                        const bool sw = up ? (a > b) : (a < b);
                        r[i] = sw ? b : a;
                        r[l] = sw ? a : b;
                    }
                }
            }
        }
    }
    // runs: element q = lane * N + i in ascending order, sentinels last
    const int32_t prev_last = (int32_t)(__shfl_up_sync(0xffffffffu, r[N - 1], 1) >> 32);
    int32_t heads = 0, total = 0;
#pragma unroll
    for (int i = 0; i < N; i++) {
        const int32_t k = (int32_t)(r[i] >> 32);
        const int32_t pk = i > 0 ? (int32_t)(r[i - 1] >> 32) : (lane > 0 ? prev_last : -1);
        heads += (k != SENT && k != pk) ? 1 : 0;
        total += k != SENT ? (int32_t)(uint32_t)r[i] : 0;
    }
    int32_t incl = heads;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int32_t y = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += y;
    }
    const int32_t runs = __shfl_sync(0xffffffffu, incl, 31);
    const eoff o = p.off[x];
    int32_t run = incl - heads - 1;   // the run in progress where this lane starts
    int32_t sum = 0;
    bool mine = false;                // that run started in this lane
    int32_t lead_run = -1, lead_sum = 0;
#pragma unroll
    for (int i = 0; i < N; i++) {
        const int32_t k = (int32_t)(r[i] >> 32);
        if (k == SENT) continue;
        const int32_t pk = i > 0 ? (int32_t)(r[i - 1] >> 32) : (lane > 0 ? prev_last : -1);
        const int32_t wv = (int32_t)(uint32_t)r[i];
        if (k != pk) {
            if (mine) {
                p.tmp_w[o + run] = sum;
            } else if (i > 0 || sum != 0) {
                lead_run = run;
                lead_sum = sum;
            }
            run++;
            mine = true;
            sum = wv;
            p.tmp_adj[o + run] = k;
        } else {
            sum += wv;
        }
    }
    if (mine) {
        p.tmp_w[o + run] = sum;
    } else if (run >= 0 && sum != 0) {
        lead_run = run;
        lead_sum = sum;
    }
    __syncwarp();   // the first lane of every run has stored its part
    if (lead_run >= 0) atomicAdd(&p.tmp_w[o + lead_run], lead_sum);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) total += __shfl_xor_sync(0xffffffffu, total, off);
    if (lane == 0) {
        p.degp[x] = runs;
        if (p.outw) p.outw[x] = total;
    }
}

// Rows of 17..32 gathered entries (class 1), one thread each with a
// 32-entry register network: for the separate launches (a warp per such row
// leaves half the warp idle; the register network needs its own kernel so
// that the other classes keep their occupancy).  It takes the class when it
// has at least ROWS32_MIN rows; fewer go to the overflow kernel's warps.
constexpr int32_t ROWS32_MIN = 2048;

static __device__ void phase_contract_rows32(DevState *st, int level, const Work &w) {
    CView p;
    if (!load_view(st, level, w, p)) return;
    const int32_t count = p.ctr->nclass[1];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    if (count >= ROWS32_MIN) {
        for (int64_t li = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; li < count; li += stride) {
            const int32_t x = p.lists[1][li];
            eoff xa, xb;
            int32_t da, db;
            members(p, x, xa, da, xb, db);
            contract_thread<32>(p, x, xa, da, xb, db);
        }
    }
    // class 6: a warp per row (the loop bound is the same for a warp's lanes)
    const int32_t count6 = p.ctr->nclass[6];
    for (int64_t li = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; li < count6; li += stride >> 5)
        contract_warp_reg(p, p.lists[6][li]);
}

// The next row of a block-per-row class, taken from a counter by the whole
// block: the rows of power-law graphs differ in length by orders of
// magnitude, so a fixed round-robin share would leave some blocks with
// several long rows while the others wait.
__device__ __forceinline__ int32_t next_row(int32_t *counter) {
    __shared__ int32_t s_row;
    __syncthreads();   // the previous row is finished and s_row read by every thread
    if (threadIdx.x == 0) s_row = atomicAdd(counter, 1);
    __syncthreads();
    return s_row;
}

// MID: the classes of up to sort_shared_max entries (warps, blocks in shared
// memory; class 1 with WARP32 always, without it only when the rows32
// kernel leaves it); BIG: the radix class, RADIX_ITEMS entries per thread
// and chunk.
template <bool MID, bool BIG, int RADIX_ITEMS, bool WARP32 = true>
static __device__ void phase_contract_overflow(DevState *st, int level, const Work &w, OverflowSmem &sm) {
    CView p;
    if (!load_view(st, level, w, p)) return;
    // every block takes part in every class in turn, so no class can be left
    // without blocks however small the grid is
    const int warp = threadIdx.x >> 5;
    constexpr int NW = CONTRACT_BLOCK / 32;
    const int64_t gw = (int64_t)blockIdx.x * NW + warp, nw = (int64_t)gridDim.x * NW;
    if (MID) {
        {
            const int32_t count = p.ctr->nclass[1];
            if (WARP32 || count < ROWS32_MIN)
                for (int64_t li = gw; li < count; li += nw) contract_warp32(p, p.lists[1][li]);
        }
        {
            const int32_t count = p.ctr->nclass[2];
            for (int64_t li = gw; li < count; li += nw)
                contract_warp_smem(p, p.lists[2][li], sm.warp.K[warp], sm.warp.V[warp], sm.warp.S[warp]);
        }
        __syncthreads();
        {
            const int32_t count = p.ctr->nclass[3];
            for (int32_t li = next_row(&p.ctr->class_next[0]); li < count; li = next_row(&p.ctr->class_next[0]))
                contract_block_smem(p, p.lists[3][li], sm.mid.keys, sm.mid.vals, sm.mid.sums, sm.mid.s_red);
        }
        __syncthreads();
    }
    if (BIG) {
        const int32_t count = p.ctr->nclass[4];
        if (count > 0) {
            int bits = 1;
            while (bits < 31 && ((int64_t)1 << bits) < (int64_t)p.cn) bits++;
            const int passes = (bits + p.radix_bits - 1) / p.radix_bits;
            for (int32_t li = next_row(&p.ctr->class_next[1]); li < count; li = next_row(&p.ctr->class_next[1]))
                contract_block_radix<RADIX_ITEMS>(p, p.lists[4][li], passes, sm.big);
        }
    }
}

// ---------------------------------------------------------------------------
// coarse xadj and the stop rule
// ---------------------------------------------------------------------------
struct DegScanOp {
    DevState *st;
    int level;
    Work w;
    int32_t cn;
    eoff *cxadj;

    __device__ bool prepare() {
        if (!(st->lv[level].flags & LV_ACTIVE)) return false;
        cn = st->ctr[level].cn;
        cxadj = st->lv[level + 1].xadj;
        return true;
    }
    __device__ int64_t count() const { return cn; }
    __device__ int32_t *tile_counter() const { return &st->ctr[level].tile_counter[1]; }
    __device__ void fail() const { stop_at(st, level, ERR_TIMEOUT); }
    __device__ uint64_t load(int64_t x) const { return (uint64_t)(uint32_t)w.degp[x]; }
    __device__ void store(int64_t x, uint64_t excl, uint64_t) const { cxadj[x] = (eoff)excl; }
    // One thread: record nnz' and decide whether level+1 is contracted
    // (stop when small enough, after too little shrinkage, or at the level cap).
    __device__ void total(uint64_t t) const {
        cxadj[cn] = (eoff)t;
        st->ctr[level].nnz_out = (eoff)t;
        DevLevel *C = &st->lv[level + 1];
        C->nnz = (eoff)t;
        const int64_t n = st->lv[level].n;
        bool next;
        if (w.batch) {   // graphs decide for themselves at the next level start
            next = cn > 0 && level + 1 <= st->max_levels && !(st->stop || st->err);
        } else {
            const bool small = cn <= st->stop_size;
            const bool capped = level + 1 >= st->max_levels;
            const bool stalled = (int64_t)cn * 1000 > n * (1000 - st->min_shrink_permille);
            next = !(small || capped || stalled || st->stop || st->err);
        }
        C->flags = LV_BUILT | (next ? LV_ACTIVE : 0);
        if (!next) st->stop = 1;
        volatile LevelSnap *s = st->snap + level;
        s->cn = cn;
        s->nnz = (eoff)t;
        s->maxdeg = st->ctr[level].maxdeg;   // the contraction kernels ended before this scan
        s->room = st->arena_cap - st->arena_used;
        s->arena_gen = st->arena_gen;
        s->stop = next ? 0 : 1;
        s->done = 1;
    }
};

// Moves every merged coarse row from its upper-bound slot to the CSR: rows
// of at most 128 gathered entries with 8 lanes each, the longer ones (the
// class lists of the contraction) with a warp each (up to MID_MAX) or a
// block each, so a hub's row is not left to 8 lanes.
static __device__ void phase_compact(DevState *st, int level, const Work &w) {
    if (!(st->lv[level].flags & LV_ACTIVE)) return;
    const Counters *ctr = &st->ctr[level];
    const int32_t cn = ctr->cn;
    const eoff *KP_RESTRICT cxadj = st->lv[level + 1].xadj;
    int32_t *KP_RESTRICT cadj = st->lv[level + 1].adjncy;
    int32_t *KP_RESTRICT cw = st->lv[level + 1].ewgt;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int gl = threadIdx.x & 7;
    for (int64_t g = t >> 3; g < cn; g += stride >> 3) {
        const eoff o = w.off[g];
        // gathered entries = the slot plus the pair's own two, as classified
        if (w.off[g + 1] - o + (w.second[g] >= 0 ? 2 : 0) > 128) continue;
        const int32_t d = w.degp[g];
        const eoff s = cxadj[g];
        for (int32_t i = gl; i < d; i += 8) {
            cadj[s + i] = w.tmp_adj[o + i];
            cw[s + i] = w.tmp_w[o + i];
        }
    }
    const int lane = threadIdx.x & 31;
    const int64_t nw = stride >> 5;
    const int32_t n3 = ctr->nclass[3], n4 = ctr->nclass[4], n6 = ctr->nclass[6];
    for (int64_t li = t >> 5; li < (int64_t)n3 + n6; li += nw) {
        const int32_t g = li < n3 ? w.lists[3][li] : w.lists[6][li - n3];
        const eoff o = w.off[g], s = cxadj[g];
        const int32_t d = w.degp[g];
        for (int32_t i = lane; i < d; i += 32) {
            cadj[s + i] = w.tmp_adj[o + i];
            cw[s + i] = w.tmp_w[o + i];
        }
    }
    for (int64_t li = blockIdx.x; li < n4; li += gridDim.x) {
        const int32_t g = w.lists[4][li];
        const eoff o = w.off[g], s = cxadj[g];
        const int32_t d = w.degp[g];
        for (int32_t i = threadIdx.x; i < d; i += blockDim.x) {
            cadj[s + i] = w.tmp_adj[o + i];
            cw[s + i] = w.tmp_w[o + i];
        }
    }
    // the few huge rows: each one over the whole grid
    const int32_t n5 = ctr->nclass[5];
    for (int32_t li = 0; li < n5; li++) {
        const int32_t g = w.lists[5][li];
        const eoff o = w.off[g], s = cxadj[g];
        const int32_t d = w.degp[g];
        for (int64_t i = t; i < d; i += stride) {
            cadj[s + i] = w.tmp_adj[o + i];
            cw[s + i] = w.tmp_w[o + i];
        }
    }
}

}  // namespace kp
