// Matching of locally heaviest edges (Section 3.3) on one level, read from
// the device level table.  Two schemes reach the same unique matching (the
// Greedy matching of Section 3.2 under the strict edge order):
//   proposals (Suitor scheme, Manne & Halappanavar 2014): every node proposes
//     to its best neighbour whose standing offer it beats, displaced
//     proposers propose again; one 128-bit CAS per proposal, no rounds;
//   handshake rounds: every free node names its best free neighbour, mutual
//     names are matched, repeated until no edge has two free ends; one
//     cooperative launch, rounds separated by bounded grid barriers.
#pragma once

#include "engine.cuh"

namespace kp {

// ---------------------------------------------------------------------------
// level begin: carve map_l and c of level l+1, reset the per-node state
// ---------------------------------------------------------------------------
template <int R, bool SUITOR>
__device__ void phase_level_begin(DevState *st, int level, const Work &w) {
    const DevLevel L = st->lv[level];
    if (!(L.flags & LV_ACTIVE)) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        int32_t *map = (int32_t *)arena_carve(st, 4ull * (unsigned long long)L.n);
        int32_t *cv = map ? (int32_t *)arena_carve(st, 4ull * (unsigned long long)L.n) : nullptr;
        int32_t *gidn = cv, *goffn = cv;
        if (cv && w.batch) {
            gidn = (int32_t *)arena_carve(st, 4ull * (unsigned long long)L.n);
            goffn = gidn ? (int32_t *)arena_carve(st, 4ull * ((unsigned long long)w.num_graphs + 1)) : nullptr;
        }
        if (!map || !cv || !gidn || !goffn) {
            st->overflow = level + 1;
            stop_at(st, level, 0);
        } else {
            st->lv[level].map = map;
            st->lv[level + 1].vwgt = cv;
            if (w.batch) {
                st->lv[level + 1].gid = gidn;
                st->lv[level + 1].goff = goffn;
            }
        }
    }
    if (w.batch) {
        // per graph: is it contracted at this level?  (the stop rule of a
        // single graph, applied to each graph of the batch)
        const int32_t *prev = level > 0 ? st->lv[level - 1].goff : nullptr;
        const int64_t gstride = (int64_t)gridDim.x * blockDim.x;
        for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < w.num_graphs; g += gstride) {
            const int64_t nc = L.goff[g + 1] - L.goff[g];
            const int64_t np = prev ? (int64_t)(prev[g + 1] - prev[g]) : -1;
            int32_t act = 0;
            if (nc == 0) {
                act = 0;   // left the batch at an earlier level
            } else if (level > 0 && nc == np) {
                w.glevels[g] = level;   // nothing matched: that copy is not a level
            } else if (nc <= (w.stops ? (int64_t)w.stops[g] : (int64_t)st->stop_size) || level >= st->max_levels ||
                       (level > 0 && nc * 1000 > np * (1000 - st->min_shrink_permille))) {
                w.glevels[g] = level + 1;
            } else {
                act = 1;
            }
            w.gactive[g] = act;
        }
    }
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < L.n; v += stride) {
        if (SUITOR) {
            Offer o;
            o.s = -1;
            o.w = 0;
            o.as = 0;
            o.au = rating_attr<R>(L.vwgt, L.outw, (int32_t)v);
            w.offer[v] = o;
        } else {
            w.match[v] = -1;
        }
    }
}

// ---------------------------------------------------------------------------
// proposals
// ---------------------------------------------------------------------------
__device__ __forceinline__ Offer ld_offer(const Offer *p) {
    Offer o;
    asm volatile("ld.global.cg.v4.s32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(o.s), "=r"(o.w), "=r"(o.as), "=r"(o.au)
                 : "l"(p)
                 : "memory");
    return o;
}

__device__ __forceinline__ bool cas_offer(Offer *addr, const Offer &expect, const Offer &desired) {
    const uint64_t elo = ((uint64_t)(uint32_t)expect.w << 32) | (uint32_t)expect.s;
    const uint64_t ehi = ((uint64_t)(uint32_t)expect.au << 32) | (uint32_t)expect.as;
    const uint64_t dlo = ((uint64_t)(uint32_t)desired.w << 32) | (uint32_t)desired.s;
    const uint64_t dhi = ((uint64_t)(uint32_t)desired.au << 32) | (uint32_t)desired.as;
    uint64_t olo, ohi;
    asm volatile(
        "{\n\t.reg .b128 e, d, o;\n\t"
        "mov.b128 e, {%2, %3};\n\t"
        "mov.b128 d, {%4, %5};\n\t"
        "atom.global.cas.b128 o, [%6], e, d;\n\t"
        "mov.b128 {%0, %1}, o;\n\t}"
        : "=l"(olo), "=l"(ohi)
        : "l"(elo), "l"(ehi), "l"(dlo), "l"(dhi), "l"(addr)
        : "memory");
    return olo == elo && ohi == ehi;
}

// Lanes per proposing node from the level's mean degree, and the row length
// above which a node is left to the later passes.
__device__ __forceinline__ int suitor_group(int32_t n, int32_t nnz) {
    const int64_t a = n > 0 ? (int64_t)nnz : 0;
    if (a <= 12ll * n) return 1;
    if (a <= 40ll * n) return 4;
    if (a <= 160ll * n) return 8;
    return 32;
}

// Rows up to this length that the first pass parks are searched by one warp
// each (the middle pass); longer rows by one block each (the wide pass).
constexpr int32_t SUITOR_WARP_ROW = 1024;

// A node's best proposal so far: the edge, its weight, and the record of the
// other end as it was read (the compare-and-swap expects that record).
struct Proposal {
    Cand c;
    int32_t w;
    Offer snap;
};

// One thread's share of a search: the entries e0, e0 + STRIDE, ... < end of
// cur's row.  An edge {cur,v} is eligible when v holds no offer or when cur's
// offer beats v's standing one at v; the best eligible edge is kept.
template <int R, int STRIDE>
__device__ __forceinline__ void scan_row(const DevLevel &L, const Work &w, const HashCtx &hc, int32_t cur,
                                         int32_t acur, int32_t e0, int32_t end, Proposal &best) {
    const int32_t *KP_RESTRICT adjncy = L.adjncy;
    const int32_t *KP_RESTRICT ewgt = L.ewgt;
    best.c.u = -1;
    best.c.num = best.c.den = best.c.h = 0;
    best.w = 0;
    best.snap = {-1, 0, 0, 0};
#pragma unroll 4
    for (int32_t e = e0; e < end; e += STRIDE) {
        const int32_t v = KP_LDG(adjncy + e);
        const int32_t wt = KP_LDG(ewgt + e);
        const Offer st = ld_offer(w.offer + v);
        Cand c;
        c.u = v;
        rating_ab<R>(wt, acur, st.au, c.num, c.den);
        c.h = edge_hash_in(hc, cur, v);
        bool eligible = st.s < 0;
        if (!eligible) {
            // compare at v: the offer of cur against the standing offer of st.s
            Cand a, b;
            a.u = cur;
            a.num = c.num;
            a.den = c.den;
            a.h = c.h;
            b.u = st.s;
            rating_ab<R>(st.w, st.as, st.au, b.num, b.den);
            b.h = edge_hash_in(hc, st.s, v);
            eligible = better(a, b, v);
        }
        if (eligible && better(c, best.c, cur)) {
            best.c = c;
            best.w = wt;
            best.snap = st;
        }
    }
}

// The best proposal over the G lanes of a group (all of them end with it).
template <int G>
__device__ __forceinline__ void reduce_proposal(unsigned gmask, int32_t cur, Proposal &best) {
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1) {
        Proposal o;
        o.c.num = __shfl_xor_sync(gmask, best.c.num, off);
        o.c.den = __shfl_xor_sync(gmask, best.c.den, off);
        o.c.h = __shfl_xor_sync(gmask, best.c.h, off);
        o.c.u = __shfl_xor_sync(gmask, best.c.u, off);
        o.w = __shfl_xor_sync(gmask, best.w, off);
        o.snap.s = __shfl_xor_sync(gmask, best.snap.s, off);
        o.snap.w = __shfl_xor_sync(gmask, best.snap.w, off);
        o.snap.as = __shfl_xor_sync(gmask, best.snap.as, off);
        o.snap.au = __shfl_xor_sync(gmask, best.snap.au, off);
        if (better(o.c, best.c, cur)) best = o;
    }
}

// Makes cur's proposal and returns the node that searches next: the suitor
// it displaced (-1 if none, or if cur found nothing to propose to), or cur
// itself when the record changed under it.
__device__ __forceinline__ int32_t propose(const Work &w, int32_t cur, int32_t acur, const Proposal &b,
                                           unsigned long long &fails) {
    if (b.c.u < 0) return -1;
    Offer mine;
    mine.s = cur;
    mine.w = b.w;
    mine.as = acur;
    mine.au = b.snap.au;
    if (cas_offer(w.offer + b.c.u, b.snap, mine)) return b.snap.s;
    fails++;
    return cur;
}

// Parks node v for a later pass: rows up to SUITOR_WARP_ROW for the middle
// pass (list0) unless the calling pass already searches rows that long,
// longer rows for the wide pass (list1).
template <int HEAVY>
__device__ __forceinline__ void park(const Work &w, Counters *ctr, int32_t v, int32_t len) {
    if (HEAVY < SUITOR_WARP_ROW && len <= SUITOR_WARP_ROW)
        w.list0[atomicAdd(&ctr->list_size[0], 1)] = v;
    else
        w.list1[atomicAdd(&ctr->list_size[2], 1)] = v;
}

// First pass: G lanes per proposing node, start nodes [0, n).  Every warp
// owns one contiguous range of start nodes; its 32/G groups each follow one
// proposal chain (a node, then whoever it displaced) and take the next start
// node of the range as soon as their chain ends, so lanes stay busy until the
// range is used up.  A node whose row is longer than HEAVY entries is parked
// instead of being scanned by so few lanes.  The order of proposals does not
// change the matching.
template <int R, int G, int HEAVY>
__device__ __forceinline__ void suitor_body(const DevLevel &L, const Work &w, Counters *ctr, int32_t *err) {
    constexpr int NG = 32 / G;
    const unsigned gmask = group_mask<G>();
    const int lane = threadIdx.x & 31;
    const int gl = lane & (G - 1);
    const int leader = lane & ~(G - 1);
    const unsigned below_leader = (1u << leader) - 1u;
    const int32_t *KP_RESTRICT xadj = L.xadj;
    const int64_t count = L.n;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t warp_id = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t chunk = (count + nwarps - 1) / nwarps;
    int64_t pos = warp_id * chunk;
    const int64_t stop = min(count, pos + chunk);
    long long iters = 0;
    unsigned long long fails = 0;
    int32_t cur = -1;
    bool aborted = false;
    for (;;) {
        // the whole warp leaves together (full-warp votes follow)
        if (__any_sync(0xffffffffu, aborted)) break;
        // give every idle group the next start node of the warp's range
        const unsigned need = __ballot_sync(0xffffffffu, cur < 0 && gl == 0);
        if (need && pos < stop) {
            const int64_t avail = min((int64_t)NG, stop - pos);
            const int rank = __popc(need & below_leader);
            if (cur < 0 && rank < avail) cur = (int32_t)(pos + rank);
            pos += min((int64_t)__popc(need), avail);
        }
        if (__ballot_sync(0xffffffffu, cur >= 0) == 0) break;
        if (cur < 0) continue;
        if (++iters > w.spin_limit) {   // a bound, not a wait: report instead of looping on
            if (gl == 0) atomicOr(err, ERR_TIMEOUT);
            cur = -1;
            aborted = true;
            continue;
        }
        const int32_t beg = KP_LDG(xadj + cur), end = KP_LDG(xadj + cur + 1);
        if (end - beg > HEAVY) {
            if (gl == 0) park<HEAVY>(w, ctr, cur, end - beg);
            cur = -1;
            continue;
        }
        const int32_t acur = rating_attr<R>(L.vwgt, L.outw, cur);
        const HashCtx hc = hash_ctx(w, L, cur);
        Proposal best;
        scan_row<R, G>(L, w, hc, cur, acur, beg + gl, end, best);
        reduce_proposal<G>(gmask, cur, best);
        int32_t next = -1;
        if (gl == 0) next = propose(w, cur, acur, best, fails);
        cur = __shfl_sync(gmask, next, leader);
    }
    if (gl == 0) {
        atomicAdd(&ctr->searches, (unsigned long long)iters);
        if (fails) atomicAdd(&ctr->failed_cas, fails);
    }
}

// The middle pass: one warp per search.  Warps take nodes parked in list0
// in turn (a counter, so rows of different lengths spread over the warps)
// and follow each node's chain; a displaced node whose row is longer than
// SUITOR_WARP_ROW is parked for the wide pass.  Power-law graphs put most of
// their entries in rows of a few dozen to a thousand entries: a warp each
// keeps eight times as many of those searches in flight as a block each.
template <int R>
__device__ __forceinline__ void suitor_warp(const DevLevel &L, const Work &w, Counters *ctr, int32_t *err) {
    const int lane = threadIdx.x & 31;
    const int32_t count = ld_relaxed_i32(&ctr->list_size[0]);
    long long iters = 0;
    unsigned long long fails = 0;
    int32_t cur = -1;
    for (;;) {
        if (cur < 0) {
            int32_t i = 0;
            if (lane == 0) i = atomicAdd(&ctr->list_size[1], 1);
            i = __shfl_sync(0xffffffffu, i, 0);
            if (i >= count) break;
            cur = w.list0[i];
        }
        if (++iters > w.spin_limit) {   // a bound, not a wait
            if (lane == 0) atomicOr(err, ERR_TIMEOUT);
            break;
        }
        const int32_t beg = KP_LDG(L.xadj + cur), end = KP_LDG(L.xadj + cur + 1);
        if (end - beg > SUITOR_WARP_ROW) {
            if (lane == 0) park<SUITOR_WARP_ROW>(w, ctr, cur, end - beg);
            cur = -1;
            continue;
        }
        const int32_t acur = rating_attr<R>(L.vwgt, L.outw, cur);
        const HashCtx hc = hash_ctx(w, L, cur);
        Proposal best;
        scan_row<R, 32>(L, w, hc, cur, acur, beg + lane, end, best);
        reduce_proposal<32>(0xffffffffu, cur, best);
        int32_t next = -1;
        if (lane == 0) next = propose(w, cur, acur, best, fails);
        cur = __shfl_sync(0xffffffffu, next, 0);
    }
    if (lane == 0) {
        atomicAdd(&ctr->searches, (unsigned long long)iters);
        if (fails) atomicAdd(&ctr->failed_cas, fails);
    }
}

// The wide pass: one block per search.  Blocks take nodes parked in list1
// in turn (a counter, so long and short rows spread over the blocks) and
// follow each node's proposal chain; every search scans the row with all
// threads of the block and reduces the best neighbour through shared memory.
// Rows of hubs (power-law graphs) are thousands of times longer than the
// mean, so this keeps a hub's search from holding one warp for its whole
// row while the rest of the GPU idles.
template <int R>
__device__ __forceinline__ void suitor_wide(const DevLevel &L, const Work &w, Counters *ctr, int32_t *err) {
    constexpr int NW = MATCH_BLOCK / 32;
    __shared__ Proposal s_best[NW];
    __shared__ int32_t s_cur;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int32_t count = ld_relaxed_i32(&ctr->list_size[2]);
    int32_t cur = -1;                 // thread 0's chain
    long long iters = 0;
    unsigned long long fails = 0;
    bool aborted = false;
    for (;;) {
        if (threadIdx.x == 0) {
            if (cur < 0 && !aborted) {
                const int32_t i = atomicAdd(&ctr->list_size[3], 1);
                cur = i < count ? w.list1[i] : -1;
            }
            if (cur >= 0 && ++iters > w.spin_limit) {   // a bound, not a wait
                atomicOr(err, ERR_TIMEOUT);
                cur = -1;
                aborted = true;
            }
            s_cur = cur;
        }
        __syncthreads();
        const int32_t c = s_cur;
        if (c < 0) break;
        const int32_t beg = KP_LDG(L.xadj + c), end = KP_LDG(L.xadj + c + 1);
        const int32_t ac = rating_attr<R>(L.vwgt, L.outw, c);
        const HashCtx hc = hash_ctx(w, L, c);
        Proposal best;
        scan_row<R, MATCH_BLOCK>(L, w, hc, c, ac, beg + (int32_t)threadIdx.x, end, best);
        reduce_proposal<32>(0xffffffffu, c, best);
        if (lane == 0) s_best[warp] = best;
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int i = 1; i < NW; i++)
                if (better(s_best[i].c, best.c, c)) best = s_best[i];
            cur = propose(w, c, ac, best, fails);
        }
        // thread 0 writes s_cur only after the barrier at the top of the next
        // search, which every thread reaches after it is done with this one
    }
    if (threadIdx.x == 0) {
        atomicAdd(&ctr->searches, (unsigned long long)iters);
        if (fails) atomicAdd(&ctr->failed_cas, fails);
    }
}

// Passes of the proposal scheme on one level.
enum : int { SUITOR_FIRST = 0, SUITOR_WARP = 1, SUITOR_WIDE = 2 };

template <int R, int PASS>
__device__ void phase_suitor(DevState *st, int level, const Work &w) {
    const DevLevel L = st->lv[level];
    if (!(L.flags & LV_ACTIVE)) return;
    Counters *ctr = &st->ctr[level];
    if (PASS == SUITOR_WIDE) {
        suitor_wide<R>(L, w, ctr, &st->err);
    } else if (PASS == SUITOR_WARP) {
        suitor_warp<R>(L, w, ctr, &st->err);
    } else {
        switch (st->suitor_lanes ? st->suitor_lanes : suitor_group(L.n, L.nnz)) {
        case 1: suitor_body<R, 1, 32>(L, w, ctr, &st->err); break;
        case 4: suitor_body<R, 4, 128>(L, w, ctr, &st->err); break;
        case 8: suitor_body<R, 8, 512>(L, w, ctr, &st->err); break;
        default: suitor_body<R, 32, 2048>(L, w, ctr, &st->err); break;
        }
    }
    // a proposal chain that ran out ends the coarsening after this level (the
    // offers stay consistent, so the level's own contraction is safe)
    if (threadIdx.x == 0 && ld_relaxed_i32(&st->err) != 0) st->stop = 1;
}

// ---------------------------------------------------------------------------
// handshake rounds
// ---------------------------------------------------------------------------
// Rates node v: its best free neighbour under the strict order, or marks v
// single when it has no free neighbour.  With recheck, v is only re-rated if
// its previous candidate has been matched meanwhile (the set of free
// neighbours only shrinks, so a still-free candidate stays the best).
template <int R, int G>
__device__ __forceinline__ void rate_node(const DevLevel &L, const Work &w, Counters *ctr, int32_t v, bool recheck) {
    const unsigned gmask = group_mask<G>();
    const int gl = threadIdx.x & (G - 1);
    const int leader = (threadIdx.x & 31) & ~(G - 1);
    int need = 0;
    if (gl == 0) {
        if (w.match[v] == -1) {
            if (!recheck) {
                need = 1;
            } else {
                const int32_t c = w.cand[v];
                need = (c < 0 || w.match[c] != -1) ? 1 : 0;
            }
        }
    }
    need = __shfl_sync(gmask, need, leader);
    if (!need) return;
    if (gl == 0) atomicAdd(&ctr->searches, 1ull);
    const int32_t beg = KP_LDG(L.xadj + v), end = KP_LDG(L.xadj + v + 1);
    const int32_t av = rating_attr<R>(L.vwgt, L.outw, v);
    const HashCtx hc = hash_ctx(w, L, v);
    Cand best;
    best.u = -1;
    best.num = best.den = best.h = 0;
    for (int32_t e = beg + gl; e < end; e += G) {
        const int32_t u = KP_LDG(L.adjncy + e);
        if (w.match[u] != -1) continue;
        Cand c;
        c.u = u;
        rating_ab<R>(KP_LDG(L.ewgt + e), av, rating_attr<R>(L.vwgt, L.outw, u), c.num, c.den);
        c.h = edge_hash_in(hc, v, u);
        if (better(c, best, v)) best = c;
    }
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1) {
        Cand o;
        o.num = __shfl_xor_sync(gmask, best.num, off);
        o.den = __shfl_xor_sync(gmask, best.den, off);
        o.h = __shfl_xor_sync(gmask, best.h, off);
        o.u = __shfl_xor_sync(gmask, best.u, off);
        if (better(o, best, v)) best = o;
    }
    if (gl == 0) {
        if (best.u < 0) {
            w.match[v] = v;   // no free neighbour: stays single (nobody reads it this phase)
            w.cand[v] = -1;
        } else {
            w.cand[v] = best.u;
        }
    }
}

template <int R, int G>
__device__ void rate_phase(const DevLevel &L, const Work &w, Counters *ctr, const int32_t *lst, int64_t cnt,
                           bool recheck) {
    const int64_t gid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
    const int64_t ngroups = (int64_t)gridDim.x * blockDim.x / G;
    for (int64_t i = gid; i < cnt; i += ngroups) rate_node<R, G>(L, w, ctr, lst ? lst[i] : (int32_t)i, recheck);
}

template <int R>
__device__ void rate_phase_any(int G, const DevLevel &L, const Work &w, Counters *ctr, const int32_t *lst,
                               int64_t cnt, bool recheck) {
    switch (G) {
    case 1: rate_phase<R, 1>(L, w, ctr, lst, cnt, recheck); break;
    case 4: rate_phase<R, 4>(L, w, ctr, lst, cnt, recheck); break;
    case 8: rate_phase<R, 8>(L, w, ctr, lst, cnt, recheck); break;
    case 16: rate_phase<R, 16>(L, w, ctr, lst, cnt, recheck); break;
    default: rate_phase<R, 32>(L, w, ctr, lst, cnt, recheck); break;
    }
}

// Handshake: v is matched when its candidate names v too; otherwise it goes
// to the next round's list.  Warp-uniform loop; appends are warp-aggregated.
__device__ __forceinline__ void hand_phase(const Work &w, const int32_t *lst, int64_t cnt, int32_t *next,
                                           int32_t *next_size) {
    const int lane = threadIdx.x & 31;
    const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < cnt; base += nthreads) {
        const int64_t i = base + lane;
        bool keep = false;
        int32_t v = -1;
        if (i < cnt) {
            v = lst ? lst[i] : (int32_t)i;
            if (w.match[v] == -1) {
                const int32_t c = w.cand[v];
                if (c >= 0 && w.cand[c] == v) w.match[v] = c;
                else keep = true;
            }
        }
        const unsigned m = __ballot_sync(0xffffffffu, keep);
        if (m) {
            int32_t pos = 0;
            if (lane == 0) pos = atomicAdd(next_size, __popc(m));
            pos = __shfl_sync(0xffffffffu, pos, 0);
            if (keep) next[pos + __popc(m & lanemask_lt())] = v;
        }
    }
}

__device__ __forceinline__ int handshake_group(int32_t n, int32_t nnz) {
    const int64_t a = n > 0 ? (int64_t)nnz : 0;
    if (a <= 3ll * n) return 1;
    if (a <= 6ll * n) return 8;
    if (a <= 14ll * n) return 16;
    return 32;
}

// Returns false when a grid barrier gave up (the caller must leave too).
template <int R>
__device__ bool phase_handshake(DevState *st, int level, const Work &w) {
    const DevLevel L = st->lv[level];
    if (!(L.flags & LV_ACTIVE)) return true;
    Counters *ctr = &st->ctr[level];
    const int G = handshake_group(L.n, L.nnz);
    if (blockIdx.x == 0 && threadIdx.x == 0) ctr->rounds = 1;
    // a barrier that gives up ends the coarsening; nodes still free then count
    // as single in the relabel, so the level's own contraction stays safe
    auto give_up = [&]() {
        if (threadIdx.x == 0) {
            atomicOr(&st->err, ERR_TIMEOUT);
            st->stop = 1;
        }
        return false;
    };
    rate_phase_any<R>(G, L, w, ctr, nullptr, L.n, false);
    if (!grid_sync(&ctr->bar, &ctr->err, w.spin_limit)) return give_up();
    hand_phase(w, nullptr, L.n, w.list0, &ctr->list_size[0]);
    if (!grid_sync(&ctr->bar, &ctr->err, w.spin_limit)) return give_up();
    int cur = 0;
    for (;;) {
        const int32_t cnt = ld_relaxed_i32(&ctr->list_size[cur]);
        if (cnt == 0) break;
        const int32_t *lst = cur ? w.list1 : w.list0;
        int32_t *nxt = cur ? w.list0 : w.list1;
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            ctr->list_size[cur ^ 1] = 0;
            ctr->rounds += 1;
        }
        rate_phase_any<R>(G, L, w, ctr, lst, cnt, true);
        if (!grid_sync(&ctr->bar, &ctr->err, w.spin_limit)) return give_up();
        hand_phase(w, lst, cnt, nxt, &ctr->list_size[cur ^ 1]);
        if (!grid_sync(&ctr->bar, &ctr->err, w.spin_limit)) return give_up();
        cur ^= 1;
    }
    return true;
}

// ---------------------------------------------------------------------------
// standalone kernels (one launch per phase)
// ---------------------------------------------------------------------------
template <int R, bool SUITOR>
__global__ void k_level_begin(DevState *st, int level, Work w) {
    phase_level_begin<R, SUITOR>(st, level, w);
}

template <int R, int PASS>
#ifndef KP_SUITOR_MIN_BLOCKS
#define KP_SUITOR_MIN_BLOCKS 3   // resident blocks per SM the register budget must allow
#endif
__global__ void __launch_bounds__(MATCH_BLOCK, KP_SUITOR_MIN_BLOCKS) k_suitor(DevState *st, int level, Work w) {
    phase_suitor<R, PASS>(st, level, w);
}

template <int R>
__global__ void __launch_bounds__(MATCH_BLOCK) k_match(DevState *st, int level, Work w) {
    phase_handshake<R>(st, level, w);
}

}  // namespace kp
