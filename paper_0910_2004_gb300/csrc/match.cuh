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
// DEG0: the separately launched form, which also reports the input's
// largest degree at level 0 (the persistent tail launches nothing the
// degree could decide).
template <int R, bool SUITOR, bool DEG0 = false>
__device__ void phase_level_begin(DevState *st, int level, const Work &w) {
    const DevLevel L = st->lv[level];
    if (!(L.flags & LV_ACTIVE)) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        // what the level carves at most: map, c', batch ids and offsets,
        // coarse xadj, entries (at most nnz), Out, each 256-byte aligned
        arena_reserve(st, (20ull + sizeof(eoff)) * (unsigned long long)L.n + 8ull * (unsigned long long)L.nnz +
                              4ull * ((unsigned long long)w.num_graphs + 1) + 8ull * 256ull);
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
    if (DEG0 && level == 0 && w.deg0_host) {
        // the input's largest degree for the host (which contraction kernels
        // to launch); the last warp to add its part writes it
        int32_t d = 0;
        for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < L.n; v += stride)
            d = max(d, (int32_t)(L.xadj[v + 1] - L.xadj[v]));
        d = __reduce_max_sync(0xffffffffu, d);
        if ((threadIdx.x & 31) == 0) {
            atomicMax(&st->maxdeg0, d);
            __threadfence();
            const int32_t warps = (int32_t)((stride + 31) >> 5);
            if (atomicAdd(&st->maxdeg0_warps, 1) == warps - 1)
                *(volatile int32_t *)w.deg0_host = atomicMax(&st->maxdeg0, 0) + 1;
        }
    }
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
// An offer record as it is now, read through L2 (other threads change it by
// 128-bit CAS).  An ordinary load, so a row's gathers can be in flight
// together; a stale record only makes the CAS that expects it fail.  The
// CAS is a compiler barrier, so a record is read afresh after every proposal.
__device__ __forceinline__ Offer ld_offer(const Offer *p) {
    const int4 t = __ldcg(reinterpret_cast<const int4 *>(p));
    Offer o;
    o.s = t.x;
    o.w = t.y;
    o.as = t.z;
    o.au = t.w;
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
__device__ __forceinline__ int suitor_group(int32_t n, eoff nnz) {
    const int64_t a = n > 0 ? (int64_t)nnz : 0;
    if (a <= 12ll * n) return 1;
    if (a <= 40ll * n) return 4;
    if (a <= 160ll * n) return 8;
    return 32;
}

// A node's best proposal so far: the edge, its weight, and the record of the
// other end as it was read (the compare-and-swap expects that record).
struct Proposal {
    Cand c;
    int32_t w;
    Offer snap;
};

// Whether cur may propose to v now (v's record as read: so): v holds no
// offer, or cur's offer beats the standing one at v.  cd gets the edge as
// seen from cur.
template <int R>
__device__ __forceinline__ bool eligible_at(const HashCtx &hc, int32_t cur, int32_t acur, int32_t v, int32_t wt,
                                            const Offer &so, Cand &cd) {
    cd.u = v;
    rating_ab<R>(wt, acur, so.au, cd.num, cd.den);
    cd.h = edge_hash_in(hc, cur, v);
    if (so.s < 0) return true;
    // compare at v: the offer of cur against the standing offer of so.s (the
    // standing edge's hash only when the ratings are equal)
    uint64_t bnum, bden;
    rating_ab<R>(so.w, so.as, so.au, bnum, bden);
    const int c = cmp_frac(cd.num, cd.den, bnum, bden);
    if (c != 0) return c > 0;
    const uint64_t bh = edge_hash_in(hc, so.s, v);
    if (cd.h != bh) return cd.h > bh;
    const int32_t alo = min(v, cur), ahi = max(v, cur), blo = min(v, so.s), bhi = max(v, so.s);
    if (alo != blo) return alo < blo;
    return ahi < bhi;
}

// One thread's share of a search: the entries e0, e0 + STRIDE, ... < end of
// cur's row; the best eligible edge is kept.
template <int R, int STRIDE>
__device__ __forceinline__ void scan_row(const DevLevel &L, const Work &w, const HashCtx &hc, int32_t cur,
                                         int32_t acur, eoff e0, eoff end, Proposal &best) {
    const int32_t *KP_RESTRICT adjncy = L.adjncy;
    const int32_t *KP_RESTRICT ewgt = L.ewgt;
    best.c.u = -1;
    best.c.num = best.c.den = best.c.h = 0;
    best.w = 0;
    best.snap = {-1, 0, 0, 0};
#pragma unroll 4
    for (eoff e = e0; e < end; e += STRIDE) {
        const int32_t v = KP_LDG(adjncy + e);
        const int32_t wt = KP_LDG(ewgt + e);
        const Offer st = ld_offer(w.offer + v);
        Cand c;
        if (eligible_at<R>(hc, cur, acur, v, wt, st, c) && better(c, best.c, cur)) {
            best.c = c;
            best.w = wt;
            best.snap = st;
        }
    }
}

// A candidate without the record it was read with.
struct Cached {
    Cand c;
    int32_t w;
};

// scan_row that also keeps the second best eligible edge of the thread's
// share and counts the eligible edges it saw (up to 3).
template <int R, int STRIDE>
__device__ __forceinline__ void scan_row_top2(const DevLevel &L, const Work &w, const HashCtx &hc, int32_t cur,
                                              int32_t acur, eoff e0, eoff end, Proposal &best, Cached &second,
                                              int32_t &seen) {
    const int32_t *KP_RESTRICT adjncy = L.adjncy;
    const int32_t *KP_RESTRICT ewgt = L.ewgt;
    best.c.u = -1;
    best.c.num = best.c.den = best.c.h = 0;
    best.w = 0;
    best.snap = {-1, 0, 0, 0};
    second.c = best.c;
    second.w = 0;
    seen = 0;
#pragma unroll 4
    for (eoff e = e0; e < end; e += STRIDE) {
        const int32_t v = KP_LDG(adjncy + e);
        const int32_t wt = KP_LDG(ewgt + e);
        const Offer st = ld_offer(w.offer + v);
        Cand c;
        if (!eligible_at<R>(hc, cur, acur, v, wt, st, c)) continue;
        seen = min(seen + 1, 3);
        if (better(c, best.c, cur)) {
            second.c = best.c;
            second.w = best.w;
            best.c = c;
            best.w = wt;
            best.snap = st;
        } else if (better(c, second.c, cur)) {
            second.c = c;
            second.w = wt;
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

// Parks node v for the wide pass (list1), with an empty candidate cache.
__device__ __forceinline__ void park_wide(const Work &w, Counters *ctr, int32_t v) {
    const int32_t slot = atomicAdd(&ctr->list_size[2], 1);
    w.list1[slot] = v;
    w.wslot[v] = slot;
    if (slot < w.cache_slots) w.cache_hdr[slot] = make_int2(0, 0);
}

// First pass: G lanes per proposing node, start nodes [0, n).  Warps take
// short runs of consecutive start nodes (4 per group) from one counter, so
// the nodes in flight on the whole GPU at any time form a narrow window that
// sweeps through the ids; on mesh-like graphs with local ids the offer
// records and rating attributes the window reads stay in L2 from their first
// read to their last instead of being fetched from DRAM once per reader.
// Every group follows one proposal chain (a node, then whoever it displaced)
// and takes the next start node of its warp's run as soon as its chain ends,
// so lanes stay busy until the counter is used up.  A node whose row is
// longer than HEAVY entries is parked for the middle pass (list0) instead of
// being scanned by so few lanes; that pass hands the rows too long for a warp
// on to the wide pass.  The order of proposals does not change the matching.
template <int R, int G, int HEAVY>
__device__ __forceinline__ void suitor_body(const DevLevel &L, const Work &w, Counters *ctr, int32_t *err) {
    constexpr int NG = 32 / G;
    constexpr int RUN = 4 * NG;   // start nodes per counter step
    const unsigned gmask = group_mask<G>();
    const int lane = threadIdx.x & 31;
    const int gl = lane & (G - 1);
    const int leader = lane & ~(G - 1);
    const unsigned below_leader = (1u << leader) - 1u;
    const eoff *KP_RESTRICT xadj = L.xadj;
    const int64_t count = L.n;
    int64_t pos = 0, stop = 0;
    long long iters = 0;
    unsigned long long fails = 0;
    int32_t cur = -1;
    bool aborted = false;
    for (;;) {
        // the whole warp leaves together (full-warp votes follow)
        if (__any_sync(0xffffffffu, aborted)) break;
        // give every idle group the next start node of the warp's run, taking
        // a new run from the counter when this one is used up
        const unsigned need = __ballot_sync(0xffffffffu, cur < 0 && gl == 0);
        if (need && pos >= stop) {
            unsigned long long base = 0;
            if (lane == 0) base = atomicAdd(&ctr->start_next, (unsigned long long)RUN);
            base = __shfl_sync(0xffffffffu, base, 0);
            pos = (int64_t)min(base, (unsigned long long)count);
            stop = min(count, pos + RUN);
        }
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
        const eoff beg = KP_LDG(xadj + cur), end = KP_LDG(xadj + cur + 1);
        if (end - beg > HEAVY) {
            if (gl == 0) w.list0[atomicAdd(&ctr->list_size[0], 1)] = cur;
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
// and follow each node's chain; a node whose row is longer than
// SUITOR_WARP_ROW is parked for the wide pass.  Power-law graphs put most of
// their entries in rows of a few dozen to a thousand entries: a warp each
// keeps eight times as many of those searches in flight as a block each.
template <int R>
__device__ __forceinline__ void suitor_warp(const DevLevel &L, const Work &w, Counters *ctr, int32_t *err) {
    const int lane = threadIdx.x & 31;
    const int32_t count = ld_relaxed_i32(&ctr->list_size[0]);
    if (count == 0) return;   // nothing parked: no counter traffic
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
        const eoff beg = KP_LDG(L.xadj + cur), end = KP_LDG(L.xadj + cur + 1);
        if (end - beg > SUITOR_WARP_ROW) {
            if (lane == 0) park_wide(w, ctr, cur);
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

// The candidate cache of a long row (wide pass).  Offers only improve, so an
// edge {c,v} that was not eligible when c's row was scanned never becomes
// eligible again.  A scan of c's row therefore keeps the best eligible
// candidates it saw, in c's order and as an exact prefix of that order, and
// c's later searches (after it is displaced) take the first of them that is
// still eligible: the same proposal a full scan would make.  Only when all
// are used up is the row scanned again.  A hub displaced many times then
// scans its row a few times instead of once per displacement.

// c's cache slot, -1 if it has none (slots left from earlier levels fail
// the check against list1).
__device__ __forceinline__ int32_t cache_slot(const Work &w, int32_t count, int32_t c) {
    const int32_t slot = __ldcg(w.wslot + c);
    if (slot < 0 || slot >= count || slot >= w.cache_slots) return -1;
    return __ldcg(w.list1 + slot) == c ? slot : -1;
}

// One proposal of c from its cache (one thread).  Returns the node that
// searches next (the displaced suitor, -1 if none, or c after a lost race),
// or -2 when the cache is used up and c's row has to be scanned again.
template <int R>
__device__ __forceinline__ int32_t propose_cached(const DevLevel &L, const Work &w, int32_t slot, int32_t c,
                                                  unsigned long long &fails) {
    __threadfence();   // the cache as c's previous search left it (another block)
    int2 hd = __ldcg(w.cache_hdr + slot);
    const int32_t ac = rating_attr<R>(L.vwgt, L.outw, c);
    const HashCtx hc = hash_ctx(w, L, c);
    for (; hd.y < hd.x; hd.y++) {
        const int2 cand = __ldcg(w.cache + (int64_t)slot * SUITOR_CACHE_K + hd.y);
        const Offer so = ld_offer(w.offer + cand.x);
        Cand cd;
        if (!eligible_at<R>(hc, c, ac, cand.x, cand.y, so, cd)) continue;
        __stcg(w.cache_hdr + slot, hd);
        __threadfence();   // the cache position is visible before the proposal is
        Offer mine;
        mine.s = c;
        mine.w = cand.y;
        mine.as = ac;
        mine.au = so.au;
        if (cas_offer(w.offer + cand.x, so, mine)) return so.s;
        fails++;
        return c;
    }
    __stcg(w.cache_hdr + slot, hd);
    return -2;
}

// The wide pass: one block per search.  Blocks take nodes parked in list1
// in turn (a counter, so long and short rows spread over the blocks) and
// follow each node's proposal chain; every search scans the row with all
// threads of the block and reduces the best neighbour through shared memory.
// Rows of hubs (power-law graphs) are thousands of times longer than the
// mean, so this keeps a hub's search from holding one warp for its whole
// row while the rest of the GPU idles.  Rows longer than SUITOR_CACHE_ROW
// fill and use their candidate cache.  TAIL: the persistent tail's form,
// whose levels are small: it takes every node the first pass parked (list0,
// no middle pass) and keeps no cache, which keeps the tail's registers.
template <int R, bool TAIL>
__device__ __forceinline__ void suitor_wide(const DevLevel &L, const Work &w, Counters *ctr, int32_t *err) {
    constexpr int NW = MATCH_BLOCK / 32;
    __shared__ Proposal s_best[NW];
    __shared__ int32_t s_tid[NW], s_last[NW];
    __shared__ int32_t s_cur, s_slot, s_win, s_stop;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr bool CACHE = !TAIL;
    const int32_t *parked = TAIL ? w.list0 : w.list1;
    int32_t *next_parked = TAIL ? &ctr->list_size[1] : &ctr->list_size[3];
    const int32_t count = ld_relaxed_i32(&ctr->list_size[TAIL ? 0 : 2]);
    if (count == 0) return;   // nothing parked (the same for every thread)
    int32_t cur = -1;                 // thread 0's chain
    long long iters = 0, scans = 0;
    unsigned long long fails = 0;
    bool aborted = false;
    for (;;) {
        if (threadIdx.x == 0) {
            // the next search: from the cache while it lasts, else a scan
            int32_t slot = -1;
            for (;;) {
                if (cur < 0 && !aborted) {
                    const int32_t i = atomicAdd(next_parked, 1);
                    cur = i < count ? parked[i] : -1;
                }
                if (cur < 0) break;
                if (++iters > w.spin_limit) {   // a bound, not a wait
                    atomicOr(err, ERR_TIMEOUT);
                    cur = -1;
                    aborted = true;
                    break;
                }
                if (!CACHE || KP_LDG(L.xadj + cur + 1) - KP_LDG(L.xadj + cur) <= SUITOR_CACHE_ROW) break;
                slot = cache_slot(w, count, cur);
                if (slot < 0) break;
                const int32_t next = propose_cached<R>(L, w, slot, cur, fails);
                if (next == -2) break;   // scan the row and refill the cache
                cur = next;
                slot = -1;
            }
            s_cur = cur;
            s_slot = slot;
        }
        __syncthreads();
        const int32_t c = s_cur;
        if (c < 0) break;
        const int32_t slot = s_slot;
        const eoff beg = KP_LDG(L.xadj + c), end = KP_LDG(L.xadj + c + 1);
        const int32_t ac = rating_attr<R>(L.vwgt, L.outw, c);
        const HashCtx hc = hash_ctx(w, L, c);
        scans++;
        if (CACHE && slot >= 0) {
            // every thread keeps its two best; SUITOR_CACHE_K rounds of a
            // block-wide argmax over the threads' next candidates fill the
            // cache, which ends after a thread's second candidate if that
            // thread saw more eligible edges than it kept
            Proposal best;
            Cached second;
            int32_t seen;
            scan_row_top2<R, MATCH_BLOCK>(L, w, hc, c, ac, beg + (eoff)threadIdx.x, end, best, second, seen);
            const int32_t kept = min(seen, 2);
            int32_t idx = 0, filled = 0;
            for (int k = 0; k < SUITOR_CACHE_K; k++) {
                Cached h;
                int32_t last = 0, tid = (int32_t)threadIdx.x;
                if (idx < kept) {
                    h.c = idx == 0 ? best.c : second.c;
                    h.w = idx == 0 ? best.w : second.w;
                    last = (idx == 1 && seen > 2) ? 1 : 0;
                } else {
                    h.c.u = -1;
                    h.c.num = h.c.den = h.c.h = 0;
                    h.w = 0;
                }
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) {
                    Cached o;
                    o.c.num = __shfl_xor_sync(0xffffffffu, h.c.num, off);
                    o.c.den = __shfl_xor_sync(0xffffffffu, h.c.den, off);
                    o.c.h = __shfl_xor_sync(0xffffffffu, h.c.h, off);
                    o.c.u = __shfl_xor_sync(0xffffffffu, h.c.u, off);
                    o.w = __shfl_xor_sync(0xffffffffu, h.w, off);
                    const int32_t ot = __shfl_xor_sync(0xffffffffu, tid, off);
                    const int32_t ol = __shfl_xor_sync(0xffffffffu, last, off);
                    if (better(o.c, h.c, c)) {
                        h = o;
                        tid = ot;
                        last = ol;
                    }
                }
                if (lane == 0) {
                    s_best[warp].c = h.c;
                    s_best[warp].w = h.w;
                    s_tid[warp] = tid;
                    s_last[warp] = last;
                }
                __syncthreads();
                if (threadIdx.x == 0) {
                    for (int i = 1; i < NW; i++)
                        if (better(s_best[i].c, h.c, c)) {
                            h.c = s_best[i].c;
                            h.w = s_best[i].w;
                            tid = s_tid[i];
                            last = s_last[i];
                        }
                    if (h.c.u >= 0) {
                        __stcg(w.cache + (int64_t)slot * SUITOR_CACHE_K + k, make_int2(h.c.u, h.w));
                        filled = k + 1;
                    }
                    s_win = h.c.u >= 0 ? tid : -1;
                    s_stop = (h.c.u < 0 || last) ? 1 : 0;
                }
                __syncthreads();
                if ((int32_t)threadIdx.x == s_win) idx++;
                if (s_stop) break;
            }
            if (threadIdx.x == 0) {
                __stcg(w.cache_hdr + slot, make_int2(filled, 0));
                cur = filled > 0 ? c : -1;   // c proposes from its cache next (or stays single)
            }
            // s_stop, s_win and s_best are written again only after the
            // barrier at the top of the next search
        } else {
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
            // thread 0 writes s_cur only after the barrier at the top of the
            // next search, which every thread reaches after it is done with this one
        }
    }
    if (threadIdx.x == 0) {
        atomicAdd(&ctr->searches, (unsigned long long)scans);
        if (fails) atomicAdd(&ctr->failed_cas, fails);
    }
}

// Passes of the proposal scheme on one level: the first, middle and wide
// passes (ordinary launches, so that the kernels of other streams keep
// running beside them: a server runs several hierarchies at once), and the
// wide pass as the persistent tail runs it right after the first.
enum : int { SUITOR_FIRST = 0, SUITOR_WARP = 1, SUITOR_WIDE = 2, SUITOR_WIDE_TAIL = 3 };

template <int R, int PASS>
__device__ void phase_suitor(DevState *st, int level, const Work &w) {
    const DevLevel L = st->lv[level];
    if (!(L.flags & LV_ACTIVE)) return;
    Counters *ctr = &st->ctr[level];
    if (PASS == SUITOR_WIDE_TAIL) {
        suitor_wide<R, true>(L, w, ctr, &st->err);
    } else if (PASS == SUITOR_WARP) {
        suitor_warp<R>(L, w, ctr, &st->err);
    } else if (PASS == SUITOR_WIDE) {
        suitor_wide<R, false>(L, w, ctr, &st->err);
    } else {
        switch (st->suitor_lanes ? st->suitor_lanes : suitor_group(L.n, L.nnz)) {
        case 1: suitor_body<R, 1, 32>(L, w, ctr, &st->err); break;
        case 2: suitor_body<R, 2, 64>(L, w, ctr, &st->err); break;
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
    const eoff beg = KP_LDG(L.xadj + v), end = KP_LDG(L.xadj + v + 1);
    const int32_t av = rating_attr<R>(L.vwgt, L.outw, v);
    const HashCtx hc = hash_ctx(w, L, v);
    Cand best;
    best.u = -1;
    best.num = best.den = best.h = 0;
    for (eoff e = beg + gl; e < end; e += G) {
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

__device__ __forceinline__ int handshake_group(int32_t n, eoff nnz) {
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
    phase_level_begin<R, SUITOR, true>(st, level, w);
}

// MINB: resident blocks per SM the register budget must allow (the
// suitor_blocks knob chooses 3 or 4 for the first pass; the parked passes use 3).
template <int R, int PASS, int MINB = 3>
__global__ void __launch_bounds__(MATCH_BLOCK, MINB) k_suitor(DevState *st, int level, Work w) {
    phase_suitor<R, PASS>(st, level, w);
}

template <int R>
__global__ void __launch_bounds__(MATCH_BLOCK) k_match(DevState *st, int level, Work w) {
    phase_handshake<R>(st, level, w);
}

}  // namespace kp
