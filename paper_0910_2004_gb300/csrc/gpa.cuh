// Global Path Algorithm (Section 3.2) on one level, read from the device
// level table: the same result as the sequential algorithm, computed in
// rounds on the whole GPU.
//
// Phase 1 of the sequential algorithm scans the edges from heaviest to
// lightest under the strict edge order and collects paths and even cycles:
// an edge is taken when both ends have fewer than two collected edges, unless
// its ends are the two ends of one path with an even number of edges.  Here
// every round decides the edges that are the best undecided edge at both of
// their ends: all heavier edges at both ends are decided by then, so both
// ends' degrees are those the sequential scan sees.  An edge with an end of
// degree 0 cannot close a cycle and is taken.  An edge {u,v} with two ends of
// degree 1 walks from u along collected edges that are heavier than it (the
// path of u as the sequential scan sees it): reaching v closes a cycle
// (taken when the path has an odd number of edges, refused otherwise);
// ending elsewhere at a node whose best undecided edge is heavier than
// {u,v} waits a round (that edge comes first in the scan and may extend the
// path) or whose best edge was taken in this round (its next best is not
// known yet); a walk that meets a collected edge lighter than {u,v} ends
// there for good (that edge was decided at its node after every heavier
// one); otherwise the edge is taken.  A node with two collected edges
// refuses all its other edges.  Decisions of one round touch disjoint nodes
// and the waiting rule orders the ones whose paths meet; the heaviest
// undecided edge never waits, so every round decides at least one edge.
//
// Phase 2: a maximum weight matching of every path and cycle by dynamic
// programming over the ratings in IEEE double (the fraction num/den of the
// rating, each part rounded to double, one correctly rounded division; a
// zero denominator is +infinity), one thread per path or cycle, in the
// sequential algorithm's order: a path from its end with the smaller id, a
// cycle from the smaller end of its closing edge (its last, lightest edge)
// along the other edges; an edge is taken only when strictly better.
#pragma once

#include "match.cuh"

namespace kp {

enum : int8_t { GPA_ACCEPT = 0, GPA_CLOSE = 1, GPA_REFUSE = 2, GPA_WAIT = 3 };

// An undirected edge with everything the strict order looks at.
struct GEdge {
    uint64_t num, den, h;
    int32_t lo, hi;
};

// Strict order on two edges: true if a comes before b.
__device__ __forceinline__ bool gedge_before(const GEdge &a, const GEdge &b) {
    const int c = cmp_frac(a.num, a.den, b.num, b.den);
    if (c != 0) return c > 0;
    if (a.h != b.h) return a.h > b.h;
    if (a.lo != b.lo) return a.lo < b.lo;
    return a.hi < b.hi;
}

// Entry of neighbour y in x's row (rows are sorted), -1 if absent.
__device__ __forceinline__ eoff gpa_entry(const DevLevel &L, int32_t x, int32_t y) {
    eoff lo = KP_LDG(L.xadj + x), hi = KP_LDG(L.xadj + x + 1) - 1;
    while (lo <= hi) {
        const eoff mid = lo + ((hi - lo) >> 1);
        const int32_t a = KP_LDG(L.adjncy + mid);
        if (a == y) return mid;
        if (a < y) lo = mid + 1;
        else hi = mid - 1;
    }
    return -1;
}

template <int R>
__device__ __forceinline__ GEdge gpa_edge(const DevLevel &L, const Work &w, int32_t x, int32_t y) {
    const eoff e = gpa_entry(L, x, y);
    const int32_t wt = e >= 0 ? KP_LDG(L.ewgt + e) : 0;
    const HashCtx hc = hash_ctx(w, L, x);
    GEdge g;
    rating_ab<R>(wt, rating_attr<R>(L.vwgt, L.outw, x), rating_attr<R>(L.vwgt, L.outw, y), g.num, g.den);
    g.h = edge_hash_in(hc, x, y);
    g.lo = min(x, y);
    g.hi = max(x, y);
    return g;
}

// The rating of {x,y} as a double for the dynamic programme.
template <int R>
__device__ __forceinline__ double gpa_weight(const DevLevel &L, int32_t x, int32_t y) {
    const eoff e = gpa_entry(L, x, y);
    const int32_t wt = e >= 0 ? KP_LDG(L.ewgt + e) : 0;
    uint64_t num, den;
    rating_ab<R>(wt, rating_attr<R>(L.vwgt, L.outw, x), rating_attr<R>(L.vwgt, L.outw, y), num, den);
    return __ull2double_rn(num) / __ull2double_rn(den);
}

// Collected neighbours of x (plain loads through L2: written by other blocks
// earlier in this launch).
__device__ __forceinline__ int2 gpa_nb(const Work &w, int32_t x) { return __ldcg(reinterpret_cast<const int2 *>(w.gnb) + x); }

// The next node of a path or cycle after x, coming from prev (-1 at an end).
__device__ __forceinline__ int32_t gpa_next(const Work &w, int32_t x, int32_t prev) {
    const int2 a = gpa_nb(w, x);
    return a.x != prev ? a.x : a.y;
}

// Best undecided edge of u: to a neighbour that is not collected with u,
// has fewer than two collected edges, and whose edge was not refused for
// closing an odd cycle.  G lanes per node; cand[u] = the neighbour or -1.
// With recheck, u keeps its candidate while that edge is still undecided
// (the undecided edges of u only ever become fewer, so it stays the best);
// a refused edge has set cand to -2.
template <int R, int G>
__device__ __forceinline__ void gpa_rate_node(const DevLevel &L, const Work &w, int32_t u, bool recheck) {
    const unsigned gmask = group_mask<G>();
    const int gl = threadIdx.x & (G - 1);
    const int2 mine = gpa_nb(w, u);
    if (mine.y >= 0) {   // two collected edges: every other edge is refused
        if (gl == 0) w.cand[u] = -1;
        return;
    }
    if (recheck) {
        const int32_t c = __ldcg(w.cand + u);
        if (c >= 0 && c != mine.x && __ldcg(w.gnb + 2 * (int64_t)c + 1) < 0) return;
    }
    const eoff beg = KP_LDG(L.xadj + u), end = KP_LDG(L.xadj + u + 1);
    const int32_t au = rating_attr<R>(L.vwgt, L.outw, u);
    const HashCtx hc = hash_ctx(w, L, u);
    Cand best;
    best.u = -1;
    best.num = best.den = best.h = 0;
    for (eoff e = beg + gl; e < end; e += G) {
        const int32_t v = KP_LDG(L.adjncy + e);
        if (v == mine.x) continue;
        if (__ldcg(w.gnb + 2 * (int64_t)v + 1) >= 0) continue;
        if (__ldcg(w.grej + e)) continue;
        Cand c;
        c.u = v;
        rating_ab<R>(KP_LDG(L.ewgt + e), au, rating_attr<R>(L.vwgt, L.outw, v), c.num, c.den);
        c.h = edge_hash_in(hc, u, v);
        if (better(c, best, u)) best = c;
    }
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1) {
        Cand o;
        o.num = __shfl_xor_sync(gmask, best.num, off);
        o.den = __shfl_xor_sync(gmask, best.den, off);
        o.h = __shfl_xor_sync(gmask, best.h, off);
        o.u = __shfl_xor_sync(gmask, best.u, off);
        if (better(o, best, u)) best = o;
    }
    if (gl == 0) w.cand[u] = best.u;
}

// Rows longer than this are rated by a whole block (listed once per level
// in ghub): a hub's row is scanned again whenever its candidate is taken,
// and G lanes would hold a round for the whole row.
constexpr int32_t GPA_HUB_ROW = 2048;

// gpa_rate_node for a hub, the block's threads over the row, the best
// edge by a block reduction.  Every decision before the scan reads the same
// words in every thread, so the block takes it together.
template <int R>
__device__ void gpa_rate_hub(const DevLevel &L, const Work &w, int32_t u, bool recheck) {
    __shared__ Cand s_best[MATCH_BLOCK / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int2 mine = gpa_nb(w, u);
    if (mine.y >= 0) {
        if (threadIdx.x == 0) w.cand[u] = -1;
        return;
    }
    if (recheck) {
        const int32_t c = __ldcg(w.cand + u);
        if (c >= 0 && c != mine.x && __ldcg(w.gnb + 2 * (int64_t)c + 1) < 0) return;
    }
    const eoff beg = KP_LDG(L.xadj + u), end = KP_LDG(L.xadj + u + 1);
    const int32_t au = rating_attr<R>(L.vwgt, L.outw, u);
    const HashCtx hc = hash_ctx(w, L, u);
    Cand best;
    best.u = -1;
    best.num = best.den = best.h = 0;
    for (eoff e = beg + (eoff)threadIdx.x; e < end; e += blockDim.x) {
        const int32_t v = KP_LDG(L.adjncy + e);
        if (v == mine.x) continue;
        if (__ldcg(w.gnb + 2 * (int64_t)v + 1) >= 0) continue;
        if (__ldcg(w.grej + e)) continue;
        Cand c;
        c.u = v;
        rating_ab<R>(KP_LDG(L.ewgt + e), au, rating_attr<R>(L.vwgt, L.outw, v), c.num, c.den);
        c.h = edge_hash_in(hc, u, v);
        if (better(c, best, u)) best = c;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        Cand o;
        o.num = __shfl_xor_sync(0xffffffffu, best.num, off);
        o.den = __shfl_xor_sync(0xffffffffu, best.den, off);
        o.h = __shfl_xor_sync(0xffffffffu, best.h, off);
        o.u = __shfl_xor_sync(0xffffffffu, best.u, off);
        if (better(o, best, u)) best = o;
    }
    if (lane == 0) s_best[warp] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
        Cand b = s_best[0];
        for (int i = 1; i < MATCH_BLOCK / 32; i++)
            if (better(s_best[i], b, u)) b = s_best[i];
        w.cand[u] = b.u;
    }
    __syncthreads();   // s_best is read before the next hub
}

// Rates the round's nodes: G lanes per node, hubs (listed in ghub) a block
// each.  A hub is in the round's list exactly when its candidate is not -1
// (nodes leave the list when they find no undecided edge, and only then).
template <int R, int G>
__device__ void gpa_rate_phase(const DevLevel &L, const Work &w, const Counters *ctr, const int32_t *lst,
                               int64_t cnt) {
    const int64_t gid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
    const int64_t ngroups = (int64_t)gridDim.x * blockDim.x / G;
    for (int64_t i = gid; i < cnt; i += ngroups) {
        const int32_t u = lst ? __ldcg(lst + i) : (int32_t)i;
        if (KP_LDG(L.xadj + u + 1) - KP_LDG(L.xadj + u) > GPA_HUB_ROW) continue;   // the same in the group
        gpa_rate_node<R, G>(L, w, u, lst != nullptr);
    }
    const int32_t nh = ld_relaxed_i32(&ctr->list_size[3]);
    for (int32_t h = blockIdx.x; h < nh; h += gridDim.x) {
        const int32_t u = __ldcg(w.ghub + h);
        if (lst && __ldcg(w.cand + u) == -1) continue;   // decided in an earlier round
        gpa_rate_hub<R>(L, w, u, lst != nullptr);
    }
}

// Mutual best edges: taken at once when an end has no collected edge, else
// listed for the cycle check.  Nodes with an undecided edge stay active.
__device__ __forceinline__ void gpa_pair_phase(const Work &w, const int32_t *lst, int64_t cnt, int32_t *next,
                                               int32_t *next_size, int32_t *pend_size) {
    const int lane = threadIdx.x & 31;
    const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < cnt; base += nthreads) {
        const int64_t i = base + lane;
        bool keep = false, pend = false;
        int32_t u = -1;
        if (i < cnt) {
            u = lst ? __ldcg(lst + i) : (int32_t)i;
            const int32_t v = __ldcg(w.cand + u);
            keep = v >= 0;
            if (v > u && __ldcg(w.cand + v) == u) {
                const int2 nu = gpa_nb(w, u), nv = gpa_nb(w, v);
                if (nu.x < 0 || nv.x < 0) {   // no cycle can close: taken
                    w.gnb[2 * (int64_t)u + (nu.x >= 0)] = v;
                    w.gnb[2 * (int64_t)v + (nv.x >= 0)] = u;
                } else {
                    pend = true;
                }
            }
        }
        unsigned m = __ballot_sync(0xffffffffu, keep);
        if (m) {
            int32_t pos = 0;
            if (lane == 0) pos = atomicAdd(next_size, __popc(m));
            pos = __shfl_sync(0xffffffffu, pos, 0);
            if (keep) next[pos + __popc(m & lanemask_lt())] = u;
        }
        m = __ballot_sync(0xffffffffu, pend);
        if (m) {
            int32_t pos = 0;
            if (lane == 0) pos = atomicAdd(pend_size, __popc(m));
            pos = __shfl_sync(0xffffffffu, pos, 0);
            if (pend) w.gpend[pos + __popc(m & lanemask_lt())] = u;
        }
    }
}

// The cycle check of pending edge {u, cand[u]} (one thread each).
template <int R>
__device__ __forceinline__ int8_t gpa_check(const DevLevel &L, const Work &w, int32_t u, int32_t *err) {
    const int32_t v = __ldcg(w.cand + u);
    const GEdge e = gpa_edge<R>(L, w, u, v);
    int32_t prev = -1, cur = u;
    int64_t steps = 0;
    for (;;) {
        const int32_t nx = gpa_next(w, cur, prev);
        if (nx < 0) break;   // the path's end
        // a lighter collected edge: the path ends here for e, and cur's edges
        // heavier than that one (so heavier than e) were all decided before it
        if (!gedge_before(gpa_edge<R>(L, w, cur, nx), e)) return GPA_ACCEPT;
        prev = cur;
        cur = nx;
        steps++;
        if (cur == v) return (steps & 1) ? GPA_CLOSE : GPA_REFUSE;   // even cycle / odd cycle
        if (steps > L.n) {   // cannot happen on a path; a bound, not a wait
            atomicOr(err, ERR_TIMEOUT);
            return GPA_WAIT;
        }
    }
    // the path's end: it waits for a heavier undecided edge there, and for
    // an end whose best edge was taken this round (its next one is not known)
    const int32_t c = __ldcg(w.cand + cur);
    if (c < 0) return GPA_ACCEPT;
    const int2 a = gpa_nb(w, cur);
    if (c == a.x || c == a.y) return GPA_WAIT;
    return gedge_before(gpa_edge<R>(L, w, cur, c), e) ? GPA_WAIT : GPA_ACCEPT;
}

// Maximum weight matching of the path x_0 = s, x_1, ... (walked away from
// `from`, -1 at a path end) by dynamic programming over `edges` edges; the
// take flags go to bit `bit` of gtake at x_i.  Returns the optimum.
template <int R>
__device__ __forceinline__ double gpa_dp_forward(const DevLevel &L, const Work &w, int32_t s, int32_t from,
                                                 int32_t edges, int bit) {
    double b2 = 0.0, b1 = 0.0;   // best[i-2], best[i-1]
    int32_t prev = from, cur = s;
    for (int32_t i = 1; i <= edges; i++) {
        const int32_t nx = gpa_next(w, cur, prev);
        const double with = b2 + gpa_weight<R>(L, cur, nx);
        const bool take = with > b1;
        const double bi = take ? with : b1;
        uint8_t f = w.gtake[nx];
        f = (uint8_t)(take ? (f | (1u << bit)) : (f & ~(1u << bit)));
        w.gtake[nx] = f;
        b2 = b1;
        b1 = bi;
        prev = cur;
        cur = nx;
    }
    return b1;
}

// Backtracking of gpa_dp_forward from the path's last node `t` (walked
// towards `from`), over `edges` edges: writes the matched pairs.
__device__ __forceinline__ void gpa_dp_back(const Work &w, int32_t t, int32_t from, int32_t edges, int bit) {
    int32_t prev = from, cur = t;
    for (int32_t i = edges; i >= 1;) {
        const int32_t p = gpa_next(w, cur, prev);   // x_{i-1}
        if ((w.gtake[cur] >> bit) & 1u) {
            w.match[cur] = p;
            w.match[p] = cur;
            if (i >= 2) {
                const int32_t q = gpa_next(w, p, cur);   // x_{i-2}
                prev = p;
                cur = q;
            }
            i -= 2;
        } else {
            prev = cur;
            cur = p;
            i -= 1;
        }
    }
}

// Phase 2 for node v (every node starts single): a path is handled by its
// end with the smaller id, a cycle by the smaller end of its closing edge.
template <int R>
__device__ __forceinline__ void gpa_solve(const DevLevel &L, const Work &w, int32_t v) {
    const int2 a = gpa_nb(w, v);
    if (a.x < 0) return;   // isolated
    if (a.y < 0) {         // a path end: walk to the other end
        int32_t prev = -1, cur = v, len = 0;
        for (;;) {
            const int32_t nx = gpa_next(w, cur, prev);
            if (nx < 0) break;
            prev = cur;
            cur = nx;
            if (++len > L.n) return;   // cannot happen on a path (a bound, not a wait)
        }
        if (v > cur) return;   // the other end does it
        gpa_dp_forward<R>(L, w, v, -1, len, 0);
        gpa_dp_back(w, cur, -1, len, 0);
        return;
    }
    const int32_t b = __ldcg(w.gclose + v);
    if (b < v) return;   // not the smaller end of a closing edge
    // the cycle as the path x_0 = v .. x_K = b plus the closing edge {b, v}
    int32_t prev = b, cur = v, K = 0;
    while (cur != b) {
        const int32_t nx = gpa_next(w, cur, prev);
        if (nx < 0 || ++K > L.n) return;   // cannot happen on a cycle (a bound, not a wait)
        prev = cur;
        cur = nx;
    }
    if (K < 3) return;   // an even cycle has at least four edges
    const double without = gpa_dp_forward<R>(L, w, v, b, K, 0);
    const int32_t x1 = gpa_next(w, v, b);
    const double with = gpa_weight<R>(L, b, v) + gpa_dp_forward<R>(L, w, x1, v, K - 2, 1);
    if (with > without) {
        w.match[v] = b;
        w.match[b] = v;
        const int32_t xk1 = gpa_next(w, b, v);   // x_{K-1}
        gpa_dp_back(w, xk1, b, K - 2, 1);
    } else {
        gpa_dp_back(w, b, v, K, 0);
    }
}

// Returns false when a grid barrier gave up (the caller must leave too).
template <int R>
__device__ bool phase_gpa(DevState *st, int level, const Work &w) {
    const DevLevel L = st->lv[level];
    if (!(L.flags & LV_ACTIVE)) return true;
    Counters *ctr = &st->ctr[level];
    const int G = handshake_group(L.n, L.nnz);
    auto give_up = [&]() {
        if (threadIdx.x == 0) {
            atomicOr(&st->err, ERR_TIMEOUT);
            st->stop = 1;
        }
        return false;
    };
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = tid; v < L.n; v += nthreads) {
        reinterpret_cast<int2 *>(w.gnb)[v] = make_int2(-1, -1);
        w.gclose[v] = -1;
        w.match[v] = (int32_t)v;
    }
    for (int64_t e = tid; e < L.nnz; e += nthreads) w.grej[e] = 0;
    // the hubs of this level (list_size[3] is zero when the level starts)
    for (int64_t v = tid; v < L.n; v += nthreads)
        if (L.xadj[v + 1] - L.xadj[v] > GPA_HUB_ROW) w.ghub[atomicAdd(&ctr->list_size[3], 1)] = (int32_t)v;
    if (!grid_sync(&ctr->bar, &ctr->err, w.spin_limit)) return give_up();
    const int32_t *lst = nullptr;   // round 1: every node
    int64_t cnt = L.n;
    int cur = 0;
    for (int64_t round = 1;; round++) {
        if (round > w.spin_limit) {   // a bound, not a wait
            if (tid == 0) atomicOr(&st->err, ERR_TIMEOUT);
            return give_up();
        }
        int32_t *nxt = cur ? w.list0 : w.list1;
        if (tid == 0) {
            ctr->list_size[cur ^ 1] = 0;
            ctr->list_size[2] = 0;
            ctr->rounds = (int32_t)round;
        }
        switch (G) {
        case 1: gpa_rate_phase<R, 1>(L, w, ctr, lst, cnt); break;
        case 8: gpa_rate_phase<R, 8>(L, w, ctr, lst, cnt); break;
        case 16: gpa_rate_phase<R, 16>(L, w, ctr, lst, cnt); break;
        default: gpa_rate_phase<R, 32>(L, w, ctr, lst, cnt); break;
        }
        if (!grid_sync(&ctr->bar, &ctr->err, w.spin_limit)) return give_up();
        gpa_pair_phase(w, lst, cnt, nxt, &ctr->list_size[cur ^ 1], &ctr->list_size[2]);
        if (!grid_sync(&ctr->bar, &ctr->err, w.spin_limit)) return give_up();
        const int32_t pc = ld_relaxed_i32(&ctr->list_size[2]);
        for (int64_t i = tid; i < pc; i += nthreads) w.gdec[i] = gpa_check<R>(L, w, __ldcg(w.gpend + i), &st->err);
        if (!grid_sync(&ctr->bar, &ctr->err, w.spin_limit)) return give_up();
        for (int64_t i = tid; i < pc; i += nthreads) {
            const int8_t d = __ldcg(w.gdec + i);
            if (d == GPA_WAIT) continue;
            const int32_t u = __ldcg(w.gpend + i), v = __ldcg(w.cand + u);
            if (d == GPA_REFUSE) {
                const eoff e1 = gpa_entry(L, u, v), e2 = gpa_entry(L, v, u);
                if (e1 >= 0) w.grej[e1] = 1;
                if (e2 >= 0) w.grej[e2] = 1;
                w.cand[u] = -2;   // both ends look for their next best edge
                w.cand[v] = -2;
                continue;
            }
            w.gnb[2 * (int64_t)u + 1] = v;   // both ends had one collected edge
            w.gnb[2 * (int64_t)v + 1] = u;
            if (d == GPA_CLOSE) {
                w.gclose[u] = v;
                w.gclose[v] = u;
            }
        }
        if (!grid_sync(&ctr->bar, &ctr->err, w.spin_limit)) return give_up();
        cnt = ld_relaxed_i32(&ctr->list_size[cur ^ 1]);
        if (cnt == 0) break;
        lst = nxt;
        cur ^= 1;
    }
    for (int64_t v = tid; v < L.n; v += nthreads) gpa_solve<R>(L, w, (int32_t)v);
    return true;
}

template <int R>
__global__ void __launch_bounds__(MATCH_BLOCK) k_gpa(DevState *st, int level, Work w) {
    phase_gpa<R>(st, level, w);
}

}  // namespace kp
