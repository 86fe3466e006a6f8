// Contraction phase: edge rating (Section 3.1), handshake matching of locally
// heaviest edges (Section 3.3), contraction (Section 2), level loop and stop
// rule (Sections 2 and 4).
//
// Per level the device work is
//   [innerOuter, level 0]  k_out_weight           Out(v)
//   k_match                one cooperative persistent launch running all
//                          handshake rounds, separated by grid barriers
//   relabel scan           coarse ids, map, c', members, row upper bounds
//   k_contract_small       coarse rows with <= 16 gathered entries: one thread
//                          gathers, sorts (register bitonic network), merges
//   k_contract_warp_list   rows of 17..32 entries: one warp, shuffle bitonic
//   k_contract_warp_smem   rows of 33..128 entries: one warp, shared memory
//   k_contract_mid         rows <= MID_MAX entries: one block, shared memory
//   k_contract_big         longer rows: one block, LSD radix sort in global
//   degree scan            coarse xadj
//   k_compact              rows moved to their final CSR place
#include <algorithm>
#include <cstring>

#include "kp_internal.cuh"

namespace kp {

constexpr int32_t SENT = 0x7fffffff;   // sorts after every node id
constexpr int MID_MAX = 2048;          // longest row handled in shared memory
constexpr int MATCH_BLOCK = 256;
constexpr int CONTRACT_BLOCK = 256;

struct Counters {
    GridBarrier bar;
    int32_t err;
    int32_t list_size[2];
    int32_t rounds;
    int32_t cn;          // coarse node count
    int32_t U;           // sum of coarse row upper bounds
    int32_t nclass[5];   // overflow lists: [1] <=32, [2] <=128, [3] <=MID_MAX, [4] longer
    int32_t nnz_out;     // coarse entry count
    unsigned long long searches;     // rating passes over a row
    unsigned long long failed_cas;   // lost proposal races
};

// ---------------------------------------------------------------------------
// ratings (Section 3.1) as exact fractions
// ---------------------------------------------------------------------------
template <int R>
__device__ __forceinline__ void rating_of(int32_t w, int32_t cv, int32_t cu, int32_t outv, int32_t outu,
                                          uint64_t &num, uint64_t &den) {
    const uint64_t W = (uint64_t)(uint32_t)w;
    if (R == KP_RATING_EXPANSION_STAR2) {
        num = W * W;
        den = (uint64_t)(uint32_t)cv * (uint64_t)(uint32_t)cu;
    } else if (R == KP_RATING_INNER_OUTER) {
        num = W;
        den = (uint64_t)((int64_t)outv + (int64_t)outu - 2 * (int64_t)w);
    } else if (R == KP_RATING_WEIGHT) {
        num = W;
        den = 1;
    } else if (R == KP_RATING_EXPANSION) {
        num = W;
        den = (uint64_t)(uint32_t)cv + (uint64_t)(uint32_t)cu;
    } else {
        num = W;
        den = (uint64_t)(uint32_t)cv * (uint64_t)(uint32_t)cu;
    }
}

// A candidate edge {v,u} seen from v.
struct Cand {
    uint64_t num, den, h;
    int32_t u;
};

// Strict order: higher rating, then higher hash, then smaller (min,max) ids.
__device__ __forceinline__ bool better(const Cand &a, const Cand &b, int32_t v) {
    if (b.u < 0) return a.u >= 0;
    if (a.u < 0) return false;
    const int c = cmp_frac(a.num, a.den, b.num, b.den);
    if (c != 0) return c > 0;
    if (a.h != b.h) return a.h > b.h;
    const int32_t alo = min(v, a.u), ahi = max(v, a.u), blo = min(v, b.u), bhi = max(v, b.u);
    if (alo != blo) return alo < blo;
    return ahi < bhi;
}

struct MatchParams {
    int32_t n;
    const int32_t *__restrict__ xadj;
    const int32_t *__restrict__ adjncy;
    const int32_t *__restrict__ ewgt;
    const int32_t *__restrict__ vwgt;
    const int32_t *__restrict__ outw;
    uint64_t seed;
    int32_t *match;   // -1 free, else partner (or self: stays single)
    int32_t *cand;    // best free neighbour from the last rating
    int32_t *list0;
    int32_t *list1;
    Counters *ctr;
    long long spin_limit;
};

// Rates node v: its best free neighbour under the strict order, or marks v
// single when it has no free neighbour.  With recheck, v is only re-rated if
// its previous candidate has been matched meanwhile (the set of free
// neighbours only shrinks, so a still-free candidate stays the best).
template <int R, int G>
__device__ __forceinline__ void rate_node(const MatchParams &p, int32_t v, bool recheck) {
    const unsigned gmask = group_mask<G>();
    const int gl = threadIdx.x & (G - 1);
    const int leader = (threadIdx.x & 31) & ~(G - 1);
    int need = 0;
    if (gl == 0) {
        if (p.match[v] == -1) {
            if (!recheck) {
                need = 1;
            } else {
                const int32_t c = p.cand[v];
                need = (c < 0 || p.match[c] != -1) ? 1 : 0;
            }
        }
    }
    need = __shfl_sync(gmask, need, leader);
    if (!need) return;
    if (gl == 0) atomicAdd(&p.ctr->searches, 1ull);
    const int32_t beg = __ldg(p.xadj + v), end = __ldg(p.xadj + v + 1);
    const int32_t cv = __ldg(p.vwgt + v);
    const int32_t outv = (R == KP_RATING_INNER_OUTER) ? __ldg(p.outw + v) : 0;
    Cand best;
    best.u = -1;
    best.num = best.den = best.h = 0;
    for (int32_t e = beg + gl; e < end; e += G) {
        const int32_t u = __ldg(p.adjncy + e);
        if (p.match[u] != -1) continue;
        const int32_t w = __ldg(p.ewgt + e);
        Cand c;
        c.u = u;
        const int32_t cu = (R == KP_RATING_INNER_OUTER || R == KP_RATING_WEIGHT) ? 0 : __ldg(p.vwgt + u);
        const int32_t outu = (R == KP_RATING_INNER_OUTER) ? __ldg(p.outw + u) : 0;
        rating_of<R>(w, cv, cu, outv, outu, c.num, c.den);
        c.h = edge_hash(p.seed, v, u);
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
            p.match[v] = v;   // no free neighbour: stays single (nobody reads it this phase)
            p.cand[v] = -1;
        } else {
            p.cand[v] = best.u;
        }
    }
}

// Handshake: v is matched when its candidate names v too; otherwise it goes
// to the next round's list.  Warp-uniform loop; appends are warp-aggregated.
__device__ __forceinline__ void hand_phase(const MatchParams &p, const int32_t *lst, int64_t cnt,
                                           int32_t *next, int32_t *next_size) {
    const int lane = threadIdx.x & 31;
    const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < cnt; base += nthreads) {
        const int64_t i = base + lane;
        bool keep = false;
        int32_t v = -1;
        if (i < cnt) {
            v = lst ? lst[i] : (int32_t)i;
            if (p.match[v] == -1) {
                const int32_t c = p.cand[v];
                if (c >= 0 && p.cand[c] == v) p.match[v] = c;
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

template <int R, int G>
__global__ void __launch_bounds__(MATCH_BLOCK) k_match(MatchParams p) {
    const int64_t gid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
    const int64_t ngroups = (int64_t)gridDim.x * blockDim.x / G;
    if (blockIdx.x == 0 && threadIdx.x == 0) p.ctr->rounds = 1;
    for (int64_t v = gid; v < p.n; v += ngroups) rate_node<R, G>(p, (int32_t)v, false);
    if (!grid_sync(&p.ctr->bar, &p.ctr->err, p.spin_limit)) return;
    hand_phase(p, nullptr, p.n, p.list0, &p.ctr->list_size[0]);
    if (!grid_sync(&p.ctr->bar, &p.ctr->err, p.spin_limit)) return;
    int cur = 0;
    for (;;) {
        const int32_t cnt = ld_relaxed_i32(&p.ctr->list_size[cur]);
        if (cnt == 0) break;
        const int32_t *lst = cur ? p.list1 : p.list0;
        int32_t *nxt = cur ? p.list0 : p.list1;
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            p.ctr->list_size[cur ^ 1] = 0;
            p.ctr->rounds += 1;
        }
        for (int64_t i = gid; i < cnt; i += ngroups) rate_node<R, G>(p, lst[i], true);
        if (!grid_sync(&p.ctr->bar, &p.ctr->err, p.spin_limit)) return;
        hand_phase(p, lst, cnt, nxt, &p.ctr->list_size[cur ^ 1]);
        if (!grid_sync(&p.ctr->bar, &p.ctr->err, p.spin_limit)) return;
        cur ^= 1;
    }
}

// ---------------------------------------------------------------------------
// proposal matching (Suitor scheme, Manne & Halappanavar 2014)
// ---------------------------------------------------------------------------
// Every node proposes to its best neighbour whose standing offer it beats; a
// displaced proposer proposes again.  Under a strict edge order the pairs of
// mutual proposals are exactly the Greedy matching (Section 3.2), i.e. the
// fixed point of the handshake rounds (Section 3.3), reached without rounds
// or grid barriers.
//
// Offer record of node u (16 bytes, updated by one 128-bit CAS): the current
// suitor s (-1: none), omega(s,u), the rating attribute of s, and u's own
// rating attribute (c for the c-based ratings, Out for innerOuter), so one
// gather per neighbour yields both ratings a comparison needs.
struct __align__(16) Offer {
    int32_t s;
    int32_t w;
    int32_t as;
    int32_t au;
};

template <int R>
__device__ __forceinline__ int32_t rating_attr(const int32_t *__restrict__ vwgt, const int32_t *__restrict__ outw,
                                               int32_t v) {
    if (R == KP_RATING_INNER_OUTER) return __ldg(outw + v);
    if (R == KP_RATING_WEIGHT) return 0;
    return __ldg(vwgt + v);
}

// The rating of an edge with weight w between nodes of attributes a and b
// (symmetric in a and b for every rating).
template <int R>
__device__ __forceinline__ void rating_ab(int32_t w, int32_t a, int32_t b, uint64_t &num, uint64_t &den) {
    rating_of<R>(w, a, b, a, b, num, den);
}

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

struct SuitorParams {
    int32_t n;
    const int32_t *__restrict__ xadj;
    const int32_t *__restrict__ adjncy;
    const int32_t *__restrict__ ewgt;
    const int32_t *__restrict__ vwgt;
    const int32_t *__restrict__ outw;
    uint64_t seed;
    Offer *offer;
    int32_t *match;
    int32_t *parked;        // nodes left to the wide pass
    int32_t *parked_size;
    Counters *ctr;
    long long spin_limit;
};

template <int R>
__global__ void k_offer_init(SuitorParams p) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < p.n; v += stride) {
        Offer o;
        o.s = -1;
        o.w = 0;
        o.as = 0;
        o.au = rating_attr<R>(p.vwgt, p.outw, (int32_t)v);
        p.offer[v] = o;
    }
}

// G lanes per proposing node.  Start nodes are [0, n) (FROM_LIST = false)
// or the parked list (FROM_LIST = true).  Every warp owns one contiguous range
// of start nodes; its 32/G groups each follow one proposal chain (a node,
// then whoever it displaced) and take the next start node of the range as
// soon as their chain ends, so lanes stay busy until the range is used up.
// With HEAVY > 0 a node whose row is longer than HEAVY entries is parked on
// p.parked instead of being scanned by so few lanes; a later FROM_LIST pass
// with G = 32 finishes those.  The order in which nodes propose does not
// change the final matching.
template <int R, int G, int HEAVY, bool FROM_LIST>
__global__ void __launch_bounds__(MATCH_BLOCK) k_suitor(SuitorParams p) {
    constexpr int NG = 32 / G;
    const unsigned gmask = group_mask<G>();
    const int lane = threadIdx.x & 31;
    const int gl = lane & (G - 1);
    const int leader = lane & ~(G - 1);
    const unsigned below_leader = (1u << leader) - 1u;
    const int64_t count = FROM_LIST ? (int64_t)ld_relaxed_i32(p.parked_size) : (int64_t)p.n;
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
            if (cur < 0 && rank < avail) cur = FROM_LIST ? p.parked[pos + rank] : (int32_t)(pos + rank);
            pos += min((int64_t)__popc(need), avail);
        }
        if (__ballot_sync(0xffffffffu, cur >= 0) == 0) break;
        if (cur < 0) continue;
        if (++iters > p.spin_limit) {   // a bound, not a wait: report instead of looping on
            if (gl == 0) atomicOr(&p.ctr->err, ERR_TIMEOUT);
            cur = -1;
            aborted = true;
            continue;
        }
        const int32_t beg = __ldg(p.xadj + cur), end = __ldg(p.xadj + cur + 1);
        if (HEAVY > 0 && end - beg > HEAVY) {   // park it for the wide pass
            if (gl == 0) p.parked[atomicAdd(p.parked_size, 1)] = cur;
            cur = -1;
            continue;
        }
        const int32_t acur = rating_attr<R>(p.vwgt, p.outw, cur);
        Cand best;
        best.u = -1;
        best.num = best.den = best.h = 0;
        int32_t bw = 0;
        Offer bsnap = {-1, 0, 0, 0};
#pragma unroll 4
        for (int32_t e = beg + gl; e < end; e += G) {
            const int32_t v = __ldg(p.adjncy + e);
            const int32_t w = __ldg(p.ewgt + e);
            const Offer st = ld_offer(p.offer + v);
            Cand c;
            c.u = v;
            rating_ab<R>(w, acur, st.au, c.num, c.den);
            c.h = edge_hash(p.seed, cur, v);
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
                b.h = edge_hash(p.seed, st.s, v);
                eligible = better(a, b, v);
            }
            if (eligible && better(c, best, cur)) {
                best = c;
                bw = w;
                bsnap = st;
            }
        }
#pragma unroll
        for (int off = G / 2; off > 0; off >>= 1) {
            Cand o;
            o.num = __shfl_xor_sync(gmask, best.num, off);
            o.den = __shfl_xor_sync(gmask, best.den, off);
            o.h = __shfl_xor_sync(gmask, best.h, off);
            o.u = __shfl_xor_sync(gmask, best.u, off);
            const int32_t ow = __shfl_xor_sync(gmask, bw, off);
            Offer os;
            os.s = __shfl_xor_sync(gmask, bsnap.s, off);
            os.w = __shfl_xor_sync(gmask, bsnap.w, off);
            os.as = __shfl_xor_sync(gmask, bsnap.as, off);
            os.au = __shfl_xor_sync(gmask, bsnap.au, off);
            if (better(o, best, cur)) {
                best = o;
                bw = ow;
                bsnap = os;
            }
        }
        int32_t next = -1;
        if (best.u >= 0 && gl == 0) {
            Offer mine;
            mine.s = cur;
            mine.w = bw;
            mine.as = acur;
            mine.au = bsnap.au;
            // success: the displaced suitor (if any) proposes next;
            // failure: the record changed under us, so cur searches again
            if (cas_offer(p.offer + best.u, bsnap, mine)) {
                next = bsnap.s;
            } else {
                next = cur;
                fails++;
            }
        }
        cur = __shfl_sync(gmask, next, leader);
    }
    if (gl == 0) {
        atomicAdd(&p.ctr->searches, (unsigned long long)iters);
        if (fails) atomicAdd(&p.ctr->failed_cas, fails);
    }
}

// The matching: pairs of mutual proposals; everyone else stays single.
__global__ void k_suitor_final(SuitorParams p) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < p.n; v += stride) {
        const int32_t s = p.offer[v].s;
        p.match[v] = (s >= 0 && p.offer[s].s == (int32_t)v) ? s : (int32_t)v;
    }
}

// Out(v) = sum of the weights of v's edges (Section 3.1), for innerOuter.
__global__ void k_out_weight(int32_t n, const int32_t *__restrict__ xadj, const int32_t *__restrict__ ewgt,
                             int32_t *__restrict__ outw) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t v = t >> 3;
    const int gl = threadIdx.x & 7;
    if (v >= n) return;
    const unsigned gmask = group_mask<8>();
    int64_t s = 0;
    for (int32_t e = xadj[v] + gl; e < xadj[v + 1]; e += 8) s += ewgt[e];
#pragma unroll
    for (int off = 4; off > 0; off >>= 1) s += __shfl_xor_sync(gmask, s, off);
    if (gl == 0) outw[v] = (int32_t)s;
}

// ---------------------------------------------------------------------------
// relabel: coarse ids, map, coarse node weights, members, row upper bounds
// ---------------------------------------------------------------------------
struct RelabelOp {
    int32_t n;
    const int32_t *match, *xadj, *vwgt;
    int32_t *map, *first, *second, *cvwgt, *off;
    Counters *ctr;
    __device__ uint64_t load(int64_t v) const {
        const int32_t p = match[v];
        if (p < v) return 0;   // not the representative of its pair
        int32_t ub = xadj[v + 1] - xadj[v];
        if (p != v) ub += xadj[p + 1] - xadj[p] - 2;   // the pair's own edge is dropped
        return (1ull << 32) | (uint32_t)ub;
    }
    __device__ void store(int64_t v, uint64_t excl, uint64_t val) const {
        if (val == 0) return;
        const int32_t x = (int32_t)(excl >> 32);
        const int32_t p = match[v];
        map[v] = x;
        first[x] = (int32_t)v;
        if (p != v) {
            map[p] = x;
            second[x] = p;
            cvwgt[x] = vwgt[v] + vwgt[p];
        } else {
            second[x] = -1;
            cvwgt[x] = vwgt[v];
        }
        off[x] = (int32_t)(excl & 0xffffffffu);
    }
    __device__ void total(uint64_t t) const {
        const int32_t cn = (int32_t)(t >> 32);
        ctr->cn = cn;
        ctr->U = (int32_t)(t & 0xffffffffu);
        off[cn] = (int32_t)(t & 0xffffffffu);
    }
};

struct DegScanOp {
    int32_t cn;
    const int32_t *degp;
    int32_t *cxadj;
    Counters *ctr;
    __device__ uint64_t load(int64_t x) const { return (uint64_t)(uint32_t)degp[x]; }
    __device__ void store(int64_t x, uint64_t excl, uint64_t) const { cxadj[x] = (int32_t)excl; }
    __device__ void total(uint64_t t) const {
        cxadj[cn] = (int32_t)t;
        ctr->nnz_out = (int32_t)t;
    }
};

struct ContractParams {
    int32_t cn;
    const int32_t *__restrict__ xadj;
    const int32_t *__restrict__ adjncy;
    const int32_t *__restrict__ ewgt;
    const int32_t *__restrict__ map;
    const int32_t *__restrict__ first;
    const int32_t *__restrict__ second;
    const int32_t *__restrict__ off;
    int32_t *tmp_adj;   // coarse row x is built at off[x]
    int32_t *tmp_w;
    int32_t *big_adj;   // radix-sort ping-pong buffers for long rows (same offsets)
    int32_t *big_w;
    int32_t *degp;      // coarse row length after merging
    int32_t *outw;      // Out of the coarse node (sum of its row), may be null
    int32_t *lists[5];  // overflow lists by class (index 1..4)
    Counters *ctr;
};

// Rows with at most G gathered entries: one G-lane group per coarse node.
// The group gathers (map(u), omega) from both members' rows, drops the
// contracted edge, sorts by coarse neighbour with a bitonic network over the
// lanes, merges equal neighbours by a segmented sum and writes the row.
// Nodes with longer rows are appended to the overflow lists.
template <int G>
__device__ __forceinline__ void contract_group(const ContractParams &p, int32_t x, int32_t xa, int32_t da,
                                               int32_t xb, int32_t db) {
    const int lane = threadIdx.x & 31;
    const int gl = lane & (G - 1);
    const int gbase = lane & ~(G - 1);
    const unsigned gmask = group_mask<G>();
    constexpr unsigned GBITS = (G == 32) ? 0xffffffffu : ((1u << G) - 1u);
    const int32_t L = da + db;
    int32_t key = SENT, val = 0;
    if (gl < L) {
        const int32_t e = gl < da ? xa + gl : xb + (gl - da);
        const int32_t t = p.map[p.adjncy[e]];
        if (t != x) {
            key = t;
            val = p.ewgt[e];
        }
    }
#pragma unroll
    for (int k = 2; k <= G; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            const int32_t ok = __shfl_xor_sync(gmask, key, j);
            const int32_t ov = __shfl_xor_sync(gmask, val, j);
            const bool up = (gl & k) == 0;
            const bool lower = (gl & j) == 0;
            const bool take = lower ? (up ? ok < key : ok > key) : (up ? ok > key : ok < key);
            if (take) {
                key = ok;
                val = ov;
            }
        }
    }
    const int32_t prev = __shfl_up_sync(gmask, key, 1, G);
    const int32_t next = __shfl_down_sync(gmask, key, 1, G);
    const bool valid = key != SENT;
    const bool head = valid && (gl == 0 || prev != key);
    const bool tail = valid && (gl == G - 1 || next != key);
    int32_t s = val;
#pragma unroll
    for (int d = 1; d < G; d <<= 1) {
        const int32_t y = __shfl_up_sync(gmask, s, d, G);
        if (gl >= d) s += y;
    }
    const unsigned heads = (__ballot_sync(gmask, head) >> gbase) & GBITS;
    const unsigned tails = (__ballot_sync(gmask, tail) >> gbase) & GBITS;
    const unsigned upto = (gl == 31) ? 0xffffffffu : ((2u << gl) - 1u);
    const unsigned hb = heads & upto;
    const int start = hb ? 31 - __clz(hb) : 0;
    const int32_t before = __shfl_sync(gmask, s, start > 0 ? start - 1 : 0, G);
    const int32_t run = s - (start > 0 ? before : 0);
    const int32_t total = __shfl_sync(gmask, s, G - 1, G);
    if (tail) {
        const int32_t idx = __popc(tails & ((1u << gl) - 1u));
        const int32_t o = p.off[x];
        p.tmp_adj[o + idx] = key;
        p.tmp_w[o + idx] = run;
    }
    if (gl == 0) {
        p.degp[x] = __popc(tails);
        if (p.outw) p.outw[x] = total;
    }
}

// Rows with at most 16 gathered entries: one thread per coarse node.  The
// entries (map(u), omega) are packed as (key << 32 | omega) in 16 registers,
// sorted by a bitonic network (sentinels last), merged run by run and
// written.  Longer rows go to the overflow lists (warp-aggregated appends).
constexpr int TNET = 16;

__device__ __forceinline__ void contract_thread(const ContractParams &p, int32_t x, int32_t xa, int32_t da,
                                                int32_t xb, int32_t db) {
    constexpr uint64_t SENT64 = (uint64_t)SENT << 32;
    uint64_t r[TNET];
#pragma unroll
    for (int i = 0; i < TNET; i++) {
        uint64_t v = SENT64;
        if (i < da + db) {
            const int32_t e = i < da ? xa + i : xb + (i - da);
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
    const int32_t o = p.off[x];
    int32_t cnt = 0, curk = -1, sum = 0, total = 0;
#pragma unroll
    for (int i = 0; i < TNET; i++) {
        const int32_t k = (int32_t)(r[i] >> 32);
        const int32_t w = (int32_t)(uint32_t)r[i];
        if (k != SENT) {
            total += w;
            if (k == curk) {
                sum += w;
            } else {
                if (curk >= 0) {
                    p.tmp_adj[o + cnt] = curk;
                    p.tmp_w[o + cnt] = sum;
                    cnt++;
                }
                curk = k;
                sum = w;
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

__global__ void __launch_bounds__(CONTRACT_BLOCK) k_contract_small(ContractParams p) {
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t x0 = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); x0 < p.cn; x0 += stride) {
        const int64_t x = x0 + lane;
        int cls = -1;
        int32_t da = 0, db = 0, xa = 0, xb = 0;
        if (x < p.cn) {
            const int32_t a = p.first[x];
            const int32_t b = p.second[x];
            xa = p.xadj[a];
            da = p.xadj[a + 1] - xa;
            if (b >= 0) {
                xb = p.xadj[b];
                db = p.xadj[b + 1] - xb;
            }
            const int32_t L = da + db;
            cls = L <= TNET ? 0 : L <= 32 ? 1 : L <= 128 ? 2 : L <= MID_MAX ? 3 : 4;
        }
#pragma unroll
        for (int c = 1; c <= 4; c++) {
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
        if (cls == 0) contract_thread(p, (int32_t)x, xa, da, xb, db);
    }
}

// Rows of 33..128 gathered entries (overflow class 2): one warp each,
// bitonic sort of up to 128 (key, omega) pairs in the warp's shared memory,
// run indices by a warp scan of the head flags, run sums by shared atomics.
constexpr int WSORT = 128;

__global__ void __launch_bounds__(CONTRACT_BLOCK) k_contract_warp_smem(ContractParams p) {
    constexpr int NW = CONTRACT_BLOCK / 32;
    __shared__ int32_t sk[NW][WSORT];
    __shared__ int32_t sv[NW][WSORT];
    __shared__ int32_t ss[NW][WSORT];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int32_t *K = sk[warp], *V = sv[warp], *S = ss[warp];
    const int32_t count = p.ctr->nclass[2];
    const int64_t warp_id = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t li = warp_id; li < count; li += nwarps) {
        const int32_t x = p.lists[2][li];
        const int32_t a = p.first[x], b = p.second[x];
        const int32_t xa = p.xadj[a], da = p.xadj[a + 1] - xa;
        const int32_t xb = b >= 0 ? p.xadj[b] : 0, db = b >= 0 ? p.xadj[b + 1] - xb : 0;
        const int32_t L = da + db;
        const int P = L <= 64 ? 64 : 128;
        for (int i = lane; i < P; i += 32) {
            int32_t key = SENT, val = 0;
            if (i < L) {
                const int32_t e = i < da ? xa + i : xb + (i - da);
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
        // P/32 consecutive items per lane
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
        const int32_t o = p.off[x];
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
}

// Rows of G < L <= 32 gathered entries (overflow class 1): one warp each.
__global__ void __launch_bounds__(CONTRACT_BLOCK) k_contract_warp_list(ContractParams p) {
    const int32_t count = p.ctr->nclass[1];
    const int64_t warp_id = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = warp_id; i < count; i += nwarps) {
        const int32_t x = p.lists[1][i];
        const int32_t a = p.first[x], b = p.second[x];
        const int32_t xa = p.xadj[a], da = p.xadj[a + 1] - xa;
        const int32_t xb = b >= 0 ? p.xadj[b] : 0, db = b >= 0 ? p.xadj[b + 1] - xb : 0;
        contract_group<32>(p, x, xa, da, xb, db);
    }
}

// Rows of 33..MID_MAX gathered entries: one block per coarse node, bitonic
// sort in shared memory, then run heads, run sums and the merged row.
__global__ void __launch_bounds__(CONTRACT_BLOCK) k_contract_mid(ContractParams p) {
    const int32_t *list = p.lists[3];
    const int32_t count = p.ctr->nclass[3];
    __shared__ int32_t keys[MID_MAX];
    __shared__ int32_t vals[MID_MAX];
    __shared__ int32_t sums[MID_MAX];
    __shared__ int32_t s_red[CONTRACT_BLOCK / 32];
    constexpr int IPT = MID_MAX / CONTRACT_BLOCK;
    for (int32_t li = blockIdx.x; li < count; li += gridDim.x) {
        const int32_t x = list[li];
        const int32_t a = p.first[x], b = p.second[x];
        const int32_t xa = p.xadj[a], da = p.xadj[a + 1] - xa;
        const int32_t xb = b >= 0 ? p.xadj[b] : 0, db = b >= 0 ? p.xadj[b + 1] - xb : 0;
        const int32_t L = da + db;
        int32_t P = 64;
        while (P < L) P <<= 1;
        for (int32_t i = threadIdx.x; i < P; i += blockDim.x) {
            int32_t key = SENT, val = 0;
            if (i < L) {
                const int32_t e = i < da ? xa + i : xb + (i - da);
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
        // run index of every element: exclusive scan of the head flags over
        // IPT consecutive items per thread
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
        const int32_t o = p.off[x];
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
            for (int w = 0; w < CONTRACT_BLOCK / 32; w++) t += s_red[w];
            p.degp[x] = (int32_t)tot;
            if (p.outw) p.outw[x] = t;
        }
        __syncthreads();
    }
}

// Rows longer than MID_MAX gathered entries: one block per coarse node.
// 1. gather (map(u), omega) without the contracted edge into tmp at off[x]
// 2. stable LSD radix sort by coarse neighbour, 8 bits per pass, ping-pong
//    between tmp and big at the same offsets (an extra copy makes the number
//    of moves odd, so the sorted row ends in big); each chunk of one element
//    per thread is ranked with warp match masks and per-warp digit counts
// 3. merge equal neighbours from big back into tmp (run sums by atomics)
__global__ void __launch_bounds__(CONTRACT_BLOCK) k_contract_big(ContractParams p, int passes) {
    const int32_t *list = p.lists[4];
    const int32_t count = p.ctr->nclass[4];
    constexpr int NW = CONTRACT_BLOCK / 32;
    __shared__ int32_t base[256];
    __shared__ int32_t chunk_tot[256];
    __shared__ int32_t wcnt[NW][256];
    __shared__ int32_t s_red[NW];
    __shared__ int32_t s_carry;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int32_t li = blockIdx.x; li < count; li += gridDim.x) {
        const int32_t x = list[li];
        const int32_t a = p.first[x], b = p.second[x];
        const int32_t xa = p.xadj[a], da = p.xadj[a + 1] - xa;
        const int32_t xb = b >= 0 ? p.xadj[b] : 0, db = b >= 0 ? p.xadj[b + 1] - xb : 0;
        const int32_t L = da + db;
        const int32_t o = p.off[x];
        // 1. gather with compaction
        if (threadIdx.x == 0) s_carry = 0;
        __syncthreads();
        for (int32_t c0 = 0; c0 < L; c0 += CONTRACT_BLOCK) {
            const int32_t i = c0 + threadIdx.x;
            int32_t t = x, w = 0;
            if (i < L) {
                const int32_t e = i < da ? xa + i : xb + (i - da);
                t = p.map[p.adjncy[e]];
                w = p.ewgt[e];
            }
            const bool keep = i < L && t != x;
            uint64_t tot;
            const int32_t pos = (int32_t)block_exclusive_scan<CONTRACT_BLOCK>(keep ? 1 : 0, &tot);
            const int32_t carry = s_carry;
            if (keep) {
                p.tmp_adj[o + carry + pos] = t;
                p.tmp_w[o + carry + pos] = w;
            }
            __syncthreads();
            if (threadIdx.x == 0) s_carry = carry + (int32_t)tot;
            __syncthreads();
        }
        const int32_t M = s_carry;   // == off[x+1] - off[x]
        // 2. radix passes
        int32_t *src_k = p.tmp_adj + o, *src_v = p.tmp_w + o;
        int32_t *dst_k = p.big_adj + o, *dst_v = p.big_w + o;
        const int moves = (passes & 1) ? passes : passes + 1;
        for (int pass = 0; pass < moves; pass++) {
            if (pass >= passes) {
                for (int32_t i = threadIdx.x; i < M; i += blockDim.x) {
                    dst_k[i] = src_k[i];
                    dst_v[i] = src_v[i];
                }
            } else {
                const int shift = 8 * pass;
                for (int i = threadIdx.x; i < 256; i += blockDim.x) base[i] = 0;
                __syncthreads();
                for (int32_t i = threadIdx.x; i < M; i += blockDim.x)
                    atomicAdd(&base[(src_k[i] >> shift) & 255], 1);
                __syncthreads();
                if (threadIdx.x == 0) {
                    int32_t run = 0;
                    for (int d = 0; d < 256; d++) {
                        const int32_t c = base[d];
                        base[d] = run;
                        run += c;
                    }
                }
                __syncthreads();
                for (int32_t c0 = 0; c0 < M; c0 += CONTRACT_BLOCK) {
                    for (int i = threadIdx.x; i < NW * 256; i += blockDim.x) (&wcnt[0][0])[i] = 0;
                    __syncthreads();
                    const int32_t i = c0 + threadIdx.x;
                    const bool valid = i < M;
                    const int32_t k = valid ? src_k[i] : 0;
                    const int32_t v = valid ? src_v[i] : 0;
                    const int d = valid ? ((k >> shift) & 255) : 256 + lane;   // invalid lanes: unique
                    const unsigned peers = __match_any_sync(0xffffffffu, d);
                    const int wr = __popc(peers & lanemask_lt());
                    if (valid && wr == 0) wcnt[warp][d] = __popc(peers);
                    __syncthreads();
                    if (threadIdx.x < 256) {
                        int32_t run = 0;
                        for (int w2 = 0; w2 < NW; w2++) {
                            const int32_t c = wcnt[w2][threadIdx.x];
                            wcnt[w2][threadIdx.x] = run;
                            run += c;
                        }
                        chunk_tot[threadIdx.x] = run;
                    }
                    __syncthreads();
                    if (valid) {
                        const int32_t r = base[d] + wcnt[warp][d] + wr;
                        dst_k[r] = k;
                        dst_v[r] = v;
                    }
                    __syncthreads();
                    if (threadIdx.x < 256) base[threadIdx.x] += chunk_tot[threadIdx.x];
                    __syncthreads();
                }
            }
            __syncthreads();
            int32_t *tk = src_k, *tv = src_v;
            src_k = dst_k;
            src_v = dst_v;
            dst_k = tk;
            dst_v = tv;
        }
        // now src == big (odd number of moves); 3. merge into tmp
        for (int32_t i = threadIdx.x; i < M; i += blockDim.x) p.tmp_w[o + i] = 0;
        if (threadIdx.x == 0) s_carry = 0;
        __syncthreads();
        int32_t wsum = 0;
        for (int32_t c0 = 0; c0 < M; c0 += CONTRACT_BLOCK) {
            const int32_t i = c0 + threadIdx.x;
            const bool valid = i < M;
            const int32_t k = valid ? src_k[i] : SENT;
            const bool head = valid && (i == 0 || src_k[i - 1] != k);
            uint64_t tot;
            const int32_t pos = (int32_t)block_exclusive_scan<CONTRACT_BLOCK>(head ? 1 : 0, &tot);
            const int32_t carry = s_carry;
            if (valid) {
                const int32_t r = carry + pos + (head ? 1 : 0) - 1;
                if (head) p.tmp_adj[o + r] = k;
                atomicAdd(&p.tmp_w[o + r], src_v[i]);
                wsum += src_v[i];
            }
            __syncthreads();
            if (threadIdx.x == 0) s_carry = carry + (int32_t)tot;
            __syncthreads();
        }
        for (int off2 = 16; off2 > 0; off2 >>= 1) wsum += __shfl_xor_sync(0xffffffffu, wsum, off2);
        if (lane == 0) s_red[warp] = wsum;
        __syncthreads();
        if (threadIdx.x == 0) {
            int32_t t = 0;
            for (int w2 = 0; w2 < NW; w2++) t += s_red[w2];
            p.degp[x] = s_carry;
            if (p.outw) p.outw[x] = t;
        }
        __syncthreads();
    }
}

// Moves every merged coarse row from its upper-bound slot to the CSR.
__global__ void k_compact(int32_t cn, const int32_t *__restrict__ off, const int32_t *__restrict__ degp,
                          const int32_t *__restrict__ cxadj, const int32_t *__restrict__ tmp_adj,
                          const int32_t *__restrict__ tmp_w, int32_t *__restrict__ cadj,
                          int32_t *__restrict__ cw) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t g = t >> 3; g < cn; g += stride >> 3) {
        const int gl = threadIdx.x & 7;
        const int32_t o = off[g], d = degp[g], s = cxadj[g];
        for (int32_t i = gl; i < d; i += 8) {
            cadj[s + i] = tmp_adj[o + i];
            cw[s + i] = tmp_w[o + i];
        }
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
namespace {

int g_coop_supported = -1;

template <int R, int G>
kp_status launch_match_rg(const MatchParams &p, cudaStream_t s) {
    static int occ = -1;
    if (occ < 0) {
        int o = 0;
        KP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_match<R, G>, MATCH_BLOCK, 0));
        occ = o > 0 ? o : 1;
    }
    int64_t want = ((int64_t)p.n * G + MATCH_BLOCK - 1) / MATCH_BLOCK;
    int64_t cap = (int64_t)occ * num_sms();
    int grid = (int)std::max<int64_t>(1, std::min(want, cap));
    MatchParams q = p;
    void *args[] = {&q};
    KP_CUDA(cudaLaunchCooperativeKernel((const void *)k_match<R, G>, dim3(grid), dim3(MATCH_BLOCK), args, 0, s));
    return KP_OK;
}

template <int R>
kp_status launch_match_r(const MatchParams &p, int G, cudaStream_t s) {
    switch (G) {
    case 4: return launch_match_rg<R, 4>(p, s);
    case 8: return launch_match_rg<R, 8>(p, s);
    case 16: return launch_match_rg<R, 16>(p, s);
    default: return launch_match_rg<R, 32>(p, s);
    }
}

kp_status launch_match(int rating, const MatchParams &p, int G, cudaStream_t s) {
    switch (rating) {
    case KP_RATING_EXPANSION_STAR2: return launch_match_r<KP_RATING_EXPANSION_STAR2>(p, G, s);
    case KP_RATING_INNER_OUTER: return launch_match_r<KP_RATING_INNER_OUTER>(p, G, s);
    case KP_RATING_WEIGHT: return launch_match_r<KP_RATING_WEIGHT>(p, G, s);
    case KP_RATING_EXPANSION: return launch_match_r<KP_RATING_EXPANSION>(p, G, s);
    case KP_RATING_EXPANSION_STAR: return launch_match_r<KP_RATING_EXPANSION_STAR>(p, G, s);
    default: return set_error(KP_ERR_UNSUPPORTED, "unknown rating");
    }
}

// One group per start node; nodes with rows longer than HEAVY are parked and
// finished by one warp each.
template <int R, int G, int HEAVY>
kp_status launch_suitor_rg(const SuitorParams &p, cudaStream_t s) {
    // persistent grid: the blocks that fit at once, fewer for small levels
    static int occ = -1;
    if (occ < 0) {
        int o = 0;
        KP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_suitor<R, G, HEAVY, false>, MATCH_BLOCK, 0));
        occ = o > 0 ? o : 1;
    }
    const int64_t want = ((int64_t)p.n * G + MATCH_BLOCK - 1) / MATCH_BLOCK;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)occ * num_sms()));
    const int grid1 = (int)std::max<int64_t>(1, std::min<int64_t>(((int64_t)p.n + 255) / 256, (int64_t)num_sms() * 8));
    k_offer_init<R><<<grid1, 256, 0, s>>>(p);
    k_suitor<R, G, HEAVY, false><<<grid, MATCH_BLOCK, 0, s>>>(p);
    if (HEAVY > 0) k_suitor<R, 32, 0, true><<<num_sms() * 4, MATCH_BLOCK, 0, s>>>(p);
    k_suitor_final<<<grid1, 256, 0, s>>>(p);
    KP_CUDA(cudaGetLastError());
    return KP_OK;
}

template <int R>
kp_status launch_suitor_r(const SuitorParams &p, int G, cudaStream_t s) {
    switch (G) {
    case 1: return launch_suitor_rg<R, 1, 32>(p, s);
    case 4: return launch_suitor_rg<R, 4, 128>(p, s);
    case 8: return launch_suitor_rg<R, 8, 512>(p, s);
    default: return launch_suitor_rg<R, 32, 0>(p, s);
    }
}

// Lanes per proposing node from the level's mean degree.
int suitor_group(double avg) {
    if (avg <= 12.0) return 1;
    if (avg <= 40.0) return 4;
    if (avg <= 160.0) return 8;
    return 32;
}

kp_status launch_suitor(int rating, const SuitorParams &p, int G, cudaStream_t s) {
    switch (rating) {
    case KP_RATING_EXPANSION_STAR2: return launch_suitor_r<KP_RATING_EXPANSION_STAR2>(p, G, s);
    case KP_RATING_INNER_OUTER: return launch_suitor_r<KP_RATING_INNER_OUTER>(p, G, s);
    case KP_RATING_WEIGHT: return launch_suitor_r<KP_RATING_WEIGHT>(p, G, s);
    case KP_RATING_EXPANSION: return launch_suitor_r<KP_RATING_EXPANSION>(p, G, s);
    case KP_RATING_EXPANSION_STAR: return launch_suitor_r<KP_RATING_EXPANSION_STAR>(p, G, s);
    default: return set_error(KP_ERR_UNSUPPORTED, "unknown rating");
    }
}

int group_for_degree(double avg) {
    if (avg <= 3.0) return 4;
    if (avg <= 6.5) return 8;
    if (avg <= 14.0) return 16;
    return 32;
}


// Scratch reused by all levels (sized for level 0).
struct Scratch {
    cudaStream_t s = nullptr;
    std::vector<void *> ptrs;
    int32_t *match = nullptr, *cand = nullptr, *list0 = nullptr, *list1 = nullptr;
    int32_t *first = nullptr, *second = nullptr, *off = nullptr, *degp = nullptr;
    int32_t *outw_a = nullptr, *outw_b = nullptr;
    int32_t *tmp_adj = nullptr, *tmp_w = nullptr, *big_adj = nullptr, *big_w = nullptr;
    int32_t *lists[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    Offer *offer = nullptr;
    uint64_t *partials = nullptr;
    Counters *ctr = nullptr;
    template <class T>
    kp_status get(T **p, int64_t count) {
        KP_TRY(dev_alloc_n(p, count, s));
        ptrs.push_back(*p);
        return KP_OK;
    }
    ~Scratch() {
        for (void *p : ptrs) dev_free(p, s);
    }
};

constexpr int KP_MAX_LEVELS = 128;

struct PinnedCounters {
    Counters *h = nullptr;
    int32_t *nnz = nullptr;
    PinnedCounters() {
        void *p = nullptr;
        if (cudaMallocHost(&p, sizeof(Counters) + sizeof(int32_t) * KP_MAX_LEVELS) != cudaSuccess) p = nullptr;
        h = (Counters *)p;
        nnz = p ? (int32_t *)((char *)p + sizeof(Counters)) : nullptr;
    }
    ~PinnedCounters() {
        if (h) cudaFreeHost(h);
    }
};

}  // namespace

kp_status validate_graph(const kp_graph *g, cudaStream_t s, int64_t spin_limit);

kp_status coarsen_impl(const kp_graph *g, const kp_options *o, cudaStream_t s, kp_hierarchy **out) {
    const int rating = o->rating;
    if (rating < 0 || rating > 4) return set_error(KP_ERR_UNSUPPORTED, "unknown rating");
    if (o->matcher != KP_MATCHER_SUITOR && o->matcher != KP_MATCHER_HANDSHAKE)
        return set_error(KP_ERR_UNSUPPORTED, "unknown matcher");
    if (g->n < 0 || g->nnz < 0) return set_error(KP_ERR_INVALID, "negative graph size");
    if (g->n > 0 && (!g->xadj || !g->vwgt || (g->nnz > 0 && (!g->adjncy || !g->ewgt))))
        return set_error(KP_ERR_INVALID, "null graph array");
    if (o->max_levels < 0 || o->min_shrink_permille < 0 || o->min_shrink_permille > 1000 || o->spin_limit <= 0)
        return set_error(KP_ERR_INVALID, "bad option value");
    if (g_coop_supported < 0) {
        int dev = 0, v = 0;
        KP_CUDA(cudaGetDevice(&dev));
        KP_CUDA(cudaDeviceGetAttribute(&v, cudaDevAttrCooperativeLaunch, dev));
        g_coop_supported = v;
    }
    if (!g_coop_supported) return set_error(KP_ERR_UNSUPPORTED, "device lacks cooperative launch");
    PhaseTimer timer(o->profile != 0, s);
    int32_t launches = 0;
    if (o->validate && g->n > 0) {
        timer.mark(KP_PHASE_VALIDATE);
        KP_TRY(validate_graph(g, s, o->spin_limit));
        timer.mark(-1);
        launches += 1;
    }

    kp_hierarchy *h = new kp_hierarchy();
    h->stream = s;
    KP_CUDA(cudaGetDevice(&h->device));
    kp_level l0;
    l0.n = g->n;
    l0.nnz = g->nnz;
    l0.xadj = const_cast<int32_t *>(g->xadj);
    l0.adjncy = const_cast<int32_t *>(g->adjncy);
    l0.ewgt = const_cast<int32_t *>(g->ewgt);
    l0.vwgt = const_cast<int32_t *>(g->vwgt);
    l0.owned = false;
    h->levels.push_back(l0);

    auto fail = [&](kp_status st) {
        kp_hierarchy_free(h);
        return st;
    };

    const int32_t n0 = g->n;
    const int32_t nnz0 = g->nnz;
    if (n0 == 0) {
        *out = h;
        return KP_OK;
    }
    Scratch sc;
    sc.s = s;
    kp_status st;
#define SC_GET(ptr, cnt)                   st = sc.get(&(ptr), (cnt));            if (st != KP_OK) return fail(st);
    SC_GET(sc.match, n0);
    SC_GET(sc.cand, n0);
    SC_GET(sc.list0, n0);
    SC_GET(sc.list1, n0);
    SC_GET(sc.first, n0);
    SC_GET(sc.second, n0);
    SC_GET(sc.off, (int64_t)n0 + 1);
    SC_GET(sc.degp, n0);
    SC_GET(sc.tmp_adj, nnz0);
    SC_GET(sc.tmp_w, nnz0);
    SC_GET(sc.big_adj, nnz0);
    SC_GET(sc.big_w, nnz0);
    for (int c = 1; c <= 4; c++) SC_GET(sc.lists[c], n0);
    SC_GET(sc.partials, scan_tiles(n0) + 1);
    if (o->matcher == KP_MATCHER_SUITOR) SC_GET(sc.offer, n0);
    SC_GET(sc.ctr, 1);
    if (rating == KP_RATING_INNER_OUTER) {
        SC_GET(sc.outw_a, n0);
        SC_GET(sc.outw_b, n0);
    }
#undef SC_GET
    thread_local PinnedCounters pinned;
    if (!pinned.h) return fail(set_error(KP_ERR_OOM, "pinned host counters"));
    Counters *hc = pinned.h;

    if (rating == KP_RATING_INNER_OUTER) {
        timer.mark(KP_PHASE_OUT);
        const int64_t threads = (int64_t)n0 * 8;
        k_out_weight<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(n0, g->xadj, g->ewgt, sc.outw_a);
        launches += 1;
    }
    int32_t *outw_cur = sc.outw_a, *outw_next = sc.outw_b;
    int32_t total_rounds = 0;
    int64_t total_matched = 0;

    for (;;) {
        kp_level &cur = h->levels.back();
        const int32_t n = cur.n;
        if (n <= o->stop_size || (int32_t)h->levels.size() - 1 >= o->max_levels) break;
        const int lvl_idx = (int)h->levels.size() - 1;
        h->per_level.push_back(kp_level_profile{});
        h->per_level.back().n = n;
        h->per_level.back().nnz = cur.nnz;
        const int32_t launches_before = launches;
        if (cudaMemsetAsync(sc.ctr, 0, sizeof(Counters), s) != cudaSuccess)
            return fail(cuda_error(cudaGetLastError(), "memset counters"));
        if (cudaMemsetAsync(sc.match, 0xff, sizeof(int32_t) * (size_t)n, s) != cudaSuccess)
            return fail(cuda_error(cudaGetLastError(), "memset match"));
        // -- matching (Section 3.3)
        MatchParams mp;
        mp.n = n;
        mp.xadj = cur.xadj;
        mp.adjncy = cur.adjncy;
        mp.ewgt = cur.ewgt;
        mp.vwgt = cur.vwgt;
        mp.outw = outw_cur;
        mp.seed = o->seed;
        mp.match = sc.match;
        mp.cand = sc.cand;
        mp.list0 = sc.list0;
        mp.list1 = sc.list1;
        mp.ctr = sc.ctr;
        mp.spin_limit = o->spin_limit;
        const int G = group_for_degree(n > 0 ? (double)cur.nnz / n : 0.0);
        timer.mark(KP_PHASE_MATCH, lvl_idx);
        if (o->matcher == KP_MATCHER_SUITOR) {
            if (cudaMemsetAsync(&sc.ctr->list_size[0], 0, sizeof(int32_t), s) != cudaSuccess)
                return fail(cuda_error(cudaGetLastError(), "memset parked"));
            SuitorParams sp;
            sp.n = n;
            sp.xadj = cur.xadj;
            sp.adjncy = cur.adjncy;
            sp.ewgt = cur.ewgt;
            sp.vwgt = cur.vwgt;
            sp.outw = outw_cur;
            sp.seed = o->seed;
            sp.offer = sc.offer;
            sp.match = sc.match;
            sp.parked = sc.list0;
            sp.parked_size = &sc.ctr->list_size[0];
            sp.ctr = sc.ctr;
            sp.spin_limit = o->spin_limit;
            const int Gs = suitor_group(n > 0 ? (double)cur.nnz / n : 0.0);
            st = launch_suitor(rating, sp, Gs, s);
            launches += (Gs < 32) ? 4 : 3;
        } else {
            st = launch_match(rating, mp, G, s);
            launches += 1;
        }
        if (st != KP_OK) return fail(st);
        // -- relabel (Section 2: pairs become one node)
        kp_level nxt;
        nxt.owned = true;
        int32_t *cmap = nullptr, *cvw = nullptr;
        st = dev_alloc_n(&cmap, n, s);
        if (st != KP_OK) return fail(st);
        cur.map = cmap;
        h->allocations.push_back(cmap);
        st = dev_alloc_n(&cvw, n, s);
        if (st != KP_OK) return fail(st);
        h->allocations.push_back(cvw);
        RelabelOp rop;
        rop.n = n;
        rop.match = sc.match;
        rop.xadj = cur.xadj;
        rop.vwgt = cur.vwgt;
        rop.map = cmap;
        rop.first = sc.first;
        rop.second = sc.second;
        rop.cvwgt = cvw;
        rop.off = sc.off;
        rop.ctr = sc.ctr;
        timer.mark(KP_PHASE_RELABEL, lvl_idx);
        if (device_scan(rop, n, sc.partials, s) != cudaSuccess)
            return fail(cuda_error(cudaGetLastError(), "relabel scan"));
        timer.mark(-1);
        launches += 3;
        if (cudaMemcpyAsync(hc, sc.ctr, sizeof(Counters), cudaMemcpyDeviceToHost, s) != cudaSuccess)
            return fail(cuda_error(cudaGetLastError(), "read counters"));
        if (cudaStreamSynchronize(s) != cudaSuccess) return fail(cuda_error(cudaGetLastError(), "sync"));
        if (hc->err & ERR_TIMEOUT)
            return fail(set_error(KP_ERR_TIMEOUT, o->matcher == KP_MATCHER_SUITOR
                                                      ? "proposal chain exceeded spin_limit steps"
                                                      : "matching grid barrier timed out"));
        total_rounds += (o->matcher == KP_MATCHER_SUITOR) ? 1 : hc->rounds;
        h->per_level.back().rounds = (o->matcher == KP_MATCHER_SUITOR) ? 1 : hc->rounds;
        h->per_level.back().searches = (int64_t)hc->searches;
        h->per_level.back().failed_cas = (int64_t)hc->failed_cas;
        const int32_t cn = hc->cn;
        const int32_t U = hc->U;
        if (cn == n) {   // nothing matched: this level is not kept
            cur.map = nullptr;
            h->per_level.back().launches = launches - launches_before;
            break;
        }
        total_matched += n - cn;
        // -- contraction (Section 2): merge parallel edges, drop the pair's edge
        nxt.n = cn;
        nxt.vwgt = cvw;
        st = dev_alloc_n(&nxt.xadj, (int64_t)cn + 1, s);
        if (st != KP_OK) return fail(st);
        h->allocations.push_back(nxt.xadj);
        st = dev_alloc_n(&nxt.adjncy, U, s);
        if (st != KP_OK) return fail(st);
        h->allocations.push_back(nxt.adjncy);
        st = dev_alloc_n(&nxt.ewgt, U, s);
        if (st != KP_OK) return fail(st);
        h->allocations.push_back(nxt.ewgt);
        ContractParams cp;
        cp.cn = cn;
        cp.xadj = cur.xadj;
        cp.adjncy = cur.adjncy;
        cp.ewgt = cur.ewgt;
        cp.map = cmap;
        cp.first = sc.first;
        cp.second = sc.second;
        cp.off = sc.off;
        cp.tmp_adj = sc.tmp_adj;
        cp.tmp_w = sc.tmp_w;
        cp.big_adj = sc.big_adj;
        cp.big_w = sc.big_w;
        cp.degp = sc.degp;
        cp.outw = (rating == KP_RATING_INNER_OUTER) ? outw_next : nullptr;
        for (int c = 0; c < 5; c++) cp.lists[c] = sc.lists[c];
        cp.ctr = sc.ctr;
        timer.mark(KP_PHASE_CONTRACT, lvl_idx);
        launches += 5;
        {
            const int64_t want = ((int64_t)cn + CONTRACT_BLOCK - 1) / CONTRACT_BLOCK;
            const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)1 << 30));
            k_contract_small<<<grid, CONTRACT_BLOCK, 0, s>>>(cp);
            // overflow classes: their sizes are only known on the device, so the
            // launches use fixed grids that stride over the lists
            k_contract_warp_list<<<num_sms() * 8, CONTRACT_BLOCK, 0, s>>>(cp);
            k_contract_warp_smem<<<num_sms() * 8, CONTRACT_BLOCK, 0, s>>>(cp);
            k_contract_mid<<<num_sms() * 4, CONTRACT_BLOCK, 0, s>>>(cp);
            int bits = 1;
            while (bits < 31 && ((int64_t)1 << bits) < (int64_t)cn) bits++;
            const int passes = (bits + 7) / 8;
            k_contract_big<<<num_sms(), CONTRACT_BLOCK, 0, s>>>(cp, passes);
        }
        timer.mark(KP_PHASE_CSR, lvl_idx);
        DegScanOp dop;
        dop.cn = cn;
        dop.degp = sc.degp;
        dop.cxadj = nxt.xadj;
        dop.ctr = sc.ctr;
        if (device_scan(dop, cn, sc.partials, s) != cudaSuccess)
            return fail(cuda_error(cudaGetLastError(), "degree scan"));
        {
            const int64_t threads = (int64_t)cn * 8;
            const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((threads + 255) / 256, (int64_t)num_sms() * 16));
            k_compact<<<grid, 256, 0, s>>>(cn, sc.off, sc.degp, nxt.xadj, sc.tmp_adj, sc.tmp_w, nxt.adjncy,
                                           nxt.ewgt);
        }
        timer.mark(-1);
        launches += 4;
        if (cudaGetLastError() != cudaSuccess) return fail(cuda_error(cudaGetLastError(), "contraction"));
        // the coarse entry count reaches the host with the next synchronisation
        const int lvl = (int)h->levels.size();
        if (lvl >= KP_MAX_LEVELS) return fail(set_error(KP_ERR_UNSUPPORTED, "too many levels"));
        if (cudaMemcpyAsync(&pinned.nnz[lvl], &sc.ctr->nnz_out, sizeof(int32_t), cudaMemcpyDeviceToHost, s) !=
            cudaSuccess)
            return fail(cuda_error(cudaGetLastError(), "read nnz"));
        nxt.nnz = U;   // upper bound until the exact count has arrived
        h->per_level.back().launches = launches - launches_before;
        h->levels.push_back(nxt);
        std::swap(outw_cur, outw_next);
        if ((int64_t)cn * 1000 > (int64_t)n * (1000 - o->min_shrink_permille)) break;
    }
    timer.mark(-1);
    h->total_rounds = total_rounds;
    h->total_matched = total_matched;
    if (cudaStreamSynchronize(s) != cudaSuccess) return fail(cuda_error(cudaGetLastError(), "final sync"));
    if (h->per_level.size() > h->levels.size() - 1) h->per_level.resize(h->levels.size() - 1);
    timer.accumulate(&h->total, h->per_level);
    h->total.launches = launches;
    h->total.rounds = total_rounds;
    h->total.n = n0;
    h->total.nnz = nnz0;
    for (const auto &lp : h->per_level) {
        h->total.searches += lp.searches;
        h->total.failed_cas += lp.failed_cas;
    }
    for (size_t l = 1; l < h->levels.size(); l++) h->levels[l].nnz = pinned.nnz[l];
    *out = h;
    return KP_OK;
}

}  // namespace kp
