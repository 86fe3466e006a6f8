/*
 * Oracle for the coarsening / projection / cut-gain path of the multilevel
 * graph partitioner in "Engineering a Scalable High Quality Graph Partitioner"
 * (Holtgrewe, Sanders, Schulz).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is a plain, sequential, deliberately
 * slow CPU statement of what the CUDA path must compute.  It is used by the
 * tests, by the smoke check and by the benchmark's CPU-baseline leg; nothing
 * in the product path may call it.  It shares no code, header or table with
 * the CUDA library.
 *
 * All arithmetic is integer.  Ratings are kept as exact fractions num/den and
 * compared with a continued-fraction expansion (no division of reals, no
 * 128-bit products), so the comparison is exact and independent of the
 * cross-multiplication the CUDA kernels use.
 *
 * Readings taken where the paper is silent:
 *  - ties between equal ratings are broken by a seeded splitmix64 hash of the
 *    edge's endpoints (higher first), then by (lo, hi) lexicographically
 *    smaller first; this makes the edge order strict, and under a strict
 *    order the locally heaviest (handshake) matching of Section 3.3 is unique
 *    and equals the Greedy matching of Section 3.2;
 *  - a rating whose denominator is 0 (c(u)c(v)=0, or innerOuter on an
 *    isolated pair) is +infinity, and two infinities are equal;
 *  - a coarse node's representative is the smaller fine id of its pair, and
 *    coarse ids are the ranks of the representatives in fine-id order.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_INVALID 1
#define OR_OVERFLOW 2
#define OR_NOMEM 3

#define RATING_EXPANSION_STAR2 0
#define RATING_INNER_OUTER 1
#define RATING_WEIGHT 2
#define RATING_EXPANSION 3
#define RATING_EXPANSION_STAR 4

/* ------------------------------------------------------------------------ */
/* Input checks (Section 2: omega > 0, c >= 0, undirected graph).            */
/* ------------------------------------------------------------------------ */

/* Returns OR_OK, OR_INVALID (malformed CSR, asymmetric, unsorted row,
 * self loop, omega <= 0, c < 0) or OR_OVERFLOW (sum c >= 2^31, sum of
 * undirected edge weights >= 2^31, nnz >= nnz_limit: the offset width's
 * range, 2^31 for 32-bit offsets). */
int or_validate(int32_t n, int64_t nnz, int64_t nnz_limit, const int64_t *xadj, const int32_t *adjncy,
                const int32_t *ewgt, const int32_t *vwgt)
{
    if (n < 0 || nnz < 0) return OR_INVALID;
    if (nnz >= nnz_limit) return OR_OVERFLOW;
    if (xadj[0] != 0 || xadj[n] != nnz) return OR_INVALID;
    for (int32_t v = 0; v < n; v++)
        if (xadj[v + 1] < xadj[v]) return OR_INVALID;
    int64_t csum = 0, wsum = 0;
    for (int32_t v = 0; v < n; v++) {
        if (vwgt[v] < 0) return OR_INVALID;
        csum += vwgt[v];
        for (int64_t e = xadj[v]; e < xadj[v + 1]; e++) {
            int32_t u = adjncy[e];
            if (u < 0 || u >= n || u == v) return OR_INVALID;
            if (ewgt[e] <= 0) return OR_INVALID;
            if (e > xadj[v] && adjncy[e - 1] >= u) return OR_INVALID;
            /* the reverse entry (u, v) must exist with the same weight */
            int64_t lo = xadj[u], hi = xadj[u + 1] - 1, found = -1;
            while (lo <= hi) {
                int64_t mid = lo + (hi - lo) / 2;
                if (adjncy[mid] == v) { found = mid; break; }
                if (adjncy[mid] < v) lo = mid + 1; else hi = mid - 1;
            }
            if (found < 0 || ewgt[found] != ewgt[e]) return OR_INVALID;
            if (u > v) wsum += ewgt[e];
        }
    }
    if (csum >= ((int64_t)1 << 31) || wsum >= ((int64_t)1 << 31)) return OR_OVERFLOW;
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Edge ratings (Section 3.1).                                               */
/* ------------------------------------------------------------------------ */

/* Out(v) = sum of omega({v,x}) over the neighbours x of v (Section 3.1). */
void or_out_weight(int32_t n, const int64_t *xadj, const int32_t *ewgt, int64_t *out)
{
    for (int32_t v = 0; v < n; v++) {
        int64_t s = 0;
        for (int64_t e = xadj[v]; e < xadj[v + 1]; e++) s += ewgt[e];
        out[v] = s;
    }
}

/* The rating of edge {u,v} as the fraction num/den (Section 3.1):
 *   weight       omega
 *   expansion    omega / (c(u) + c(v))
 *   expansion*   omega / (c(u) c(v))
 *   expansion*2  omega^2 / (c(u) c(v))
 *   innerOuter   omega / (Out(u) + Out(v) - 2 omega)            */
void or_rating(int rating, int64_t w, int64_t cu, int64_t cv, int64_t outu, int64_t outv,
               uint64_t *num, uint64_t *den)
{
    switch (rating) {
    case RATING_WEIGHT:         *num = (uint64_t)w;     *den = 1; break;
    case RATING_EXPANSION:      *num = (uint64_t)w;     *den = (uint64_t)(cu + cv); break;
    case RATING_EXPANSION_STAR: *num = (uint64_t)w;     *den = (uint64_t)cu * (uint64_t)cv; break;
    case RATING_INNER_OUTER:    *num = (uint64_t)w;     *den = (uint64_t)(outu + outv - 2 * w); break;
    default:                    *num = (uint64_t)w * (uint64_t)w; *den = (uint64_t)cu * (uint64_t)cv; break;
    }
}

/* Exact comparison of a/b with c/d for nonnegative integers, numerators > 0;
 * a zero denominator means +infinity.  Returns +1, 0, -1.
 * Method: compare the continued-fraction expansions term by term.  With
 * a/b = q1 + r1/b and c/d = q2 + r2/d, unequal integer parts decide; with
 * equal ones the order of r1/b and r2/d is the reverse of the order of their
 * reciprocals b/r1 and d/r2, which is compared the same way.               */
int or_frac_cmp(uint64_t a, uint64_t b, uint64_t c, uint64_t d)
{
    if (b == 0 && d == 0) return 0;
    if (b == 0) return 1;
    if (d == 0) return -1;
    for (;;) {
        uint64_t q1 = a / b, r1 = a % b, q2 = c / d, r2 = c % d;
        if (q1 != q2) return q1 > q2 ? 1 : -1;
        if (r1 == 0 && r2 == 0) return 0;
        if (r1 == 0) return -1;
        if (r2 == 0) return 1;
        /* r1/b > r2/d  <=>  d/r2 > b/r1: continue with (d/r2, b/r1) */
        uint64_t na = d, nb = r2, nc = b, nd = r1;
        a = na; b = nb; c = nc; d = nd;
    }
}

/* splitmix64 output function (Steele, Lea, Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014): the state x is advanced by
 * the golden-ratio increment and then mixed. */
uint64_t or_splitmix64(uint64_t x)
{
    uint64_t z = x + 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

/* Tie-break hash of the undirected edge {u,v}: symmetric in u and v. */
uint64_t or_edge_hash(uint64_t seed, int32_t u, int32_t v)
{
    uint64_t lo = (uint64_t)(uint32_t)(u < v ? u : v);
    uint64_t hi = (uint64_t)(uint32_t)(u < v ? v : u);
    return or_splitmix64(seed ^ ((lo << 32) | hi));
}

/* One undirected edge with everything the strict order looks at. */
typedef struct {
    uint64_t num, den, h;
    int32_t lo, hi, w;
} or_edge;

/* Strict total order on edges: +1 if x comes before y (is "heavier"). */
static int or_edge_better(const or_edge *x, const or_edge *y)
{
    int r = or_frac_cmp(x->num, x->den, y->num, y->den);
    if (r != 0) return r;
    if (x->h != y->h) return x->h > y->h ? 1 : -1;
    if (x->lo != y->lo) return x->lo < y->lo ? 1 : -1;
    if (x->hi != y->hi) return x->hi < y->hi ? 1 : -1;
    return 0;
}

static void or_make_edge(or_edge *e, int rating, uint64_t seed, int32_t u, int32_t v, int32_t w,
                         const int32_t *vwgt, const int64_t *out)
{
    e->lo = u < v ? u : v;
    e->hi = u < v ? v : u;
    e->w = w;
    or_rating(rating, w, vwgt[u], vwgt[v], out ? out[u] : 0, out ? out[v] : 0, &e->num, &e->den);
    e->h = or_edge_hash(seed, u, v);
}

/* Exposed for tests: order of edges {u1,v1} (weight w1) and {u2,v2}. */
int or_edge_order(int rating, uint64_t seed, const int32_t *vwgt, const int64_t *out,
                  int32_t u1, int32_t v1, int32_t w1, int32_t u2, int32_t v2, int32_t w2)
{
    or_edge a, b;
    or_make_edge(&a, rating, seed, u1, v1, w1, vwgt, out);
    or_make_edge(&b, rating, seed, u2, v2, w2, vwgt, out);
    return or_edge_better(&a, &b);
}

static int or_cmp_desc(const void *pa, const void *pb)
{
    return -or_edge_better((const or_edge *)pa, (const or_edge *)pb);
}

/* ------------------------------------------------------------------------ */
/* Matching (Sections 2, 3.2, 3.3).                                          */
/* ------------------------------------------------------------------------ */

/* Greedy matching (Section 3.2): scan the edges from heaviest to lightest
 * under the strict order and take an edge when both ends are still free.
 * match[v] = partner, or v when v stays unmatched.  Returns |M|, or -1.   */
int64_t or_greedy_matching(int32_t n, const int64_t *xadj, const int32_t *adjncy,
                           const int32_t *ewgt, const int32_t *vwgt, int rating,
                           uint64_t seed, int32_t *match)
{
    int64_t m = xadj[n] / 2;
    or_edge *edges = (or_edge *)malloc(sizeof(or_edge) * (size_t)(m > 0 ? m : 1));
    int64_t *out = NULL;
    if (!edges) return -1;
    if (rating == RATING_INNER_OUTER) {
        out = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
        if (!out) { free(edges); return -1; }
        or_out_weight(n, xadj, ewgt, out);
    }
    int64_t k = 0;
    for (int32_t v = 0; v < n; v++)
        for (int64_t e = xadj[v]; e < xadj[v + 1]; e++)
            if (adjncy[e] > v)
                or_make_edge(&edges[k++], rating, seed, v, adjncy[e], ewgt[e], vwgt, out);
    qsort(edges, (size_t)k, sizeof(or_edge), or_cmp_desc);
    for (int32_t v = 0; v < n; v++) match[v] = v;
    int64_t size = 0;
    for (int64_t i = 0; i < k; i++) {
        int32_t a = edges[i].lo, b = edges[i].hi;
        if (match[a] == a && match[b] == b) {
            match[a] = b;
            match[b] = a;
            size++;
        }
    }
    free(edges);
    free(out);
    return size;
}

/* Handshake matching (Section 3.3), simulated round by round: in every round
 * each free node that has a free neighbour picks the heaviest edge to a free
 * neighbour; edges picked from both ends are matched; rounds repeat until no
 * edge has two free ends.  cand1 (optional) receives the first round's picks
 * (-1 for a node with no neighbour).  Returns |M|, or -1 on allocation
 * failure; *rounds receives the number of rounds that matched something. */
int64_t or_handshake_matching(int32_t n, const int64_t *xadj, const int32_t *adjncy,
                              const int32_t *ewgt, const int32_t *vwgt, int rating,
                              uint64_t seed, int32_t *match, int32_t *rounds, int32_t *cand1)
{
    int32_t *cand = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int64_t *out = NULL;
    if (!cand) return -1;
    if (rating == RATING_INNER_OUTER) {
        out = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
        if (!out) { free(cand); return -1; }
        or_out_weight(n, xadj, ewgt, out);
    }
    for (int32_t v = 0; v < n; v++) match[v] = -1;   /* -1 = free */
    int64_t size = 0;
    int32_t r = 0;
    for (;;) {
        int any_pick = 0;
        for (int32_t v = 0; v < n; v++) {
            cand[v] = -1;
            if (match[v] != -1) continue;
            or_edge best, cur;
            for (int64_t e = xadj[v]; e < xadj[v + 1]; e++) {
                int32_t u = adjncy[e];
                if (match[u] != -1) continue;
                or_make_edge(&cur, rating, seed, v, u, ewgt[e], vwgt, out);
                if (cand[v] == -1 || or_edge_better(&cur, &best) > 0) {
                    best = cur;
                    cand[v] = u;
                }
            }
            if (cand[v] != -1) any_pick = 1;
        }
        if (r == 0 && cand1) memcpy(cand1, cand, sizeof(int32_t) * (size_t)n);
        if (!any_pick) break;
        int64_t matched_now = 0;
        for (int32_t v = 0; v < n; v++) {
            int32_t u = cand[v];
            if (u != -1 && cand[u] == v && v < u) {
                match[v] = u;
                match[u] = v;
                matched_now++;
            }
        }
        size += matched_now;
        r++;
    }
    for (int32_t v = 0; v < n; v++)
        if (match[v] == -1) match[v] = v;
    if (rounds) *rounds = r;
    free(cand);
    free(out);
    return size;
}

/* The rating of edge {u,v} as a real number for the dynamic programme of
 * the Global Path Algorithm: the fraction num/den of or_rating evaluated in
 * IEEE double (num and den converted with rounding to nearest, then one
 * correctly rounded division; a zero denominator gives +infinity). */
static double or_rating_real(const or_edge *e)
{
    return (double)e->num / (double)e->den;
}

/* One maximum weight matching of a path x_0 - x_1 - ... - x_L with edge
 * weights w[1..L] (w[i] joins x_{i-1} and x_i), by dynamic programming:
 * best[i] = max(best[i-1], best[i-2] + w[i]), taking edge i only when that
 * is strictly larger.  The matched pairs are written into match[]; returns
 * best[L].  best[] and take[] are scratch of L+1 entries. */
static double or_path_dp(int32_t L, const int32_t *x, const double *w, double *best, char *take,
                         int32_t *match)
{
    best[0] = 0.0;
    take[0] = 0;
    for (int32_t i = 1; i <= L; i++) {
        double with = (i >= 2 ? best[i - 2] : 0.0) + w[i];
        take[i] = with > best[i - 1];
        best[i] = take[i] ? with : best[i - 1];
    }
    for (int32_t i = L; i >= 1;) {
        if (take[i]) {
            match[x[i - 1]] = x[i];
            match[x[i]] = x[i - 1];
            i -= 2;
        } else {
            i -= 1;
        }
    }
    return best[L];
}

/* Global Path Algorithm (Section 3.2, after Maue and Sanders).
 * Phase 1 scans the edges from heaviest to lightest under the strict order
 * and collects a set of paths and even cycles: an edge is taken when both
 * ends have fewer than two collected edges, unless its ends are the two ends
 * of one path with an even number of edges (taking it would close an odd
 * cycle).  Joining the two ends of a path with an odd number of edges closes
 * an even cycle; that edge, the last one of its cycle, is the cycle's
 * closing edge.
 * Phase 2 computes a maximum weight matching of every path and every cycle
 * by dynamic programming over the ratings (or_rating_real):
 *  - a path is walked from its end with the smaller id;
 *  - a cycle with closing edge {a,b}, a < b, is walked from a along its
 *    other edges to b, giving the path x_0 = a, ..., x_{k-1} = b; the cycle's
 *    matching is the better of that path's matching and the closing edge
 *    plus the matching of x_1 .. x_{k-2}, the closing edge only when strictly
 *    better.
 * match[v] = partner, or v when v stays unmatched; nbr2 (may be NULL)
 * receives the two collected neighbours of every node (-1 where fewer).
 * Returns |M|, or -1 on allocation failure. */
int64_t or_gpa_matching(int32_t n, const int64_t *xadj, const int32_t *adjncy,
                        const int32_t *ewgt, const int32_t *vwgt, int rating,
                        uint64_t seed, int32_t *match, int32_t *nbr2)
{
    int64_t m = xadj[n] / 2;
    size_t nn = (size_t)(n > 0 ? n : 1);
    or_edge *edges = (or_edge *)malloc(sizeof(or_edge) * (size_t)(m > 0 ? m : 1));
    int64_t *out = NULL;
    int32_t *nb = (int32_t *)malloc(sizeof(int32_t) * 2 * nn);      /* collected neighbours */
    double *nw = (double *)malloc(sizeof(double) * 2 * nn);         /* their ratings */
    int32_t *parent = (int32_t *)malloc(sizeof(int32_t) * nn);     /* union-find over paths */
    int64_t *len = (int64_t *)malloc(sizeof(int64_t) * nn);        /* edges of a root's path */
    int32_t *closing = (int32_t *)malloc(sizeof(int32_t) * nn);    /* a cycle's closing edge: other end */
    int32_t *x = (int32_t *)malloc(sizeof(int32_t) * (nn + 1));
    double *w = (double *)malloc(sizeof(double) * (nn + 1));
    double *best = (double *)malloc(sizeof(double) * (nn + 1));
    char *take = (char *)malloc(nn + 1);
    char *seen = (char *)calloc(nn, 1);
    int64_t result = -1;
    if (!edges || !nb || !nw || !parent || !len || !closing || !x || !w || !best || !take || !seen) goto done;
    if (rating == RATING_INNER_OUTER) {
        out = (int64_t *)malloc(sizeof(int64_t) * nn);
        if (!out) goto done;
        or_out_weight(n, xadj, ewgt, out);
    }
    int64_t k = 0;
    for (int32_t v = 0; v < n; v++)
        for (int64_t e = xadj[v]; e < xadj[v + 1]; e++)
            if (adjncy[e] > v)
                or_make_edge(&edges[k++], rating, seed, v, adjncy[e], ewgt[e], vwgt, out);
    qsort(edges, (size_t)k, sizeof(or_edge), or_cmp_desc);
    for (int32_t v = 0; v < n; v++) {
        nb[2 * v] = nb[2 * v + 1] = -1;
        parent[v] = v;
        len[v] = 0;
        closing[v] = -1;
        match[v] = v;
    }
    /* phase 1: paths and even cycles */
    for (int64_t i = 0; i < k; i++) {
        int32_t a = edges[i].lo, b = edges[i].hi;
        if (nb[2 * a + 1] >= 0 || nb[2 * b + 1] >= 0) continue;   /* an end has two edges */
        int32_t ra = a, rb = b;   /* the paths' roots (path halving on the way) */
        while (parent[ra] != ra) { parent[ra] = parent[parent[ra]]; ra = parent[ra]; }
        while (parent[rb] != rb) { parent[rb] = parent[parent[rb]]; rb = parent[rb]; }
        if (ra == rb && len[ra] % 2 == 0) continue;               /* would close an odd cycle */
        double r = or_rating_real(&edges[i]);
        nb[2 * a + (nb[2 * a] >= 0)] = b;
        nw[2 * a + (nb[2 * a + 1] == b)] = r;
        nb[2 * b + (nb[2 * b] >= 0)] = a;
        nw[2 * b + (nb[2 * b + 1] == a)] = r;
        if (ra == rb) {
            len[ra] += 1;
            closing[a] = b;
            closing[b] = a;
        } else {
            parent[rb] = ra;
            len[ra] += len[rb] + 1;
        }
    }
    /* phase 2a: paths, each from its end with the smaller id */
    for (int32_t v = 0; v < n; v++) {
        if (seen[v] || nb[2 * v] < 0 || nb[2 * v + 1] >= 0) continue;   /* not an unseen path end */
        int32_t L = 0, prev = -1, cur = v;
        x[0] = v;
        seen[v] = 1;
        for (;;) {
            int32_t s = nb[2 * cur] == prev ? 1 : 0;
            int32_t nxt = nb[2 * cur + s];
            if (nxt < 0) break;
            w[++L] = nw[2 * cur + s];
            x[L] = nxt;
            seen[nxt] = 1;
            prev = cur;
            cur = nxt;
        }
        or_path_dp(L, x, w, best, take, match);
    }
    /* phase 2b: cycles, each cut at its closing edge {a,b}, a < b */
    for (int32_t a = 0; a < n; a++) {
        int32_t b = closing[a];
        if (b < a || seen[a]) continue;
        int32_t K = 0, prev = b, cur = a;   /* leave a by its edge that is not {a,b} */
        x[0] = a;
        seen[a] = 1;
        while (cur != b) {
            int32_t s = nb[2 * cur] == prev ? 1 : 0;
            int32_t nxt = nb[2 * cur + s];
            w[++K] = nw[2 * cur + s];
            x[K] = nxt;
            seen[nxt] = 1;
            prev = cur;
            cur = nxt;
        }
        /* x_0 = a .. x_K = b along the path; the closing edge joins x_K, x_0 */
        double wc = nw[2 * a + (nb[2 * a + 1] == b)];
        int32_t *keep = (int32_t *)malloc(sizeof(int32_t) * (size_t)(K + 1));
        if (!keep) goto done;
        for (int32_t i = 0; i <= K; i++) keep[i] = match[x[i]];
        double without = or_path_dp(K, x, w, best, take, match);
        for (int32_t i = 0; i <= K; i++) match[x[i]] = keep[i];   /* undo, then try with {a,b} */
        double with = wc + (K >= 3 ? or_path_dp(K - 2, x + 1, w + 1, best, take, match) : 0.0);
        if (with > without) {
            match[a] = b;
            match[b] = a;
        } else {
            for (int32_t i = 0; i <= K; i++) match[x[i]] = keep[i];
            or_path_dp(K, x, w, best, take, match);
        }
        free(keep);
    }
    if (nbr2)
        for (int32_t v = 0; v < 2 * n; v++) nbr2[v] = nb[v];
    result = 0;
    for (int32_t v = 0; v < n; v++)
        if (match[v] > v) result++;
done:
    free(edges); free(out); free(nb); free(nw); free(parent); free(len); free(closing);
    free(x); free(w); free(best); free(take); free(seen);
    return result;
}

/* Checks that match[] is the Greedy matching of the graph under the strict
 * order, using a characterisation that needs no sort: a matching M is the
 * Greedy matching iff every edge e not in M touches an edge of M that comes
 * before e in the order.  (Induction over the order: the first edge not in M
 * with no such neighbour would have been taken by Greedy.)
 * Returns -1 if match[] passes, else the smallest node at which a check fails
 * (asymmetric match, matched non-edge, or an undominated non-matching edge). */
int64_t or_check_greedy_matching(int32_t n, const int64_t *xadj, const int32_t *adjncy,
                                 const int32_t *ewgt, const int32_t *vwgt, int rating,
                                 uint64_t seed, const int32_t *match)
{
    int64_t *out = NULL;
    if (rating == RATING_INNER_OUTER) {
        out = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
        if (!out) return -2;
        or_out_weight(n, xadj, ewgt, out);
    }
    /* the matched edge at each node, as an or_edge; weight looked up in CSR */
    or_edge *medge = (or_edge *)malloc(sizeof(or_edge) * (size_t)(n > 0 ? n : 1));
    if (!medge) { free(out); return -2; }
    int64_t bad = -1;
    for (int32_t v = 0; v < n && bad < 0; v++) {
        int32_t p = match[v];
        if (p < 0 || p >= n || match[p] != v) { bad = v; break; }
        if (p == v) continue;
        int32_t w = -1;
        for (int64_t e = xadj[v]; e < xadj[v + 1]; e++)
            if (adjncy[e] == p) w = ewgt[e];
        if (w < 0) { bad = v; break; }
        or_make_edge(&medge[v], rating, seed, v, p, w, vwgt, out);
    }
    for (int32_t v = 0; v < n && bad < 0; v++) {
        for (int64_t e = xadj[v]; e < xadj[v + 1]; e++) {
            int32_t u = adjncy[e];
            if (match[v] == u) continue;
            or_edge cur;
            or_make_edge(&cur, rating, seed, v, u, ewgt[e], vwgt, out);
            int dominated = 0;
            if (match[v] != v && or_edge_better(&medge[v], &cur) > 0) dominated = 1;
            if (match[u] != u && or_edge_better(&medge[u], &cur) > 0) dominated = 1;
            if (!dominated) { bad = v; break; }
        }
    }
    free(medge);
    free(out);
    return bad;
}

/* The same characterisation checked only at the listed nodes (graphs too
 * large for a whole pass): v's match is symmetric and an edge, and every edge
 * of v outside M is dominated by the matched edge of v or of its other end.
 * The matched edge of a node is looked up when needed (no n-sized table);
 * Out (innerOuter) is computed for the whole graph.  Returns -1 if every
 * listed node passes, else the first listed node that fails. */
static int or_matched_edge(const int64_t *xadj, const int32_t *adjncy, const int32_t *ewgt,
                           const int32_t *vwgt, const int64_t *out, int rating, uint64_t seed,
                           int32_t n, const int32_t *match, int32_t v, or_edge *me)
{
    int32_t p = match[v];
    if (p < 0 || p >= n || match[p] != v) return -1;
    if (p == v) return 0;
    int32_t w = -1;
    for (int64_t e = xadj[v]; e < xadj[v + 1]; e++)
        if (adjncy[e] == p) w = ewgt[e];
    if (w < 0) return -1;
    or_make_edge(me, rating, seed, v, p, w, vwgt, out);
    return 1;
}

int64_t or_check_greedy_matching_at(int32_t n, const int64_t *xadj, const int32_t *adjncy,
                                    const int32_t *ewgt, const int32_t *vwgt, int rating,
                                    uint64_t seed, const int32_t *match, int64_t count,
                                    const int32_t *nodes)
{
    int64_t *out = NULL;
    if (rating == RATING_INNER_OUTER) {
        out = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
        if (!out) return -2;
        or_out_weight(n, xadj, ewgt, out);
    }
    int64_t bad = -1;
    for (int64_t i = 0; i < count && bad < 0; i++) {
        int32_t v = nodes[i];
        if (v < 0 || v >= n) { bad = v; break; }
        or_edge mv;
        int hv = or_matched_edge(xadj, adjncy, ewgt, vwgt, out, rating, seed, n, match, v, &mv);
        if (hv < 0) { bad = v; break; }
        for (int64_t e = xadj[v]; e < xadj[v + 1]; e++) {
            int32_t u = adjncy[e];
            if (match[v] == u) continue;
            or_edge cur, mu;
            or_make_edge(&cur, rating, seed, v, u, ewgt[e], vwgt, out);
            int hu = or_matched_edge(xadj, adjncy, ewgt, vwgt, out, rating, seed, n, match, u, &mu);
            if (hu < 0) { bad = v; break; }
            int dominated = 0;
            if (hv > 0 && or_edge_better(&mv, &cur) > 0) dominated = 1;
            if (hu > 0 && or_edge_better(&mu, &cur) > 0) dominated = 1;
            if (!dominated) { bad = v; break; }
        }
    }
    free(out);
    return bad;
}

/* ------------------------------------------------------------------------ */
/* Contraction (Section 2).                                                  */
/* ------------------------------------------------------------------------ */

typedef struct { int32_t t, w; } or_entry;

static int or_cmp_target(const void *pa, const void *pb)
{
    const or_entry *a = (const or_entry *)pa, *b = (const or_entry *)pb;
    return (a->t > b->t) - (a->t < b->t);
}

/* Contracts every matched edge {u,v} into one node x with c(x) = c(u)+c(v);
 * parallel edges {x,w} are merged into one with the summed weight, and the
 * contracted edge itself disappears (Section 2).  The representative of x is
 * min(u,v) and x's id is the rank of its representative among all
 * representatives in fine-id order; rows of the coarse CSR are sorted.
 * Outputs (caller-allocated, sizes <= the fine ones): map[n], cxadj[cn+1],
 * cadjncy/cewgt[cnnz], cvwgt[cn].  Returns cn, or -1 on allocation failure;
 * *cnnz receives the coarse entry count. */
int32_t or_contract(int32_t n, const int64_t *xadj, const int32_t *adjncy, const int32_t *ewgt,
                    const int32_t *vwgt, const int32_t *match, int32_t *map, int64_t *cnnz,
                    int64_t *cxadj, int32_t *cadjncy, int32_t *cewgt, int32_t *cvwgt)
{
    /* coarse ids: rank of the representative in fine-id order */
    int32_t cn = 0;
    for (int32_t v = 0; v < n; v++) {
        int32_t rep = match[v] < v ? match[v] : v;
        if (rep == v) map[v] = cn++;
    }
    for (int32_t v = 0; v < n; v++) {
        int32_t rep = match[v] < v ? match[v] : v;
        map[v] = map[rep];
    }
    /* members of every coarse node, in fine-id order */
    int32_t *first = (int32_t *)malloc(sizeof(int32_t) * (size_t)(cn > 0 ? cn : 1));
    int32_t *second = (int32_t *)malloc(sizeof(int32_t) * (size_t)(cn > 0 ? cn : 1));
    int32_t maxdeg = 0;
    for (int32_t v = 0; v < n; v++)
        if (xadj[v + 1] - xadj[v] > maxdeg) maxdeg = (int32_t)(xadj[v + 1] - xadj[v]);
    or_entry *buf = (or_entry *)malloc(sizeof(or_entry) * (size_t)(2 * maxdeg + 1));
    if (!first || !second || !buf) { free(first); free(second); free(buf); return -1; }
    for (int32_t v = 0; v < n; v++) {
        int32_t rep = match[v] < v ? match[v] : v;
        if (rep == v) { first[map[v]] = v; second[map[v]] = (match[v] != v) ? match[v] : -1; }
    }
    int64_t pos = 0;
    cxadj[0] = 0;
    for (int32_t x = 0; x < cn; x++) {
        int32_t mem[2] = { first[x], second[x] };
        int32_t len = 0;
        int64_t c = 0;
        for (int i = 0; i < 2; i++) {
            int32_t v = mem[i];
            if (v < 0) continue;
            c += vwgt[v];
            for (int64_t e = xadj[v]; e < xadj[v + 1]; e++) {
                int32_t t = map[adjncy[e]];
                if (t == x) continue;            /* the contracted edge */
                buf[len].t = t;
                buf[len].w = ewgt[e];
                len++;
            }
        }
        cvwgt[x] = (int32_t)c;
        qsort(buf, (size_t)len, sizeof(or_entry), or_cmp_target);
        for (int32_t i = 0; i < len;) {
            int32_t j = i;
            int64_t w = 0;
            while (j < len && buf[j].t == buf[i].t) { w += buf[j].w; j++; }
            cadjncy[pos] = buf[i].t;
            cewgt[pos] = (int32_t)w;
            pos++;
            i = j;
        }
        cxadj[x + 1] = pos;
    }
    *cnnz = pos;
    free(first);
    free(second);
    free(buf);
    return cn;
}

/* One coarse node x of the contraction, from its members a and b (b = -1:
 * x has one member) and the map of every fine node: the images of the
 * members' neighbours other than x itself, equal images merged with summed
 * weights, in ascending order; *c = c(a) + c(b) (Section 2).  cadjncy and
 * cewgt hold deg(a) + deg(b) entries.  Returns the row's length, or -1 on
 * allocation failure. */
int32_t or_coarse_row(const int64_t *xadj, const int32_t *adjncy, const int32_t *ewgt, const int32_t *vwgt,
                      const int32_t *map, int32_t x, int32_t a, int32_t b, int32_t *cadjncy, int32_t *cewgt,
                      int64_t *c)
{
    int32_t mem[2] = { a, b };
    int64_t cap = (xadj[a + 1] - xadj[a]) + (b >= 0 ? xadj[b + 1] - xadj[b] : 0);
    or_entry *buf = (or_entry *)malloc(sizeof(or_entry) * (size_t)(cap > 0 ? cap : 1));
    if (!buf) return -1;
    int32_t len = 0;
    *c = 0;
    for (int i = 0; i < 2; i++) {
        int32_t v = mem[i];
        if (v < 0) continue;
        *c += vwgt[v];
        for (int64_t e = xadj[v]; e < xadj[v + 1]; e++) {
            int32_t t = map[adjncy[e]];
            if (t == x) continue;
            buf[len].t = t;
            buf[len].w = ewgt[e];
            len++;
        }
    }
    qsort(buf, (size_t)len, sizeof(or_entry), or_cmp_target);
    int32_t k = 0;
    for (int32_t i = 0; i < len;) {
        int32_t j = i;
        int64_t w = 0;
        while (j < len && buf[j].t == buf[i].t) { w += buf[j].w; j++; }
        cadjncy[k] = buf[i].t;
        cewgt[k] = (int32_t)w;
        k++;
        i = j;
    }
    free(buf);
    return k;
}

/* ------------------------------------------------------------------------ */
/* Projection (Section 2, uncontraction) and cut / gain (Sections 2, 5.2).   */
/* ------------------------------------------------------------------------ */

/* Uncontraction of one level: the fine node v joins the block of the coarse
 * node it was contracted into. */
void or_project_level(int32_t n_fine, const int32_t *map, const int32_t *coarse_part,
                      int32_t *fine_part)
{
    for (int32_t v = 0; v < n_fine; v++) fine_part[v] = coarse_part[map[v]];
}

/* Cut, block weights and per-node FM gain of a k-way partition.
 *   cut        sum over blocks i<j of omega(E_ij)            (Section 2)
 *   block_w[b] c(V_b)                                         (Section 2)
 *   gain[v]    decrease of the cut when v moves to block target[v]
 *              (Section 5.2); with k > 2 the target is the adjacent block
 *              with the largest connection (smallest id on ties); a node with
 *              no neighbour in another block gets target -1 and gain -int(v).
 * Returns OR_OK, or OR_INVALID if a block id is outside [0,k). */
int or_cut_gain(int32_t n, const int64_t *xadj, const int32_t *adjncy, const int32_t *ewgt,
                const int32_t *vwgt, const int32_t *part, int32_t k, int64_t *cut,
                int64_t *block_w, int64_t *gain, int32_t *target)
{
    if (k < 1) return OR_INVALID;
    for (int32_t v = 0; v < n; v++)
        if (part[v] < 0 || part[v] >= k) return OR_INVALID;
    for (int32_t b = 0; b < k; b++) block_w[b] = 0;
    for (int32_t v = 0; v < n; v++) block_w[part[v]] += vwgt[v];
    int64_t c = 0;
    for (int32_t v = 0; v < n; v++)
        for (int64_t e = xadj[v]; e < xadj[v + 1]; e++)
            if (adjncy[e] > v && part[adjncy[e]] != part[v]) c += ewgt[e];
    *cut = c;
    int64_t *conn = (int64_t *)calloc((size_t)k, sizeof(int64_t));
    if (!conn) return OR_NOMEM;
    for (int32_t v = 0; v < n; v++) {
        for (int64_t e = xadj[v]; e < xadj[v + 1]; e++) conn[part[adjncy[e]]] += ewgt[e];
        int64_t internal = conn[part[v]];
        int32_t best = -1;
        for (int64_t e = xadj[v]; e < xadj[v + 1]; e++) {
            int32_t b = part[adjncy[e]];
            if (b == part[v]) continue;
            if (best == -1 || conn[b] > conn[best] || (conn[b] == conn[best] && b < best)) best = b;
        }
        target[v] = best;
        gain[v] = (best == -1 ? 0 : conn[best]) - internal;
        for (int64_t e = xadj[v]; e < xadj[v + 1]; e++) conn[part[adjncy[e]]] = 0;
    }
    free(conn);
    return OR_OK;
}
