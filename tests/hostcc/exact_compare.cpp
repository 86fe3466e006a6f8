// Runs the library's exact rating comparison, tie-break hash and strict edge
// order (paper_0910_2004_gb300/csrc/kp_internal.cuh, engine.cuh) on the
// host, one query per input line:
//   c a b d e  -> cmp_frac(a, b, d, e) (-1, 0 or 1)
//   s x        -> splitmix64(x)
//   h seed u v -> edge_hash(seed, u, v)
//   b R seed v u1 w1 u2 w2 av a1 a2 -> better() of the candidates {v,u1}
//                 and {v,u2} of node v under rating R (av, a1, a2: the rating
//                 attribute of v, u1, u2), both ways round: "x y"
//   e R seed cur v w s ws acur as av -> eligible_at(): whether cur (attribute
//                 acur) may offer the edge {cur,v} of weight w to v, whose
//                 record holds suitor s (-1: none) over an edge of weight ws,
//                 s's attribute as and v's own av (paper_0910_2004_gb300/csrc/match.cuh)
//   g R seed x1 y1 w1 ax1 ay1 x2 y2 w2 ax2 ay2 -> gedge_before() of the edges
//                 {x1,y1} and {x2,y2} (the Global Path Algorithm's order,
//                 paper_0910_2004_gb300/csrc/gpa.cuh), both ways round: "x y"
// Built with g++ and the stand-ins of cuda_stubs.h by tests/test_exact_compare_host.py.
#include <cstdio>

#include "gpa.cuh"
#include "match.cuh"

namespace {

template <int R>
kp::Cand cand(uint64_t seed, int32_t v, int32_t u, int32_t w, int32_t av, int32_t au) {
    kp::Cand c;
    kp::rating_ab<R>(w, av, au, c.num, c.den);
    c.h = kp::edge_hash(seed, v, u);
    c.u = u;
    return c;
}

template <int R>
void eligible(uint64_t seed, int32_t cur, int32_t v, int32_t w, int32_t s, int32_t ws, int32_t acur, int32_t as,
              int32_t av) {
    kp::HashCtx hc;
    hc.seed = seed;
    hc.base = 0;
    kp::Offer so;
    so.s = s;
    so.w = ws;
    so.as = as;
    so.au = av;
    kp::Cand cd;
    printf("%d\n", (int)kp::eligible_at<R>(hc, cur, acur, v, w, so, cd));
}

template <int R>
kp::GEdge gedge(uint64_t seed, int32_t x, int32_t y, int32_t w, int32_t ax, int32_t ay) {
    kp::GEdge g;
    kp::rating_ab<R>(w, ax, ay, g.num, g.den);
    g.h = kp::edge_hash(seed, x, y);
    g.lo = x < y ? x : y;
    g.hi = x < y ? y : x;
    return g;
}

template <int R>
void gorder(uint64_t seed, const int32_t *e) {
    const kp::GEdge a = gedge<R>(seed, e[0], e[1], e[2], e[3], e[4]), b = gedge<R>(seed, e[5], e[6], e[7], e[8], e[9]);
    printf("%d %d\n", (int)kp::gedge_before(a, b), (int)kp::gedge_before(b, a));
}

template <int R>
void order(uint64_t seed, int32_t v, int32_t u1, int32_t w1, int32_t u2, int32_t w2, int32_t av, int32_t a1,
           int32_t a2) {
    const kp::Cand x = cand<R>(seed, v, u1, w1, av, a1), y = cand<R>(seed, v, u2, w2, av, a2);
    printf("%d %d\n", (int)kp::better(x, y, v), (int)kp::better(y, x, v));
}

}  // namespace

int main() {
    char op[4];
    while (scanf("%3s", op) == 1) {
        if (op[0] == 'c') {
            unsigned long long a, b, c, d;
            if (scanf("%llu %llu %llu %llu", &a, &b, &c, &d) != 4) return 2;
            printf("%d\n", kp::cmp_frac(a, b, c, d));
        } else if (op[0] == 's') {
            unsigned long long x;
            if (scanf("%llu", &x) != 1) return 2;
            printf("%llu\n", (unsigned long long)kp::splitmix64(x));
        } else if (op[0] == 'h') {
            unsigned long long s;
            int u, v;
            if (scanf("%llu %d %d", &s, &u, &v) != 3) return 2;
            printf("%llu\n", (unsigned long long)kp::edge_hash(s, u, v));
        } else if (op[0] == 'b') {
            int r, v, u1, w1, u2, w2, av, a1, a2;
            unsigned long long seed;
            if (scanf("%d %llu %d %d %d %d %d %d %d %d", &r, &seed, &v, &u1, &w1, &u2, &w2, &av, &a1, &a2) != 10)
                return 2;
            switch (r) {
            case KP_RATING_EXPANSION_STAR2: order<KP_RATING_EXPANSION_STAR2>(seed, v, u1, w1, u2, w2, av, a1, a2); break;
            case KP_RATING_INNER_OUTER: order<KP_RATING_INNER_OUTER>(seed, v, u1, w1, u2, w2, av, a1, a2); break;
            case KP_RATING_WEIGHT: order<KP_RATING_WEIGHT>(seed, v, u1, w1, u2, w2, av, a1, a2); break;
            case KP_RATING_EXPANSION: order<KP_RATING_EXPANSION>(seed, v, u1, w1, u2, w2, av, a1, a2); break;
            case KP_RATING_EXPANSION_STAR: order<KP_RATING_EXPANSION_STAR>(seed, v, u1, w1, u2, w2, av, a1, a2); break;
            default: return 2;
            }
        } else if (op[0] == 'e') {
            int r, cur, v, w, s, ws, acur, as, av;
            unsigned long long seed;
            if (scanf("%d %llu %d %d %d %d %d %d %d %d", &r, &seed, &cur, &v, &w, &s, &ws, &acur, &as, &av) != 10)
                return 2;
            switch (r) {
            case KP_RATING_EXPANSION_STAR2: eligible<KP_RATING_EXPANSION_STAR2>(seed, cur, v, w, s, ws, acur, as, av); break;
            case KP_RATING_INNER_OUTER: eligible<KP_RATING_INNER_OUTER>(seed, cur, v, w, s, ws, acur, as, av); break;
            case KP_RATING_WEIGHT: eligible<KP_RATING_WEIGHT>(seed, cur, v, w, s, ws, acur, as, av); break;
            case KP_RATING_EXPANSION: eligible<KP_RATING_EXPANSION>(seed, cur, v, w, s, ws, acur, as, av); break;
            case KP_RATING_EXPANSION_STAR: eligible<KP_RATING_EXPANSION_STAR>(seed, cur, v, w, s, ws, acur, as, av); break;
            default: return 2;
            }
        } else if (op[0] == 'g') {
            int r, e[10];
            unsigned long long seed;
            if (scanf("%d %llu", &r, &seed) != 2) return 2;
            for (int i = 0; i < 10; i++)
                if (scanf("%d", &e[i]) != 1) return 2;
            switch (r) {
            case KP_RATING_EXPANSION_STAR2: gorder<KP_RATING_EXPANSION_STAR2>(seed, e); break;
            case KP_RATING_INNER_OUTER: gorder<KP_RATING_INNER_OUTER>(seed, e); break;
            case KP_RATING_WEIGHT: gorder<KP_RATING_WEIGHT>(seed, e); break;
            case KP_RATING_EXPANSION: gorder<KP_RATING_EXPANSION>(seed, e); break;
            case KP_RATING_EXPANSION_STAR: gorder<KP_RATING_EXPANSION_STAR>(seed, e); break;
            default: return 2;
            }
        } else {
            return 2;
        }
    }
    return 0;
}
