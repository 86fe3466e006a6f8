// Suitor proposals on the host with the library's own row search: every
// search is the kernel's scan_row<R,1> (the best neighbour whose standing
// offer the node beats, from the 16-byte offer records,
// paper_0910_2004_gb300/csrc/match.cuh); the 128-bit compare-and-swap that
// places a proposal is restated as a compare of the whole record and a write,
// and the searching nodes are taken in an order drawn from `order_seed`.
// Input:  R seed order_seed n nnz / xadj[n+1] / adjncy[nnz] / ewgt[nnz] / vwgt[n] / outw[n]
// Output: for every node with a nonempty row, on the initial (empty) offer
//         records: scan_row's best and scan_row_top2's best, second best and
//         count of eligible edges (up to 3), "b b2 s2 c2"; then the suitor
//         of every record after the proposals settle (-1: none); then, for
//         every node, scan_row's best on the settled records (-1: none)
// Built with g++ and the stand-ins of cuda_stubs.h by tests/test_suitor_host.py.
#include <cstdio>
#include <random>
#include <vector>

#include "match.cuh"

const uint3 threadIdx = {0, 0, 0};
const uint3 blockIdx = {0, 0, 0};
const dim3 blockDim(1, 1, 1);
const dim3 gridDim(1, 1, 1);

namespace {

template <class T>
bool read(std::vector<T> &v, size_t count) {
    v.resize(count);
    for (size_t i = 0; i < count; i++) {
        long long x;
        if (scanf("%lld", &x) != 1) return false;
        v[i] = (T)x;
    }
    return true;
}

bool same(const kp::Offer &a, const kp::Offer &b) { return a.s == b.s && a.w == b.w && a.as == b.as && a.au == b.au; }

template <int R>
int run(const kp::DevLevel &L, kp::Work &w, unsigned long long order_seed) {
    const int32_t n = L.n;
    for (int32_t v = 0; v < n; v++) w.offer[v] = kp::Offer{-1, 0, 0, kp::rating_attr<R>(L.vwgt, L.outw, v)};
    const kp::HashCtx hc{w.seed, 0};
    for (int32_t v = 0; v < n; v++) {
        if (L.xadj[v + 1] == L.xadj[v]) continue;
        const int32_t av = kp::rating_attr<R>(L.vwgt, L.outw, v);
        kp::Proposal b, b2;
        kp::Cached second;
        int32_t seen = 0;
        kp::scan_row<R, 1>(L, w, hc, v, av, L.xadj[v], L.xadj[v + 1], b);
        kp::scan_row_top2<R, 1>(L, w, hc, v, av, L.xadj[v], L.xadj[v + 1], b2, second, seen);
        printf("%d %d %d %d\n", b.c.u, b2.c.u, second.c.u, seen);
    }
    std::mt19937_64 rng(order_seed);
    std::vector<int32_t> pending(n);
    for (int32_t v = 0; v < n; v++) pending[(size_t)v] = v;
    long long steps = 0;
    while (!pending.empty()) {
        if (++steps > 4 * ((long long)n + L.nnz) + 16) return -1;   // offers only rise
        const size_t i = (size_t)(rng() % pending.size());
        const int32_t cur = pending[i];
        pending[i] = pending.back();
        pending.pop_back();
        const int32_t acur = kp::rating_attr<R>(L.vwgt, L.outw, cur);
        kp::Proposal b;
        kp::scan_row<R, 1>(L, w, hc, cur, acur, L.xadj[cur], L.xadj[cur + 1], b);
        if (b.c.u < 0) continue;
        kp::Offer &rec = w.offer[b.c.u];
        if (!same(rec, b.snap)) {   // the record changed under the search: search again
            pending.push_back(cur);
            continue;
        }
        const int32_t displaced = rec.s;
        rec = kp::Offer{cur, b.w, acur, b.snap.au};
        if (displaced >= 0) pending.push_back(displaced);
    }
    for (int32_t v = 0; v < n; v++) printf("%d\n", w.offer[v].s);
    for (int32_t v = 0; v < n; v++) {
        kp::Proposal b;
        kp::scan_row<R, 1>(L, w, hc, v, kp::rating_attr<R>(L.vwgt, L.outw, v), L.xadj[v], L.xadj[v + 1], b);
        printf("%d\n", b.c.u);
    }
    return 0;
}

}  // namespace

int main() {
    int R, n;
    long long nnz;
    unsigned long long seed, order_seed;
    if (scanf("%d %llu %llu %d %lld", &R, &seed, &order_seed, &n, &nnz) != 5 || n < 0 || nnz < 0) return 2;
    std::vector<kp::eoff> xadj;
    std::vector<int32_t> adj, ew, vw, outw;
    if (!read(xadj, (size_t)n + 1) || !read(adj, (size_t)nnz) || !read(ew, (size_t)nnz) || !read(vw, (size_t)n) ||
        !read(outw, (size_t)n))
        return 2;
    std::vector<kp::Offer> offer((size_t)n);
    kp::DevLevel L{};
    L.n = n;
    L.nnz = (kp::eoff)nnz;
    L.xadj = xadj.data();
    L.adjncy = adj.data();
    L.ewgt = ew.data();
    L.vwgt = vw.data();
    L.outw = outw.data();
    kp::Work w{};
    w.seed = seed;
    w.offer = offer.data();
    int st;
    switch (R) {
    case KP_RATING_EXPANSION_STAR2: st = run<KP_RATING_EXPANSION_STAR2>(L, w, order_seed); break;
    case KP_RATING_INNER_OUTER: st = run<KP_RATING_INNER_OUTER>(L, w, order_seed); break;
    case KP_RATING_WEIGHT: st = run<KP_RATING_WEIGHT>(L, w, order_seed); break;
    case KP_RATING_EXPANSION: st = run<KP_RATING_EXPANSION>(L, w, order_seed); break;
    case KP_RATING_EXPANSION_STAR: st = run<KP_RATING_EXPANSION_STAR>(L, w, order_seed); break;
    default: return 2;
    }
    return st < 0 ? 4 : 0;
}
