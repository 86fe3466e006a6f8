// Runs the library's second phase of the Global Path Algorithm (gpa_solve in
// paper_0910_2004_gb300/csrc/gpa.cuh: a maximum weight matching of every
// collected path and cycle by dynamic programming) on the host, for every
// node in turn, from phase 1's collected neighbours and closing edges given
// as input:
//   R n nnz / xadj[n+1] / adjncy[nnz] / ewgt[nnz] / vwgt[n] / outw[n] /
//   gnb[2n] (collected neighbours, -1 after the present ones) / gclose[n]
//   (the other end of the closing edge of a cycle at its two ends, else -1)
// Output: match[n] (v itself when unmatched).
// Built with g++ and the stand-ins of cuda_stubs.h by tests/test_gpa_phase2_host.py.
#include <cstdio>
#include <vector>

#include "gpa.cuh"

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

template <int R>
void solve_all(const kp::DevLevel &L, const kp::Work &w) {
    for (int32_t v = 0; v < L.n; v++) kp::gpa_solve<R>(L, w, v);
}

}  // namespace

int main() {
    int R, n;
    long long nnz;
    if (scanf("%d %d %lld", &R, &n, &nnz) != 3 || n < 0 || nnz < 0) return 2;
    std::vector<kp::eoff> xadj;
    std::vector<int32_t> adj, ew, vw, outw, gnb, gclose, match((size_t)n);
    if (!read(xadj, (size_t)n + 1) || !read(adj, (size_t)nnz) || !read(ew, (size_t)nnz) || !read(vw, (size_t)n) ||
        !read(outw, (size_t)n) || !read(gnb, 2 * (size_t)n) || !read(gclose, (size_t)n))
        return 2;
    std::vector<uint8_t> take((size_t)n, 0);
    for (int32_t v = 0; v < n; v++) match[(size_t)v] = v;
    kp::DevLevel L{};
    L.n = n;
    L.nnz = (kp::eoff)nnz;
    L.xadj = xadj.data();
    L.adjncy = adj.data();
    L.ewgt = ew.data();
    L.vwgt = vw.data();
    L.outw = outw.data();
    kp::Work w{};
    w.gnb = gnb.data();
    w.gclose = gclose.data();
    w.gtake = take.data();
    w.match = match.data();
    switch (R) {
    case KP_RATING_EXPANSION_STAR2: solve_all<KP_RATING_EXPANSION_STAR2>(L, w); break;
    case KP_RATING_INNER_OUTER: solve_all<KP_RATING_INNER_OUTER>(L, w); break;
    case KP_RATING_WEIGHT: solve_all<KP_RATING_WEIGHT>(L, w); break;
    case KP_RATING_EXPANSION: solve_all<KP_RATING_EXPANSION>(L, w); break;
    case KP_RATING_EXPANSION_STAR: solve_all<KP_RATING_EXPANSION_STAR>(L, w); break;
    default: return 2;
    }
    for (int32_t v = 0; v < n; v++) printf("%d\n", match[(size_t)v]);
    return 0;
}
