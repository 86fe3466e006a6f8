// Handshake rounds on the host as the cooperative kernel runs them
// (phase_handshake in paper_0910_2004_gb300/csrc/match.cuh): the library's
// own rate_node<R,1> rates each node (its best free neighbour, or single);
// the handshake step between the rates (a node is matched when its candidate
// names it too, else it stays for the next round) restates the kernel's.
// Input:  R seed n nnz / xadj[n+1] / adjncy[nnz] / ewgt[nnz] / vwgt[n] / outw[n]
// Output: rounds, then the first round's candidates cand[n] (-1: none), then
//         match[n] (v itself when single)
// Built with g++ and the stand-ins of cuda_stubs.h by tests/test_handshake_host.py.
#include <cstdio>
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

template <int R>
int run(const kp::DevLevel &L, kp::Work &w, std::vector<int32_t> &cand1) {
    const int32_t n = L.n;
    kp::Counters ctr{};
    std::vector<int32_t> lst(n), nxt;
    for (int32_t v = 0; v < n; v++) lst[(size_t)v] = v;
    int rounds = 0;
    bool recheck = false;
    while (!lst.empty()) {
        if (++rounds > n + 2) return -1;   // every round but the last matches an edge
        for (int32_t v : lst) kp::rate_node<R, 1>(L, w, &ctr, v, recheck);
        if (!recheck) cand1.assign(w.cand, w.cand + n);
        recheck = true;
        nxt.clear();
        for (int32_t v : lst) {
            if (w.match[v] != -1) continue;
            const int32_t c = w.cand[v];
            if (c >= 0 && w.cand[c] == v) w.match[v] = c;
            else nxt.push_back(v);
        }
        lst.swap(nxt);
    }
    return rounds;
}

}  // namespace

int main() {
    int R, n;
    long long nnz;
    unsigned long long seed;
    if (scanf("%d %llu %d %lld", &R, &seed, &n, &nnz) != 4 || n < 0 || nnz < 0) return 2;
    std::vector<kp::eoff> xadj;
    std::vector<int32_t> adj, ew, vw, outw;
    if (!read(xadj, (size_t)n + 1) || !read(adj, (size_t)nnz) || !read(ew, (size_t)nnz) || !read(vw, (size_t)n) ||
        !read(outw, (size_t)n))
        return 2;
    std::vector<int32_t> match((size_t)n, -1), cand((size_t)n, -1), cand1;
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
    w.match = match.data();
    w.cand = cand.data();
    int rounds;
    switch (R) {
    case KP_RATING_EXPANSION_STAR2: rounds = run<KP_RATING_EXPANSION_STAR2>(L, w, cand1); break;
    case KP_RATING_INNER_OUTER: rounds = run<KP_RATING_INNER_OUTER>(L, w, cand1); break;
    case KP_RATING_WEIGHT: rounds = run<KP_RATING_WEIGHT>(L, w, cand1); break;
    case KP_RATING_EXPANSION: rounds = run<KP_RATING_EXPANSION>(L, w, cand1); break;
    case KP_RATING_EXPANSION_STAR: rounds = run<KP_RATING_EXPANSION_STAR>(L, w, cand1); break;
    default: return 2;
    }
    if (rounds < 0) return 4;
    printf("%d\n", rounds);
    for (int32_t v = 0; v < n; v++) printf("%d\n", cand1.empty() ? -1 : cand1[(size_t)v]);
    for (int32_t v = 0; v < n; v++) printf("%d\n", match[(size_t)v]);
    return 0;
}
