// Runs the Global Path Algorithm of one level on the host the way the
// cooperative kernel schedules it (phase_gpa in
// paper_0910_2004_gb300/csrc/gpa.cuh), one node at a time within each phase:
// the library's own gpa_rate_node<R,1> (best undecided edge), gpa_check<R>
// (the walk deciding a pending edge) and gpa_solve<R> (phase 2) are called;
// the bookkeeping between them (mutual pairs, degree-0 takes, applying the
// decisions after every check) restates the kernel's.  Rows must have at
// most GPA_HUB_ROW entries (hubs take the block-wide rating).
// Input:  R seed n nnz / xadj[n+1] / adjncy[nnz] / ewgt[nnz] / vwgt[n] / outw[n]
// Output: rounds, then match[n] (v itself when unmatched), then the collected
//         neighbours gnb[2n] (-1 after the present ones)
// Built with g++ and the stand-ins of cuda_stubs.h by tests/test_gpa_rounds_host.py.
#include <cstdio>
#include <vector>

#include "gpa.cuh"

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
int run(const kp::DevLevel &L, kp::Work &w) {
    const int32_t n = L.n;
    int32_t err = 0;
    std::vector<int32_t> lst(n), nxt;
    for (int32_t v = 0; v < n; v++) lst[(size_t)v] = v;
    bool first = true;
    int rounds = 0;
    while (!lst.empty()) {
        if (++rounds > 4 * n + 16) return -1;   // every round decides an edge
        for (int32_t u : lst) kp::gpa_rate_node<R, 1>(L, w, u, !first);
        first = false;
        // mutual best edges: taken when an end has no collected edge, else pending
        std::vector<int32_t> pend;
        nxt.clear();
        for (int32_t u : lst) {
            const int32_t v = w.cand[u];
            if (v >= 0) nxt.push_back(u);
            if (v > u && w.cand[v] == u) {
                int32_t *nu = w.gnb + 2 * (int64_t)u, *nv = w.gnb + 2 * (int64_t)v;
                if (nu[0] < 0 || nv[0] < 0) {
                    nu[nu[0] >= 0] = v;
                    nv[nv[0] >= 0] = u;
                } else {
                    pend.push_back(u);
                }
            }
        }
        std::vector<int8_t> dec(pend.size());
        for (size_t i = 0; i < pend.size(); i++) dec[i] = kp::gpa_check<R>(L, w, pend[i], &err);
        for (size_t i = 0; i < pend.size(); i++) {
            if (dec[i] == kp::GPA_WAIT) continue;
            const int32_t u = pend[i], v = w.cand[u];
            if (dec[i] == kp::GPA_REFUSE) {
                const kp::eoff e1 = kp::gpa_entry(L, u, v), e2 = kp::gpa_entry(L, v, u);
                if (e1 >= 0) w.grej[e1] = 1;
                if (e2 >= 0) w.grej[e2] = 1;
                w.cand[u] = -2;
                w.cand[v] = -2;
                continue;
            }
            w.gnb[2 * (int64_t)u + 1] = v;
            w.gnb[2 * (int64_t)v + 1] = u;
            if (dec[i] == kp::GPA_CLOSE) {
                w.gclose[u] = v;
                w.gclose[v] = u;
            }
        }
        lst.swap(nxt);
    }
    if (err) return -1;
    for (int32_t v = 0; v < n; v++) kp::gpa_solve<R>(L, w, v);
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
    for (int32_t v = 0; v < n; v++)
        if (xadj[(size_t)v + 1] - xadj[(size_t)v] > kp::GPA_HUB_ROW) return 3;
    std::vector<int32_t> gnb(2 * (size_t)n, -1), gclose((size_t)n, -1), match((size_t)n), cand((size_t)n, -1);
    std::vector<uint8_t> grej((size_t)nnz + 1, 0), take((size_t)n, 0);
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
    w.seed = seed;
    w.gnb = gnb.data();
    w.gclose = gclose.data();
    w.gtake = take.data();
    w.grej = grej.data();
    w.cand = cand.data();
    w.match = match.data();
    int rounds;
    switch (R) {
    case KP_RATING_EXPANSION_STAR2: rounds = run<KP_RATING_EXPANSION_STAR2>(L, w); break;
    case KP_RATING_INNER_OUTER: rounds = run<KP_RATING_INNER_OUTER>(L, w); break;
    case KP_RATING_WEIGHT: rounds = run<KP_RATING_WEIGHT>(L, w); break;
    case KP_RATING_EXPANSION: rounds = run<KP_RATING_EXPANSION>(L, w); break;
    case KP_RATING_EXPANSION_STAR: rounds = run<KP_RATING_EXPANSION_STAR>(L, w); break;
    default: return 2;
    }
    if (rounds < 0) return 4;
    printf("%d\n", rounds);
    for (int32_t v = 0; v < n; v++) printf("%d\n", match[(size_t)v]);
    for (size_t i = 0; i < gnb.size(); i++) printf("%d\n", gnb[i]);
    return 0;
}
