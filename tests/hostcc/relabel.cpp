// The coarse relabelling of a level on the host (RelabelOp in
// paper_0910_2004_gb300/csrc/contract.cuh, the element functions of the
// kernel's single-pass scan): the library's own load() (is v the
// representative of its pair, and the pair's row bound) and store() (map,
// members, coarse node weight and row offset from the exclusive prefix) are
// called around a plain sequential prefix sum.
// Input:  form n / xadj[n+1] / vwgt[n] / rec[n]
//         form 1: rec = the suitor in each node's offer record (-1: none; a
//         pair is two nodes whose records name each other); form 0: rec =
//         the handshake match array (-1: free, v: single, else the partner)
// Output: cn U / map[n] / first[cn] / second[cn] / cvwgt[cn] / off[cn]
// Built with g++ and the stand-ins of cuda_stubs.h by tests/test_relabel_host.py.
#include <cstdio>
#include <vector>

#include "contract.cuh"

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

template <bool SUITOR>
void run(int32_t n, const std::vector<kp::eoff> &xadj, const std::vector<int32_t> &vwgt, std::vector<int32_t> &rec) {
    std::vector<kp::Offer> offer((size_t)n);
    for (int32_t v = 0; v < n; v++) offer[(size_t)v] = kp::Offer{rec[(size_t)v], 1, 1, 1};
    std::vector<int32_t> map((size_t)n, -7), first((size_t)n, -7), second((size_t)n, -7), cvwgt((size_t)n, -7);
    std::vector<kp::eoff> off((size_t)n, -7);
    kp::RelabelOp<SUITOR> op{};
    op.n = n;
    op.xadj = xadj.data();
    op.vwgt = vwgt.data();
    op.gid = nullptr;
    op.map = map.data();
    op.cvwgt = cvwgt.data();
    op.gidn = nullptr;
    op.w.batch = 0;
    op.w.offer = offer.data();
    op.w.match = rec.data();
    op.w.first = first.data();
    op.w.second = second.data();
    op.w.off = off.data();
    std::vector<uint64_t> val((size_t)n);
    for (int32_t v = 0; v < n; v++) val[(size_t)v] = op.load(v);
    uint64_t excl = 0;
    for (int32_t v = 0; v < n; v++) {
        op.store(v, excl, val[(size_t)v]);
        excl += val[(size_t)v];
    }
    const int32_t cn = (int32_t)(excl >> 32);
    printf("%d %llu\n", cn, (unsigned long long)(excl & 0xffffffffu));
    for (int32_t v = 0; v < n; v++) printf("%d ", map[(size_t)v]);
    printf("\n");
    for (const std::vector<int32_t> *a : {&first, &second, &cvwgt}) {
        for (int32_t x = 0; x < cn; x++) printf("%d ", (*a)[(size_t)x]);
        printf("\n");
    }
    for (int32_t x = 0; x < cn; x++) printf("%lld ", (long long)off[(size_t)x]);
    printf("\n");
}

}  // namespace

int main() {
    int form, n;
    if (scanf("%d %d", &form, &n) != 2 || n < 0) return 2;
    std::vector<kp::eoff> xadj;
    std::vector<int32_t> vwgt, rec;
    if (!read(xadj, (size_t)n + 1) || !read(vwgt, (size_t)n) || !read(rec, (size_t)n)) return 2;
    if (form == 1) run<true>(n, xadj, vwgt, rec);
    else run<false>(n, xadj, vwgt, rec);
    return 0;
}
