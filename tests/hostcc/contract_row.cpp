// Runs the library's one-thread contraction of a coarse row
// (contract_thread<T> in paper_0910_2004_gb300/csrc/contract.cuh: gather the
// two members' entries, drop those mapped to the row itself, sort by coarse
// neighbour in a register network, sum equal neighbours) on the host.
// One query per line:
//   T x da db gap k_1 w_1 ... k_n w_n     (n = da + db <= T)
// the first member's entries at 0..da-1, the second's after `gap` unused
// slots; k_i is the coarse id of entry i's neighbour.  Output:
//   cnt total k_1 s_1 ... k_cnt s_cnt
// Built with g++ and the stand-ins of cuda_stubs.h by tests/test_contract_row_host.py.
#include <cstdio>
#include <vector>

#include "contract.cuh"

int main() {
    int T, x, da, db, gap;
    while (scanf("%d %d %d %d %d", &T, &x, &da, &db, &gap) == 5) {
        const int n = da + db;
        if (n > T || (T != 16 && T != 32) || x < 0 || gap < 0) return 2;
        std::vector<int32_t> adj((size_t)n + gap), ew((size_t)n + gap, 0), map((size_t)n + gap, -7);
        for (int i = 0; i < n; i++) {
            const int e = i < da ? i : gap + i;
            if (scanf("%d %d", &map[(size_t)e], &ew[(size_t)e]) != 2) return 2;
        }
        for (size_t e = 0; e < adj.size(); e++) adj[e] = (int32_t)e;   // neighbour e sits at entry e
        const int at = 3;                                               // the row's slot in the buffers
        std::vector<kp::eoff> off((size_t)x + 1, 0);
        off[(size_t)x] = at;
        std::vector<int32_t> tadj(at + T, -1), tw(at + T, -1), degp((size_t)x + 1, -1), outw((size_t)x + 1, -1);
        kp::CView p{};
        p.adjncy = adj.data();
        p.ewgt = ew.data();
        p.map = map.data();
        p.off = off.data();
        p.tmp_adj = tadj.data();
        p.tmp_w = tw.data();
        p.degp = degp.data();
        p.outw = outw.data();
        if (T == 16) kp::contract_thread<16>(p, x, 0, da, da + gap, db);
        else kp::contract_thread<32>(p, x, 0, da, da + gap, db);
        printf("%d %d", degp[(size_t)x], outw[(size_t)x]);
        for (int i = 0; i < degp[(size_t)x]; i++) printf(" %d %d", tadj[(size_t)at + i], tw[(size_t)at + i]);
        printf("\n");
    }
    return 0;
}
