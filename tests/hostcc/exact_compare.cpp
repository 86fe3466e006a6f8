// Runs the library's exact rating comparison and tie-break hash
// (paper_0910_2004_gb300/csrc/kp_internal.cuh) on the host, one query per
// input line:  c a b d e  -> cmp_frac(a, b, d, e) (-1, 0 or 1)
//              s x        -> splitmix64(x)
//              h seed u v -> edge_hash(seed, u, v)
// Built with g++ and the stand-ins of cuda_stubs.h by tests/test_exact_compare_host.py.
#include <cstdio>

#include "kp_internal.cuh"

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
        } else {
            return 2;
        }
    }
    return 0;
}
