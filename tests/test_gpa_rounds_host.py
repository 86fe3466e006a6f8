"""The Global Path Algorithm as the GPU kernel runs it, on the CPU: the
library's own rating (gpa_rate_node), cycle check (gpa_check) and dynamic
programme (gpa_solve), compiled by the host compiler and called in the
kernel's round schedule by tests/hostcc/gpa_rounds.cpp, one node at a time
within each phase (CPU only).  The collected paths and cycles must be the
oracle's phase 1 and the matching the oracle's Global Path Algorithm
matching (Section 3.2), for every rating.

The GPU kernel itself is compared with the oracle by the -m gpu tests; here
the same device functions meet many more small graphs with ties, zero node
weights and closed cycles in a few seconds, and a fault planted in one of
them shows which rule it broke."""
import numpy as np
import pytest

import oracle as O
from paper_0910_2004_gb300 import inputs as I
from tests.test_exact_compare_host import host_program
from tests.test_gpa_round_scheme import RATINGS, random_cases

RATING_IDS = {"expansion*2": 0, "innerOuter": 1, "weight": 2, "expansion": 3, "expansion*": 4}


@pytest.fixture(scope="module")
def gpa_rounds(tmp_path_factory):
    return host_program("gpa_rounds.cpp", str(tmp_path_factory.mktemp("hostcc") / "gpa_rounds"))


def run_case(gpa_rounds, g, rating, seed):
    out = O.out_weight(g).astype(np.int64)
    lines = [f"{RATING_IDS[rating]} {seed} {g.n} {g.nnz}"]
    for arr in (g.xadj, g.adjncy, g.ewgt, g.vwgt, out):
        lines.append(" ".join(str(int(x)) for x in arr))
    res = gpa_rounds(lines)
    rounds, match, gnb = res[0], res[1:1 + g.n], res[1 + g.n:]
    want_match, _, nbr2 = O.gpa_matching(g, rating, seed)
    got_nb = [sorted(x for x in gnb[2 * v:2 * v + 2] if x >= 0) for v in range(g.n)]
    want_nb = [sorted(int(x) for x in nbr2[2 * v:2 * v + 2] if x >= 0) for v in range(g.n)]
    return rounds, got_nb == want_nb, match == [int(x) for x in want_match]


@pytest.mark.parametrize("rating", RATINGS)
def test_kernel_functions_in_rounds_equal_the_oracle(gpa_rounds, rating):
    for t, rng, g in random_cases(80, 13000):
        seed = int(rng.integers(0, 2 ** 40))
        _, same_paths, same_match = run_case(gpa_rounds, g, rating, seed)
        assert same_paths and same_match, (t, rating, same_paths, same_match)


@pytest.mark.parametrize("g, rating", [(I.grid2d(24, 24), "expansion*2"), (I.grid2d(12, 12), "weight"),
                                        (I.grid3d(7, 7, 7), "innerOuter"), (I.rgg2d(2000, 3), "expansion*2"),
                                        (I.rmat(9, 2), "expansion*2"), (I.path_graph(300), "weight"),
                                        (I.path_graph(300, increasing=False), "weight"), (I.star_graph(60), "weight")])
def test_structured_graphs(gpa_rounds, g, rating):
    rounds, same_paths, same_match = run_case(gpa_rounds, g, rating, 5)
    assert same_paths and same_match
    assert 1 <= rounds <= 4 * g.n + 16
