"""Handshake rounds (Section 3.3) as the GPU kernel runs them, on the CPU:
the library's own rate_node (a node's best free neighbour under the strict
order), compiled by the host compiler and called in the kernel's round loop
by tests/hostcc/handshake_rounds.cpp (CPU only).

Checked against the oracle's literal round-by-round simulation: the first
round's candidates, the matching, and the number of rounds (the kernel
counts one more when free nodes remain after the last matching round: that
round finds them single)."""
import numpy as np
import pytest

import oracle as O
from paper_0910_2004_gb300 import inputs as I
from tests.test_exact_compare_host import host_program
from tests.test_gpa_round_scheme import RATINGS, random_cases

RATING_IDS = {"expansion*2": 0, "innerOuter": 1, "weight": 2, "expansion": 3, "expansion*": 4}


@pytest.fixture(scope="module")
def handshake(tmp_path_factory):
    return host_program("handshake_rounds.cpp", str(tmp_path_factory.mktemp("hostcc") / "handshake_rounds"))


def run_case(handshake, g, rating, seed):
    out = O.out_weight(g).astype(np.int64)
    lines = [f"{RATING_IDS[rating]} {seed} {g.n} {g.nnz}"]
    for arr in (g.xadj, g.adjncy, g.ewgt, g.vwgt, out):
        lines.append(" ".join(str(int(x)) for x in arr))
    res = handshake(lines)
    rounds, cand1, match = res[0], res[1:1 + g.n], res[1 + g.n:]
    want_match, _, want_rounds, want_cand1 = O.handshake_matching(g, rating, seed)
    return (cand1 == [int(x) for x in want_cand1], match == [int(x) for x in want_match],
            rounds in (want_rounds, want_rounds + 1), (rounds, want_rounds))


@pytest.mark.parametrize("rating", RATINGS)
def test_kernel_rating_in_rounds_equals_the_oracle(handshake, rating):
    for t, rng, g in random_cases(80, 17000):
        seed = int(rng.integers(0, 2 ** 40))
        ok_cand, ok_match, ok_rounds, r = run_case(handshake, g, rating, seed)
        assert ok_cand and ok_match and ok_rounds, (t, rating, ok_cand, ok_match, r)


@pytest.mark.parametrize("g, rating", [(I.grid2d(24, 24), "expansion*2"), (I.grid2d(12, 12), "weight"),
                                        (I.grid3d(7, 7, 7), "innerOuter"), (I.rgg2d(2000, 3), "expansion*2"),
                                        (I.rmat(9, 2), "innerOuter"), (I.path_graph(120), "weight"),
                                        (I.star_graph(60), "expansion")])
def test_structured_graphs(handshake, g, rating):
    ok_cand, ok_match, ok_rounds, r = run_case(handshake, g, rating, 9)
    assert ok_cand and ok_match and ok_rounds, r


def test_increasing_path_takes_one_edge_per_round(handshake):
    """The closed form: on a path with increasing weights only the heaviest
    free edge is mutual, so n/2 rounds match one edge each."""
    g = I.path_graph(64)
    _, ok_match, ok_rounds, (rounds, want) = run_case(handshake, g, "weight", 1)
    assert ok_match and ok_rounds and want == 32
