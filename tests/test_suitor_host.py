"""Suitor proposals with the kernel's own row search on the CPU: every search
is the library's scan_row (the best neighbour whose standing offer the node
beats, read from the 16-byte offer records), compiled by the host compiler
and driven by tests/hostcc/suitor_schedule.cpp in seeded random schedules;
only the 128-bit compare-and-swap is restated (compare the whole record,
then write).  CPU only.

Checked against the oracle: the settled matching is Greedy's (Section 3.2,
the locally dominant matching under the strict order) for every rating and
schedule; on empty offer records scan_row_top2 (which fills the candidate
cache of long rows) returns a node's best and second best neighbours in the
strict order and the count of eligible edges up to 3; on the settled records
a node with a standing offer has no eligible edge above its target and a
node without one has no eligible edge at all (the fixed point: offers only
rise, so no search would place a better proposal)."""
import numpy as np
import pytest

import oracle as O
from paper_0910_2004_gb300 import inputs as I
from tests.test_exact_compare_host import host_program
from tests.test_gpa_round_scheme import RATINGS, edge_keys, random_cases

RATING_IDS = {"expansion*2": 0, "innerOuter": 1, "weight": 2, "expansion": 3, "expansion*": 4}


@pytest.fixture(scope="module")
def suitor(tmp_path_factory):
    return host_program("suitor_schedule.cpp", str(tmp_path_factory.mktemp("hostcc") / "suitor_schedule"))


def run_case(suitor, g, rating, seed, order_seed):
    out = O.out_weight(g).astype(np.int64)
    lines = [f"{RATING_IDS[rating]} {seed} {order_seed} {g.n} {g.nnz}"]
    for arr in (g.xadj, g.adjncy, g.ewgt, g.vwgt, out):
        lines.append(" ".join(str(int(x)) for x in arr))
    res = suitor(lines)
    rows = [v for v in range(g.n) if g.xadj[v + 1] > g.xadj[v]]
    first = res[:4 * len(rows)]
    suitors = res[4 * len(rows):4 * len(rows) + g.n]
    after = res[4 * len(rows) + g.n:]
    match = [s if s >= 0 and suitors[s] == v else v for v, s in enumerate(suitors)]
    target = [-1] * g.n                       # where each node's offer stands
    for x, s in enumerate(suitors):
        if s >= 0:
            assert target[s] == -1, "a node's offer stands at one record at most"
            target[s] = x
    # expected first searches: neighbours in the strict order, from the oracle's ratings and hash
    key = edge_keys(g, rating, seed)
    want_first = []
    for v in rows:
        nb = sorted((int(u) for u in g.adjncy[int(g.xadj[v]):int(g.xadj[v + 1])]), key=lambda u: key(v, u),
                    reverse=True)
        want_first += [nb[0], nb[0], nb[1] if len(nb) > 1 else -1, min(len(nb), 3)]
    greedy, _ = O.greedy_matching(g, rating, seed)
    settled = all(b == -1 or (t >= 0 and key(v, b) < key(v, t)) for v, (b, t) in enumerate(zip(after, target)))
    return first == want_first, match == [int(x) for x in greedy], settled


@pytest.mark.parametrize("rating", RATINGS)
def test_kernel_search_in_random_schedules_settles_on_greedy(suitor, rating):
    for t, rng, g in random_cases(60, 15000):
        seed = int(rng.integers(0, 2 ** 40))
        for order_seed in (1, 2):
            ok_first, ok_match, ok_after = run_case(suitor, g, rating, seed, 1000 * t + order_seed)
            assert ok_first and ok_match and ok_after, (t, rating, order_seed, ok_first, ok_match, ok_after)


@pytest.mark.parametrize("g, rating", [(I.grid2d(24, 24), "expansion*2"), (I.grid2d(12, 12), "weight"),
                                        (I.grid3d(7, 7, 7), "innerOuter"), (I.rgg2d(2000, 3), "expansion*2"),
                                        (I.rmat(9, 2), "innerOuter"), (I.path_graph(300), "weight"),
                                        (I.star_graph(60), "expansion")])
def test_structured_graphs(suitor, g, rating):
    for order_seed in (3, 4):
        assert run_case(suitor, g, rating, 7, order_seed) == (True, True, True)
