"""The second phase of the Global Path Algorithm (Section 3.2: a maximum
weight matching of every collected path and even cycle by dynamic
programming) as the GPU runs it, compiled by the host compiler and run on
the CPU from the oracle's first phase (CPU only).

The GPU's phase 2 (gpa_solve) reads phase 1's collected neighbours and the
closing edge of each cycle; here both come from the oracle (the closing edge
is a cycle's last edge in the strict order), so the matching it writes must
equal the oracle's Global Path Algorithm matching exactly: the ratings in
IEEE double, sums in the programme's order, an edge taken only when strictly
better, a path walked from its end with the smaller id, a cycle cut at its
closing edge.  Together with tests/test_gpa_round_scheme.py (phase 1 in
rounds) this covers the GPU's form of both phases on the CPU."""
import numpy as np
import pytest

import oracle as O
from paper_0910_2004_gb300 import inputs as I
from tests.test_exact_compare_host import host_program
from tests.test_gpa_round_scheme import RATINGS, edge_keys, random_cases

RATING_IDS = {"expansion*2": 0, "innerOuter": 1, "weight": 2, "expansion": 3, "expansion*": 4}


@pytest.fixture(scope="module")
def phase2(tmp_path_factory):
    return host_program("gpa_phase2.cpp", str(tmp_path_factory.mktemp("hostcc") / "gpa_phase2"))


def phase1_inputs(g, rating, seed, nbr2):
    """gnb (present neighbours first) and gclose (each cycle's last edge in
    the strict order, at both of its ends) from the oracle's phase 1."""
    n = g.n
    nb = [[int(x) for x in nbr2[2 * v:2 * v + 2] if x >= 0] for v in range(n)]
    gnb = [x for v in range(n) for x in (nb[v] + [-1, -1])[:2]]
    gclose = [-1] * n
    key = edge_keys(g, rating, seed)
    seen = [False] * n
    for s in range(n):
        if seen[s] or len(nb[s]) != 2:
            continue
        comp, stack = [], [s]
        seen[s] = True
        while stack:
            x = stack.pop()
            comp.append(x)
            for y in nb[x]:
                if not seen[y]:
                    seen[y] = True
                    stack.append(y)
        if all(len(nb[x]) == 2 for x in comp):          # a cycle
            edges = {(min(x, y), max(x, y)) for x in comp for y in nb[x]}
            a, b = min(edges, key=lambda e: key(*e))       # the smallest key comes last in the order
            gclose[a], gclose[b] = b, a
    return gnb, gclose


def run_case(phase2, g, rating, seed):
    match, _, nbr2 = O.gpa_matching(g, rating, seed)
    gnb, gclose = phase1_inputs(g, rating, seed, nbr2)
    out = O.out_weight(g).astype(np.int64)
    lines = [f"{RATING_IDS[rating]} {g.n} {g.nnz}"]
    for arr in (g.xadj, g.adjncy, g.ewgt, g.vwgt, out, gnb, gclose):
        lines.append(" ".join(str(int(x)) for x in arr))
    got = phase2(lines)
    return got, [int(x) for x in match], sum(1 for x in gclose if x >= 0) // 2


@pytest.mark.parametrize("rating", RATINGS)
def test_phase2_equals_the_oracle_on_random_graphs(phase2, rating):
    cycles = 0
    for t, rng, g in random_cases(60, 11000):
        seed = int(rng.integers(0, 2 ** 40))
        got, want, c = run_case(phase2, g, rating, seed)
        assert got == want, (t, rating)
        cycles += c
    assert cycles > 0, "the cases include closed cycles"


@pytest.mark.parametrize("g, rating", [(I.grid2d(20, 20), "expansion*2"), (I.grid2d(12, 12), "weight"),
                                        (I.grid3d(6, 6, 6), "innerOuter"), (I.rgg2d(1500, 3), "expansion*2"),
                                        (I.rmat(8, 2), "expansion*2"), (I.path_graph(201), "weight"),
                                        (I.path_graph(200, increasing=False), "weight"), (I.star_graph(30), "weight")])
def test_phase2_on_structured_graphs(phase2, g, rating):
    got, want, _ = run_case(phase2, g, rating, 5)
    assert got == want
