"""Suitor proposals (Manne and Halappanavar's Suitor algorithm), the GPU's
default way to the matching of Sections 3.2-3.3, restated on the host and
checked against the oracle's Greedy matching.  CPU only.

Every node proposes to its best neighbour (in the strict edge order) whose
standing offer it beats; a node whose offer is beaten proposes again.  Under
a strict order the proposals settle on the locally dominant matching, which
is Greedy's, whatever order the proposals run in: the GPU runs them from
thousands of warps at once, in passes over parked rows, so this test runs
them in seeded random schedules.  The GPU kernels themselves are compared
with the oracle in the -m gpu parity tests; this test pins the
reformulation, and that the tie break is part of it."""
import numpy as np
import pytest

import oracle as O
from paper_0910_2004_gb300 import inputs as I
from tests.test_gpa_round_scheme import RATINGS, edge_keys, random_cases


def suitor_matching(g, rating: str, seed: int, schedule: np.random.Generator, key=None):
    """match[v] (v itself when unmatched) after the proposals settle, with the
    pending proposers taken in a random order drawn from `schedule`."""
    key = key or edge_keys(g, rating, seed)
    n = g.n
    rows = [[int(x) for x in g.adjncy[int(g.xadj[v]):int(g.xadj[v + 1])]] for v in range(n)]
    suitor = [-1] * n                 # the standing offer at each node
    pending = list(range(n))
    steps = 0
    while pending:
        steps += 1
        assert steps <= n + int(g.nnz) + 1, "every proposal raises an offer, and offers only rise"
        u = pending.pop(int(schedule.integers(len(pending))))
        best = -1
        for v in rows[u]:
            if suitor[v] >= 0 and not key(u, v) > key(suitor[v], v):
                continue                  # v holds an offer at least as good
            if best < 0 or key(u, v) > key(u, best):
                best = v
        if best < 0:
            continue
        displaced = suitor[best]
        suitor[best] = u
        if displaced >= 0:
            pending.append(displaced)
    return np.array([suitor[v] if suitor[v] >= 0 and suitor[suitor[v]] == v else v for v in range(n)],
                    dtype=np.int32)


def greedy(g, rating, seed):
    match, _ = O.greedy_matching(g, rating, seed)
    return match


@pytest.mark.parametrize("rating", RATINGS)
def test_any_schedule_settles_on_greedy(rating):
    for t, rng, g in random_cases(50, 9000):
        seed = int(rng.integers(0, 2 ** 40))
        want = greedy(g, rating, seed)
        for s in range(3):
            got = suitor_matching(g, rating, seed, np.random.default_rng(1000 * t + s))
            assert np.array_equal(got, want), (t, rating, s)


@pytest.mark.parametrize("g, rating", [(I.grid2d(24, 24), "expansion*2"), (I.grid3d(7, 7, 7), "innerOuter"),
                                        (I.rgg2d(2000, 4), "expansion*2"), (I.rmat(9, 3), "innerOuter"),
                                        (I.path_graph(300), "weight"), (I.path_graph(300, increasing=False), "weight"),
                                        (I.star_graph(50), "expansion")])
def test_structured_graphs(g, rating):
    want = greedy(g, rating, 11)
    for s in range(2):
        assert np.array_equal(suitor_matching(g, rating, 11, np.random.default_rng(s)), want)


def test_the_tie_break_is_needed():
    """Ratings alone are not a strict order on a unit-weight grid: compared by
    rating only (the first equal offer kept), the proposals end in neither
    Greedy's matching nor one matching for every schedule."""
    g = I.grid2d(16, 16)
    full = edge_keys(g, "weight", 3)
    rating_only = lambda u, v: full(u, v)[0]
    want = greedy(g, "weight", 3)
    outs = [suitor_matching(g, "weight", 3, np.random.default_rng(s), key=rating_only) for s in range(4)]
    assert all(not np.array_equal(o, want) for o in outs)
    assert any(not np.array_equal(outs[0], o) for o in outs[1:])
    assert np.array_equal(suitor_matching(g, "weight", 3, np.random.default_rng(0)), want)
