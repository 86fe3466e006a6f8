"""The round form of the Global Path Algorithm's first phase (Section 3.2), the
schedule the cooperative GPU kernel follows, restated on the host and checked
against the sequential oracle.  CPU only.

The sequential phase takes the edges one by one in the strict order and keeps
an edge when both ends have fewer than two collected edges and it does not
close an odd cycle.  The round form decides, in every round, the edges that
are the best undecided edge at both of their ends:

- an edge with an end of degree 0 is taken (it cannot close a cycle);
- otherwise both ends have degree 1; walking from u along collected edges
  heavier than {u,v} either reaches v (a cycle: taken when the path has an
  odd number of edges, so the cycle is even, refused otherwise), or stops at
  a lighter collected edge (the path ends there for good: taken), or reaches
  a path end x, where {u,v} waits a round when x's best undecided edge is
  heavier or was taken in this same round (x's next edge is not known yet),
  and is taken otherwise.

The GPU kernel itself is compared with the oracle in tests/test_gpu_gpa.py;
this test pins the reformulation, and that the same-round rule is needed."""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from paper_0910_2004_gb300 import inputs as I

RATINGS = ["expansion*2", "innerOuter", "weight", "expansion", "expansion*"]


def edge_keys(g, rating: str, seed: int):
    """key(u, v): the strict edge order (Section 3.1 ratings as exact fractions,
    then the seeded hash, then the smaller (min, max) first) as a tuple that
    compares larger for the earlier edge."""
    out = O.out_weight(g)
    weight = {}
    for v in range(g.n):
        for e in range(int(g.xadj[v]), int(g.xadj[v + 1])):
            weight[(v, int(g.adjncy[e]))] = int(g.ewgt[e])

    def rating_of(a, b):
        w, ca, cb = weight[(a, b)], int(g.vwgt[a]), int(g.vwgt[b])
        num, den = {"expansion*2": (w * w, ca * cb), "innerOuter": (w, int(out[a]) + int(out[b]) - 2 * w),
                    "weight": (w, 1), "expansion": (w, ca + cb), "expansion*": (w, ca * cb)}[rating]
        return math.inf if den == 0 else Fraction(num, den)

    cache = {}

    def key(u, v):
        a, b = min(u, v), max(u, v)
        if (a, b) not in cache:
            cache[(a, b)] = (rating_of(a, b), O.edge_hash(seed, a, b), -a, -b)
        return cache[(a, b)]

    return key


def rounds_phase1(g, rating: str, seed: int, wait_on_same_round_take: bool = True):
    """Collected neighbours of every node after the rounds, and the round count."""
    key = edge_keys(g, rating, seed)
    n = g.n
    rows = [[int(x) for x in g.adjncy[int(g.xadj[v]):int(g.xadj[v + 1])]] for v in range(n)]
    coll = [[] for _ in range(n)]
    refused = set()
    active = list(range(n))
    rounds = 0
    while active:
        rounds += 1
        assert rounds <= int(g.nnz) + 2, "every round decides at least one edge"
        # rate: each node's best undecided edge
        best = [-1] * n
        for u in active:
            if len(coll[u]) >= 2:
                continue
            for v in rows[u]:
                if v in coll[u] or len(coll[v]) >= 2 or (min(u, v), max(u, v)) in refused:
                    continue
                if best[u] < 0 or key(u, v) > key(u, best[u]):
                    best[u] = v
        # pair: mutually best edges; those with an end of degree 0 are taken
        pending = []
        for u in active:
            v = best[u]
            if v > u and best[v] == u:
                if not coll[u] or not coll[v]:
                    coll[u].append(v)
                    coll[v].append(u)
                else:
                    pending.append((u, v))
        # check: walks read the collected edges (after the pair phase's takes)
        decision = {}
        for u, v in pending:
            k = key(u, v)
            prev, cur, steps, d = -1, u, 0, None
            while d is None:
                nxt = [x for x in coll[cur] if x != prev]
                if not nxt or not key(cur, nxt[0]) > k:
                    break
                prev, cur, steps = cur, nxt[0], steps + 1
                if cur == v:
                    d = "take" if steps % 2 == 1 else "refuse"
            if d is None:
                if [x for x in coll[cur] if x != prev]:
                    d = "take"                           # a lighter collected edge ends the path
                elif best[cur] >= 0 and best[cur] in coll[cur]:
                    d = "wait" if wait_on_same_round_take else "take"
                elif best[cur] >= 0 and key(cur, best[cur]) > k:
                    d = "wait"
                else:
                    d = "take"
            decision[(u, v)] = d
        # apply
        for (u, v), d in decision.items():
            if d == "refuse":
                refused.add((u, v))
            elif d == "take":
                coll[u].append(v)
                coll[v].append(u)
        active = [u for u in active if best[u] >= 0]
    return [sorted(c) for c in coll], rounds


def sequential_phase1(g, rating: str, seed: int):
    _, _, nbr2 = O.gpa_matching(g, rating, seed)
    return [sorted(int(x) for x in nbr2[2 * v:2 * v + 2] if x >= 0) for v in range(g.n)]


def random_cases(count: int, first_seed: int):
    for t in range(first_seed, first_seed + count):
        rng = np.random.default_rng(t)
        n = int(rng.integers(2, 70))
        g = I.random_small_graph(n, float(rng.uniform(0.03, 0.5)), seed=t, wmax=int(rng.choice([1, 2, 5, 1000])),
                                 cmax=int(rng.choice([1, 2, 4, 50])), allow_zero_c=(t % 4 == 0))
        yield t, rng, g


@pytest.mark.parametrize("rating", RATINGS)
def test_rounds_reach_the_sequential_paths_and_cycles(rating):
    for t, rng, g in random_cases(60, 7000):
        seed = int(rng.integers(0, 2 ** 40))
        got, _ = rounds_phase1(g, rating, seed)
        assert got == sequential_phase1(g, rating, seed), (t, rating)


@pytest.mark.parametrize("g, rating", [(I.grid2d(20, 20), "expansion*2"), (I.grid3d(6, 6, 6), "innerOuter"),
                                        (I.rgg2d(1500, 3), "expansion*2"), (I.rmat(8, 2), "expansion*2"),
                                        (I.path_graph(200), "weight"), (I.star_graph(40), "weight")])
def test_rounds_on_structured_graphs(g, rating):
    got, rounds = rounds_phase1(g, rating, 5)
    assert got == sequential_phase1(g, rating, 5)
    assert rounds <= g.nnz + 2


def test_the_same_round_wait_is_needed():
    """Without waiting when the path end's best edge was taken in the same
    round, a take at that end hides its next edge and the result differs
    from the sequential one on some inputs."""
    differ = 0
    for t, rng, g in random_cases(120, 7000):
        for rating in ("expansion*2", "weight"):
            seed = int(rng.integers(0, 2 ** 40))
            want = sequential_phase1(g, rating, seed)
            assert rounds_phase1(g, rating, seed)[0] == want
            differ += rounds_phase1(g, rating, seed, wait_on_same_round_take=False)[0] != want
    assert differ > 0
