"""Pins of the oracle's Global Path Algorithm (Section 3.2): phase 1 restated
with exact fractions, a sort and a breadth-first search instead of union-find;
the dynamic programme against brute-force maximum weight matchings of every
path and cycle it works on; the 1/2-approximation against brute force on tiny
graphs; closed forms on paths, cycles, triangles and stars.  CPU only."""
import itertools
import math
import random
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from paper_0910_2004_gb300 import inputs as I

RATING_NAMES = ["expansion*2", "innerOuter", "weight", "expansion", "expansion*"]


def _edges(g):
    return [(v, int(g.adjncy[e]), int(g.ewgt[e])) for v in range(g.n) for e in range(g.xadj[v], g.xadj[v + 1])
            if int(g.adjncy[e]) > v]


def _rating(r, g, out, u, v, w):
    cu, cv = int(g.vwgt[u]), int(g.vwgt[v])
    num, den = {
        "expansion*2": (w * w, cu * cv), "innerOuter": (w, int(out[u]) + int(out[v]) - 2 * w),
        "weight": (w, 1), "expansion": (w, cu + cv), "expansion*": (w, cu * cv)}[r]
    return math.inf if den == 0 else Fraction(num, den)


def _collect(g, rating, seed):
    """Phase 1 restated: edges in the strict order (exact fractions, then the
    seeded hash, then ids); an edge is taken when both ends have fewer than
    two taken edges and, if a walk along taken edges leads from one end to
    the other, that walk has an odd number of edges."""
    out = O.out_weight(g)
    key = lambda e: (_rating(rating, g, out, e[0], e[1], e[2]), O.edge_hash(seed, e[0], e[1]), -e[0], -e[1])
    adj = {v: [] for v in range(g.n)}
    for a, b, w in sorted(_edges(g), key=key, reverse=True):
        if len(adj[a]) >= 2 or len(adj[b]) >= 2:
            continue
        # walk from a along taken edges (a is a path end: at most one edge)
        prev, cur, steps, reaches_b = None, a, 0, False
        while True:
            nxt = [x for x in adj[cur] if x != prev]
            if not nxt:
                break
            prev, cur, steps = cur, nxt[0], steps + 1
            if cur == b:
                reaches_b = True
                break
        if reaches_b and steps % 2 == 0:
            continue
        adj[a].append(b)
        adj[b].append(a)
    return adj


def _components(adj):
    seen, comps = set(), []
    for v in adj:
        if v in seen or not adj[v]:
            continue
        stack, comp = [v], set()
        while stack:
            x = stack.pop()
            if x in comp:
                continue
            comp.add(x)
            stack += adj[x]
        seen |= comp
        comps.append(comp)
    return comps


def _brute_mwm(edge_list, weights):
    best = Fraction(0)
    for r in range(len(edge_list) + 1):
        for sub in itertools.combinations(range(len(edge_list)), r):
            used = set()
            if all(not (edge_list[i][0] in used or edge_list[i][1] in used or used.update(edge_list[i][:2]))
                   for i in sub):
                best = max(best, sum((weights[i] for i in sub), Fraction(0)))
    return best


def _match_weight(g, rating, match, pairs=None):
    out = O.out_weight(g)
    tot = Fraction(0)
    for a, b, w in _edges(g):
        if match[a] == b and (pairs is None or (a, b) in pairs):
            tot += _rating(rating, g, out, a, b, w)
    return tot


@pytest.mark.parametrize("rating", RATING_NAMES)
def test_collection_is_phase_one_restated(rating):
    for t in range(80):
        g = I.random_small_graph(n=random.Random(t).randint(2, 30), p=0.3, seed=2000 + t,
                                 wmax=[1, 4, 50][t % 3], cmax=[1, 3, 7][t % 3], allow_zero_c=(t % 9 == 0))
        m, size, nbr2 = O.gpa_matching(g, rating, t)
        want = _collect(g, rating, t)
        for v in range(g.n):
            got = sorted(int(x) for x in nbr2[2 * v:2 * v + 2] if x >= 0)
            assert got == sorted(want[v]), (t, v)
        # paths and even cycles only; the matching uses collected edges only
        for comp in _components(want):
            deg = [len(want[v]) for v in comp]
            assert max(deg) <= 2
            if min(deg) == 2:
                assert len(comp) % 2 == 0
        for v in range(g.n):
            assert m[m[v]] == v and (m[v] == v or int(m[v]) in want[v])
        assert size == sum(1 for v in range(g.n) if m[v] > v)


@pytest.mark.parametrize("rating", ["weight", "expansion*2"])
def test_dynamic_programme_is_optimal_on_every_path_and_cycle(rating):
    """With integer ratings (weight; expansion*2 with unit node weights) the
    double sums are exact, so the matching of every component must reach the
    component's brute-force maximum."""
    checked = 0
    for t in range(150):
        g = I.random_small_graph(n=16, p=0.3, seed=3000 + t, wmax=9, cmax=1)
        m, _, _ = O.gpa_matching(g, rating, t)
        adj = _collect(g, rating, t)
        out = O.out_weight(g)
        wt = {(a, b): _rating(rating, g, out, a, b, w) for a, b, w in _edges(g)}
        for comp in _components(adj):
            el = sorted({(min(v, u), max(v, u)) for v in comp for u in adj[v]})
            if len(el) > 14:
                continue
            opt = _brute_mwm(el, [wt[e] for e in el])
            got = sum((wt[e] for e in el if m[e[0]] == e[1]), Fraction(0))
            assert got == opt, (t, el)
            checked += 1
    assert checked > 200


@pytest.mark.parametrize("rating", ["expansion*2", "weight", "expansion*"])
def test_half_approximation_brute_force(rating):
    """GPA is a 1/2-approximation of a maximum weight matching (Section 3.2)."""
    checked = 0
    for t in range(300):
        g = I.random_small_graph(n=7, p=0.5, seed=4000 + t, wmax=9, cmax=4)
        el = [(a, b) for a, b, _ in _edges(g)]
        if not 1 <= len(el) <= 14:
            continue
        out = O.out_weight(g)
        wts = [_rating(rating, g, out, a, b, w) for a, b, w in _edges(g)]
        opt = _brute_mwm(el, wts)
        m, _, _ = O.gpa_matching(g, rating, t)
        assert 2 * _match_weight(g, rating, m) >= opt
        checked += 1
    assert checked > 100


def _cycle(weights):
    n = len(weights)
    lo = np.arange(n)
    hi = (lo + 1) % n
    return I.from_edges(n, np.minimum(lo, hi), np.maximum(lo, hi), np.asarray(weights))


def test_closed_forms():
    # a path with increasing weights 1..L: the optimum takes L, L-2, ...
    for n in [2, 3, 10, 11]:
        m, size, _ = O.gpa_matching(I.path_graph(n), "weight", 0)
        want = list(range(n))
        for i in range(n - 2, -1, -2):
            want[i], want[i + 1] = i + 1, i
        assert list(m) == want and size == n // 2
    # ties in the dynamic programme keep the edge nearer the path's end with
    # the smaller id (an edge is taken only when strictly better)
    m, size, _ = O.gpa_matching(I.from_edges(3, np.array([0, 1]), np.array([1, 2])), "weight", 0)
    assert list(m) == [1, 0, 2]
    m, size, _ = O.gpa_matching(I.from_edges(3, np.array([0, 2]), np.array([2, 1])), "weight", 0)
    assert list(m) == [2, 1, 0]   # the path 0 - 2 - 1, walked from 0
    # a triangle: the lightest edge would close an odd cycle; the collected
    # path of the two heavier edges is matched by its heavier edge
    m, size, nbr2 = O.gpa_matching(_cycle([5, 3, 4]), "weight", 0)   # edges {0,1}=5, {1,2}=3, {0,2}=4
    assert size == 1 and m[0] == 1 and m[2] == 2
    assert sorted(nbr2[2:4].tolist()) == [-1, 0]                   # node 1 keeps only {0,1}
    # an even cycle is collected whole (its lightest edge closes it, an even
    # cycle); its optimum {1,2},{3,4},{5,0} = 5+5+6 beats {0,1},{2,3},{4,5} = 4+1+1
    m, size, nbr2 = O.gpa_matching(_cycle([4, 5, 1, 5, 1, 6]), "weight", 0)
    assert all((nbr2[2 * v:2 * v + 2] >= 0).all() for v in range(6))
    assert list(m) == [5, 2, 1, 4, 3, 0] and size == 3
    # a 5-cycle: the closing edge is refused (odd), four edges stay collected
    m, size, nbr2 = O.gpa_matching(_cycle([9, 8, 7, 6, 5]), "weight", 0)
    assert size == 2 and m[0] == 1 and m[2] == 3 and m[4] == 4
    # a star: the centre keeps its two heaviest edges, the heaviest is matched
    g = I.from_edges(6, np.zeros(5, np.int64), np.arange(1, 6), np.array([3, 9, 4, 7, 1]))
    m, size, nbr2 = O.gpa_matching(g, "weight", 0)
    assert size == 1 and m[0] == 2 and sorted(nbr2[0:2].tolist()) == [2, 4]


def test_gpa_hierarchy_conserves_weights():
    """The contraction invariants hold with GPA matchings too."""
    g = I.rgg2d(3000, 5, wmax=16)
    h = O.coarsen(g, "expansion*2", 3, 40, matcher="gpa")
    assert len(h.levels) > 3
    for l, mp in enumerate(h.maps):
        a, b = h.levels[l], h.levels[l + 1]
        assert int(a.vwgt.sum()) == int(b.vwgt.sum())
        assert b.n == a.n - h.matched[l]
