"""Pins for the oracle (CPU only).

Every check here compares the oracle with something other than itself: values
fixed by the paper's definitions and worked by hand, closed forms, invariants
the paper states (Section 2: contraction conserves node weight and merges
parallel edges; a matching has maximum degree one; Section 3.2: Greedy is a
1/2-approximation), an independent exact-rational library (fractions), brute
force on tiny graphs, and published values (splitmix64 test vectors, the
paper's instance sizes).
"""
import itertools
import math
import os
import random
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from paper_0910_2004_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
RATING_NAMES = ["expansion*2", "innerOuter", "weight", "expansion", "expansion*"]


def _golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


# --------------------------------------------------------------------------
# hash and exact comparison
# --------------------------------------------------------------------------

def test_splitmix64_published_vectors():
    gamma = 0x9E3779B97F4A7C15
    for idx, hexval in _golden("splitmix64_seed0.txt"):
        state = (int(idx) * gamma) & ((1 << 64) - 1)
        assert O.splitmix64(state) == int(hexval, 16)


def test_edge_hash_symmetric_and_seeded():
    for u, v in [(0, 1), (5, 3), (123456, 7)]:
        assert O.edge_hash(9, u, v) == O.edge_hash(9, v, u)
    assert O.edge_hash(1, 2, 3) != O.edge_hash(2, 2, 3)
    # the hashed state is seed xor (lo << 32 | hi)
    assert O.edge_hash(0, 3, 2) == O.splitmix64((2 << 32) | 3)


def test_frac_cmp_matches_fractions():
    rng = random.Random(5)
    cases = [(1, 0, 1, 0), (1, 0, 5, 3), (5, 3, 1, 0), (4, 2, 2, 1), (1, 3, 1, 4),
             (2**62 - 1, 2**62 - 3, 2**62 - 2, 2**62 - 4), (10, 7, 13, 9)]
    for _ in range(3000):
        bits = rng.choice([3, 10, 31, 62])
        a, c = rng.randint(1, 2**bits), rng.randint(1, 2**bits)
        b, d = rng.randint(0, 2**bits), rng.randint(0, 2**bits)
        if rng.random() < 0.2:   # equal values written differently
            f = rng.randint(1, 2**(bits // 2) + 1)
            c, d = a * f, b * f
            if c >= 2**64 or d >= 2**64:
                continue
        cases.append((a, b, c, d))
    for a, b, c, d in cases:
        inf1, inf2 = b == 0, d == 0
        if inf1 or inf2:
            want = (inf1 > inf2) - (inf1 < inf2)
        else:
            x, y = Fraction(a, b), Fraction(c, d)
            want = (x > y) - (x < y)
        assert O.frac_cmp(a, b, c, d) == want, (a, b, c, d)


# --------------------------------------------------------------------------
# ratings by hand (Section 3.1)
# --------------------------------------------------------------------------

def _triangle():
    # nodes 0,1,2 with c = (1,2,3); omega(0,1)=2, omega(1,2)=3, omega(0,2)=1
    return I.from_edges(3, np.array([0, 1, 0]), np.array([1, 2, 2]), np.array([2, 3, 1]),
                        vwgt=np.array([1, 2, 3]))


def test_ratings_hand_worked_triangle():
    g = _triangle()
    # Out = (3, 5, 4).  By hand:
    #   expansion*2: (0,1) 4/2=2   (1,2) 9/6=1.5   (0,2) 1/3
    #   innerOuter : (0,1) 2/(3+5-4)=0.5  (1,2) 3/(5+4-6)=1  (0,2) 1/(3+4-2)=0.2
    #   weight     : 2, 3, 1
    #   expansion  : 2/3, 3/5, 1/4
    #   expansion* : 1, 1/2, 1/3
    assert list(O.out_weight(g)) == [3, 5, 4]
    expect_first = {"expansion*2": (0, 1), "innerOuter": (1, 2), "weight": (1, 2),
                    "expansion": (0, 1), "expansion*": (0, 1)}
    out = O.out_weight(g)
    for r, (a, b) in expect_first.items():
        match, size = O.greedy_matching(g, r, 0)
        assert size == 1
        assert match[a] == b and match[b] == a
        other = ({0, 1, 2} - {a, b}).pop()
        assert match[other] == other
    # full order, expansion*2: (0,1) > (1,2) > (0,2)
    vw = g.vwgt
    assert O.edge_order("expansion*2", 0, vw, out, (0, 1, 2), (1, 2, 3)) == 1
    assert O.edge_order("expansion*2", 0, vw, out, (1, 2, 3), (0, 2, 1)) == 1
    # innerOuter: (1,2) > (0,1) > (0,2)
    assert O.edge_order("innerOuter", 0, vw, out, (1, 2, 3), (0, 1, 2)) == 1
    assert O.edge_order("innerOuter", 0, vw, out, (0, 1, 2), (0, 2, 1)) == 1
    # expansion*: (0,1)=1 > (1,2)=1/2 > (0,2)=1/3
    assert O.edge_order("expansion*", 0, vw, out, (0, 1, 2), (1, 2, 3)) == 1
    assert O.edge_order("expansion*", 0, vw, out, (1, 2, 3), (0, 2, 1)) == 1


def test_tie_break_hash_then_ids():
    # all ratings equal on a 4-cycle with unit weights: order = hash, then ids
    g = I.from_edges(4, np.array([0, 1, 2, 0]), np.array([1, 2, 3, 3]))
    for seed in range(20):
        match, size = O.greedy_matching(g, "expansion*2", seed)
        edges = [(0, 1), (1, 2), (2, 3), (0, 3)]
        top = max(edges, key=lambda e: (O.edge_hash(seed, *e), -e[0], -e[1]))
        assert match[top[0]] == top[1]
        assert size == 2


def test_infinite_ratings():
    # innerOuter on an isolated pair: denominator 0 -> +inf, beats any finite edge
    g = I.from_edges(5, np.array([0, 2, 3]), np.array([1, 3, 4]), np.array([1, 50, 60]))
    m, s = O.greedy_matching(g, "innerOuter", 3)
    assert m[0] == 1 and m[1] == 0
    # expansion*2 with c(v) = 0: every edge at v is +inf
    g = I.from_edges(4, np.array([0, 1, 2]), np.array([1, 2, 3]), np.array([1, 100, 1]),
                     vwgt=np.array([1, 1, 1, 0]))
    m, s = O.greedy_matching(g, "expansion*2", 0)
    assert m[2] == 3 and m[0] == 1


# --------------------------------------------------------------------------
# matching (Sections 2, 3.2, 3.3)
# --------------------------------------------------------------------------

def _edges(g):
    out = []
    for v in range(g.n):
        for e in range(g.xadj[v], g.xadj[v + 1]):
            u = int(g.adjncy[e])
            if u > v:
                out.append((v, u, int(g.ewgt[e])))
    return out


def _rating_fraction(r, g, out, u, v, w):
    cu, cv = int(g.vwgt[u]), int(g.vwgt[v])
    num, den = {
        "expansion*2": (w * w, cu * cv), "innerOuter": (w, int(out[u]) + int(out[v]) - 2 * w),
        "weight": (w, 1), "expansion": (w, cu + cv), "expansion*": (w, cu * cv)}[r]
    return math.inf if den == 0 else Fraction(num, den)


def _matching_checks(g, match, size):
    n = g.n
    assert all(0 <= match[v] < n for v in range(n))
    assert all(match[match[v]] == v for v in range(n))          # max degree one
    nbr = {(v, int(u)) for v in range(n) for u in g.adjncy[g.xadj[v]:g.xadj[v + 1]]}
    for v in range(n):
        if match[v] != v:
            assert (v, int(match[v])) in nbr                     # matched pairs are edges
    for v, u, _ in _edges(g):
        assert not (match[v] == v and match[u] == u)             # maximal
    assert size == sum(1 for v in range(n) if match[v] > v)


@pytest.mark.parametrize("rating", RATING_NAMES)
def test_greedy_equals_handshake_random(rating):
    for t in range(120):
        g = I.random_small_graph(n=random.Random(t).randint(2, 40), p=0.25, seed=t,
                                 wmax=[1, 3, 40][t % 3], cmax=[1, 3, 9][t % 3],
                                 allow_zero_c=(t % 7 == 0))
        seed = t * 7919
        mg, sg = O.greedy_matching(g, rating, seed)
        mh, sh, rounds, _ = O.handshake_matching(g, rating, seed)
        _matching_checks(g, mg, sg)
        assert (mg == mh).all() and sg == sh
        assert O.check_greedy_matching(g, rating, seed, mg) == -1


def test_greedy_equals_handshake_grids():
    for g, r in [(I.grid2d(33, 17), "expansion*2"), (I.grid3d(9, 7, 5), "innerOuter"),
                 (I.rgg2d(3000, 2, wmax=16), "expansion*2"), (I.rmat(9, 4), "innerOuter")]:
        mg, sg = O.greedy_matching(g, r, 11)
        mh, sh, _, _ = O.handshake_matching(g, r, 11)
        assert (mg == mh).all()
        assert O.check_greedy_matching(g, r, 11, mg) == -1


def test_checker_rejects_wrong_matchings():
    g = I.grid2d(10, 10)
    m, _ = O.greedy_matching(g, "expansion*2", 4)
    assert O.check_greedy_matching(g, "expansion*2", 4, m) == -1
    # unmatch one pair: an undominated edge appears
    bad = m.copy()
    v = int(np.nonzero(bad != np.arange(100))[0][0])
    u = int(bad[v])
    bad[v], bad[u] = v, u
    assert O.check_greedy_matching(g, "expansion*2", 4, bad) >= 0
    # the Greedy matching of another seed is a different valid maximal matching
    m2, _ = O.greedy_matching(g, "expansion*2", 5)
    assert not (m2 == m).all()
    assert O.check_greedy_matching(g, "expansion*2", 4, m2) >= 0


@pytest.mark.parametrize("rating", ["expansion*2", "innerOuter", "weight"])
def test_checker_at_listed_nodes_agrees_with_the_whole_pass(rating):
    """The per-node form of the Greedy characterisation (for graphs too large
    for a whole pass) passes exactly where the whole pass does: on every
    Greedy matching, and it finds each planted defect."""
    rng = np.random.default_rng(3)
    for t, g in enumerate([I.grid2d(10, 10), I.random_small_graph(80, 0.08, 5, wmax=7, cmax=3),
                           I.rmat(9, 4), I.circulant(101, I.circulant_strides(101, 5, 2))]):
        nodes = np.arange(g.n, dtype=np.int32)
        m, _ = O.greedy_matching(g, rating, t)
        assert O.check_greedy_matching_at(g, rating, t, m, nodes) == -1
        assert O.check_greedy_matching_at(g, rating, t, m, rng.permutation(nodes)[:7]) == -1
        # unmatch one pair; match another seed's matching; break symmetry
        bad1 = m.copy()
        v = int(np.nonzero(bad1 != nodes)[0][0])
        bad1[v], bad1[int(m[v])] = v, int(m[v])
        bad2, _ = O.greedy_matching(g, rating, t + 100)
        bad3 = m.copy()
        bad3[v] = v
        for bad in (bad1, bad2, bad3):
            whole = O.check_greedy_matching(g, rating, t, bad)
            if whole == -1:      # another seed may give the same matching
                assert (bad == m).all()
                continue
            # found over all nodes (at `whole` or at a neighbour, which sees
            # the broken matched edge of `whole`) and at `whole` alone
            assert O.check_greedy_matching_at(g, rating, t, bad, nodes) != -1
            assert O.check_greedy_matching_at(g, rating, t, bad, [whole]) == whole


def test_coarse_row_equals_the_contraction():
    """One coarse row from its members (for sampled checks of large graphs)
    equals that row of the whole contraction, whose invariants are pinned in
    test_contraction_invariants."""
    for t, g in enumerate([I.grid2d(12, 9), I.random_small_graph(70, 0.1, 8, wmax=9, cmax=4), I.rmat(10, 3),
                           I.star_graph(30), I.circulant(97, I.circulant_strides(97, 6, 4))]):
        match, _ = O.greedy_matching(g, "expansion*2", t)
        cg, mp = O.contract(g, match)
        rows = [(int(mp[v]), v, int(match[v]) if int(match[v]) != v else -1)
                for v in range(g.n) if int(match[v]) >= v]
        assert len(rows) == cg.n
        for (x, _, _), (adj, w, c) in zip(rows, O.coarse_rows(g, mp, rows)):
            lo, hi = int(cg.xadj[x]), int(cg.xadj[x + 1])
            assert np.array_equal(adj, cg.adjncy[lo:hi]) and np.array_equal(w, cg.ewgt[lo:hi]), (t, x)
            assert c == int(cg.vwgt[x])


def _brute_force_mwm(g, weights):
    edges = _edges(g)
    best = Fraction(0)
    for r in range(len(edges) + 1):
        for sub in itertools.combinations(range(len(edges)), r):
            used = set()
            ok = True
            for i in sub:
                a, b, _ = edges[i]
                if a in used or b in used:
                    ok = False
                    break
                used.update((a, b))
            if ok:
                best = max(best, sum((weights[i] for i in sub), Fraction(0)))
    return best


@pytest.mark.parametrize("rating", ["expansion*2", "weight", "expansion*"])
def test_half_approximation_brute_force(rating):
    """Greedy is a 1/2-approximation of a maximum weight matching (Section 3.2),
    checked by enumerating all matchings of tiny graphs (rating = weight)."""
    checked = 0
    for t in range(400):
        g = I.random_small_graph(n=7, p=0.5, seed=1000 + t, wmax=9, cmax=4)
        edges = _edges(g)
        if not 1 <= len(edges) <= 14:
            continue
        out = O.out_weight(g)
        wts = [_rating_fraction(rating, g, out, a, b, w) for a, b, w in edges]
        opt = _brute_force_mwm(g, wts)
        m, _ = O.greedy_matching(g, rating, t)
        got = sum((wts[i] for i, (a, b, _) in enumerate(edges) if m[a] == b), Fraction(0))
        assert 2 * got >= opt
        checked += 1
    assert checked > 100


def test_greedy_by_fraction_sort_small():
    """Greedy restated with Python's exact Fractions and sort."""
    for t in range(60):
        g = I.random_small_graph(n=25, p=0.2, seed=500 + t, wmax=6, cmax=5)
        for rating in RATING_NAMES:
            out = O.out_weight(g)
            es = _edges(g)
            key = lambda e: (_rating_fraction(rating, g, out, *e), O.edge_hash(t, e[0], e[1]),
                             -e[0], -e[1])
            free = set(range(g.n))
            want = list(range(g.n))
            for a, b, w in sorted(es, key=key, reverse=True):
                if a in free and b in free:
                    free -= {a, b}
                    want[a], want[b] = b, a
            m, _ = O.greedy_matching(g, rating, t)
            assert list(m) == want


def test_path_with_increasing_weights():
    """On a path whose edge (i,i+1) weighs i+1, Greedy (weight rating) takes
    the last edge, then every second one going down: closed form."""
    for n in [2, 3, 10, 11, 64]:
        g = I.path_graph(n)
        m, size = O.greedy_matching(g, "weight", 0)
        want = list(range(n))
        i = n - 2
        while i >= 0:
            want[i], want[i + 1] = i + 1, i
            i -= 2
        assert list(m) == want
        mh, _, rounds, _ = O.handshake_matching(g, "weight", 0)
        assert (mh == m).all()
        assert rounds == size   # one locally heaviest edge per round


# --------------------------------------------------------------------------
# contraction (Section 2) and projection
# --------------------------------------------------------------------------

def _cut_py(g, part):
    return sum(w for v, u, w in _edges(g) if part[v] != part[u])


@pytest.mark.parametrize("rating", ["expansion*2", "innerOuter"])
def test_contraction_invariants(rating):
    for t, g in enumerate([I.random_small_graph(60, 0.1, 3, wmax=5, cmax=4), I.grid2d(20, 13),
                           I.rgg2d(2000, 4, wmax=16), I.rmat(10, 2), I.star_graph(40)]):
        match, size = O.greedy_matching(g, rating, t)
        cg, mp = O.contract(g, match)
        assert O.validate(cg) == 0                                      # symmetric sorted, no self loops
        assert cg.n == g.n - size                                       # n' = n - |M|
        assert int(cg.vwgt.astype(np.int64).sum()) == int(g.vwgt.astype(np.int64).sum())
        wm = sum(w for v, u, w in _edges(g) if match[v] == u)
        assert int(cg.ewgt.astype(np.int64).sum()) // 2 == int(g.ewgt.astype(np.int64).sum()) // 2 - wm
        # matched pairs share a coarse node, distinct pairs do not
        for v in range(g.n):
            assert mp[v] == mp[match[v]]
        reps = sorted(set(min(v, int(match[v])) for v in range(g.n)))
        assert [int(mp[r]) for r in reps] == list(range(cg.n))
        # any coarse partition has the same cut and block weights when projected
        for k in [2, 3, 7]:
            cp = I.random_partition(cg.n, k, seed=t * 10 + k)
            fp = O.project([mp], cp)
            assert _cut_py(cg, cp) == _cut_py(g, fp)
            a = O.cut_gain(cg, cp, k, 0.03)
            b = O.cut_gain(g, fp, k, 0.03)
            assert a["cut"] == b["cut"] and (a["block_w"] == b["block_w"]).all()


def test_hierarchy_grid64_stop_rule():
    g = I.grid2d(64, 64)
    h = O.coarsen(g, "expansion*2", 1, stop_size=40)
    ns = [l.n for l in h.levels]
    assert ns[0] == 4096 and ns[-1] <= 40 and all(x > 40 for x in ns[:-1])
    for a, b, mm in zip(ns, ns[1:], h.matched):
        assert b == a - mm
    # cut of any coarse partition survives projection through all levels
    for k in [2, 5]:
        cp = I.random_balanced_partition(ns[-1], k, seed=k)
        fp = O.project(h.maps, cp)
        assert O.cut_gain(h.levels[-1], cp, k, 0.03)["cut"] == O.cut_gain(g, fp, k, 0.03)["cut"]


def test_stop_rules_no_progress_and_max_levels():
    # no edges: nothing to match, hierarchy is the input alone
    g = I.from_edges(50, np.zeros(0, np.int64), np.zeros(0, np.int64))
    h = O.coarsen(g, "expansion*2", 0, stop_size=2)
    assert len(h.levels) == 1
    # a star loses one leaf per level: stops on the shrink rule after one level
    h = O.coarsen(I.star_graph(100), "expansion*2", 0, stop_size=2)
    assert [l.n for l in h.levels] == [101, 100]
    # max_levels caps the number of contractions
    h = O.coarsen(I.grid2d(64, 64), "expansion*2", 1, stop_size=2, max_levels=3)
    assert len(h.maps) == 3


# --------------------------------------------------------------------------
# cut, balance, gain (Sections 2, 5.2)
# --------------------------------------------------------------------------

def test_cut_closed_forms():
    g = I.grid2d(64, 64)
    part = np.array([0 if (v % 64) < 32 else 1 for v in range(4096)], dtype=np.int32)
    r = O.cut_gain(g, part, 2, 0.03)
    assert r["cut"] == 64
    assert list(r["block_w"]) == [2048, 2048]
    # L_max = (1.03 * 4096)/2 + 1 = 2110.44 -> 2110
    assert r["L_max"] == 2110 and r["imbalance"] == 0
    g3 = I.grid3d(32, 32, 32)
    part3 = (np.arange(32 ** 3) // (32 * 32) >= 16).astype(np.int32)
    assert O.cut_gain(g3, part3, 2, 0.03)["cut"] == 32 * 32
    # a single block: no cut, every gain is -deg(v), no target
    one = np.zeros(4096, dtype=np.int32)
    r = O.cut_gain(g, one, 1, 0.0)
    deg = np.diff(g.xadj)
    assert r["cut"] == 0 and (r["gain"] == -deg).all() and (r["target"] == -1).all()
    assert r["L_max"] == 4096 + 1


def test_l_max_hand_values():
    assert O.l_max(4096, 1, 2, 0.03) == 2110
    assert O.l_max(1000, 7, 4, 0.0) == 257
    assert O.l_max(1000, 0, 3, 0.5) == 500       # 1.5*1000/3 = 500 exactly
    assert O.l_max(999, 0, 64, 0.03) == 16        # 16.077 -> 16


def test_gain_is_cut_decrease():
    """Moving v to target(v) lowers the cut by exactly gain(v) (Section 5.2),
    recomputed by brute force; no other block gives a larger decrease."""
    for t in range(40):
        g = I.random_small_graph(30, 0.15, 70 + t, wmax=7)
        for k in [2, 3, 5]:
            part = I.random_partition(g.n, k, seed=t)
            r = O.cut_gain(g, part, k, 0.03)
            base = _cut_py(g, part)
            assert r["cut"] == base
            for v in range(g.n):
                best = None
                for b in range(k):
                    if b == part[v]:
                        continue
                    p2 = part.copy()
                    p2[v] = b
                    dec = base - _cut_py(g, p2)
                    adjacent = any(part[u] == b for u in g.adjncy[g.xadj[v]:g.xadj[v + 1]])
                    if adjacent and (best is None or dec > best[0]):
                        best = (dec, b)
                if best is None:
                    assert r["target"][v] == -1
                    inside = sum(int(g.ewgt[e]) for e in range(g.xadj[v], g.xadj[v + 1]))
                    assert r["gain"][v] == -inside
                else:
                    assert r["gain"][v] == best[0] and r["target"][v] == best[1]


# --------------------------------------------------------------------------
# validation and generators
# --------------------------------------------------------------------------

def test_validate_rejects():
    g = I.grid2d(4, 4)
    assert O.validate(g) == 0
    bad = I.CSRGraph(g.xadj.copy(), g.adjncy.copy(), g.ewgt.copy(), g.vwgt.copy())
    bad.ewgt[0] = 2                      # asymmetric weight
    assert O.validate(bad) == 1
    bad = I.CSRGraph(g.xadj.copy(), g.adjncy.copy(), g.ewgt.copy(), g.vwgt.copy())
    bad.adjncy[0], bad.adjncy[1] = bad.adjncy[1], bad.adjncy[0]   # unsorted row
    assert O.validate(bad) == 1
    bad = I.CSRGraph(g.xadj.copy(), g.adjncy.copy(), g.ewgt.copy(), g.vwgt.copy())
    bad.vwgt[3] = -1
    assert O.validate(bad) == 1
    big = I.CSRGraph(g.xadj.copy(), g.adjncy.copy(), g.ewgt.copy(), g.vwgt.copy())
    big.vwgt[:] = 2**27                  # sum c = 2^31
    assert O.validate(big) == 2


def test_paper_rgg_instance_sizes():
    """The generator with the paper's radius 0.55 sqrt(ln n / n) reproduces the
    printed instance sizes of rgg17 and rgg18 within 1% (Section 6, Table 1)."""
    rows = {r[0]: (int(r[1]), int(r[2])) for r in _golden("paper_instances.txt")}
    for name in ["rgg17", "rgg18"]:
        n, m = rows[name]
        g = I.rgg2d(n, 3, radius=0.55 * math.sqrt(math.log(n) / n))
        assert abs(g.nnz / m - 1) < 0.01


def test_generators_shapes():
    g = I.grid2d(64, 64)
    assert g.n == 4096 and g.m == 8064
    g = I.grid3d(8, 8, 8)
    assert g.m == 3 * 64 * 7
    g = I.rgg2d(1 << 14, 1)
    assert abs(g.nnz / g.n - 6.0) < 0.3
    assert O.validate(g) == 0
    g = I.rmat(10, 1)
    assert O.validate(g) == 0 and g.ewgt.max() > 1
    p = I.random_balanced_partition(1000, 7, 3)
    assert np.bincount(p, minlength=7).max() - np.bincount(p, minlength=7).min() <= 1


# ---------------------------------------------------------------------------
# Section 5: quotient graph and bounded boundary search
# ---------------------------------------------------------------------------

def test_quotient_graph_of_grid_strips_closed_form():
    """A 12x9 grid cut into vertical strips of widths 3, 4, 5: the quotient
    graph is the path 0-1-2 and each edge weighs the strip height (9 unit
    edges cross each strip border)."""
    g = I.grid2d(12, 9)
    xs = np.arange(g.n) % 12
    part = np.where(xs < 3, 0, np.where(xs < 7, 1, 2)).astype(np.int32)
    xadj, adj, w = O.quotient_graph(g, part, 3)
    assert list(xadj) == [0, 1, 3, 4]
    assert list(adj) == [1, 0, 2, 1]
    assert list(w) == [9, 9, 9, 9]


def test_quotient_graph_weights_sum_to_twice_the_cut():
    for seed in range(20):
        rng = np.random.default_rng(seed)
        g = I.random_small_graph(int(rng.integers(2, 60)), 0.15, seed=seed, wmax=9)
        k = int(rng.integers(1, 7))
        part = I.random_partition(g.n, k, seed=seed)
        xadj, adj, w = O.quotient_graph(g, part, k)
        assert int(w.sum()) == 2 * O.cut_gain(g, part, k, 0.0)["cut"]
        # symmetric, sorted rows, no self loops
        for a in range(k):
            row = list(adj[xadj[a]:xadj[a + 1]])
            assert row == sorted(row) and a not in row
            for b, c in zip(row, w[xadj[a]:xadj[a + 1]]):
                j = list(adj[xadj[b]:xadj[b + 1]]).index(a)
                assert w[xadj[b] + j] == c


def test_boundary_band_closed_forms():
    # a path split in the middle: distance to the split point
    g = I.path_graph(11)
    part = (np.arange(11) >= 5).astype(np.int32)
    d = O.boundary_band(g, part, 100)
    assert list(d) == [4, 3, 2, 1, 0, 0, 1, 2, 3, 4, 5]
    assert list(O.boundary_band(g, part, 2)) == [-1, -1, 2, 1, 0, 0, 1, 2, -1, -1, -1]
    # grid strips: the distance to the nearest strip border in x
    g = I.grid2d(12, 5)
    xs = np.arange(g.n) % 12
    part = np.where(xs < 3, 0, np.where(xs < 7, 1, 2)).astype(np.int32)
    want = np.where(xs < 3, 2 - xs, np.where(xs < 7, np.minimum(xs - 3, 6 - xs), xs - 7))
    assert np.array_equal(O.boundary_band(g, part, 100), want)
    # the pair (0, 1): block 2 is out, block 1's border with block 2 is not a source
    d = O.boundary_band(g, part, 100, pair=(0, 1))
    want = np.where(xs < 3, 2 - xs, np.where(xs < 7, xs - 3, -2))
    assert np.array_equal(d, want)


def test_boundary_band_brute_force():
    """Each node's distance by its own breadth-first search inside its block
    to the nearest node with a neighbour in another block."""
    from collections import deque
    for seed in range(25):
        rng = np.random.default_rng(100 + seed)
        g = I.random_small_graph(int(rng.integers(2, 50)), float(rng.uniform(0.03, 0.2)), seed=seed)
        k = int(rng.integers(1, 5))
        part = I.random_partition(g.n, k, seed=seed)
        depth = int(rng.integers(0, 6))
        got = O.boundary_band(g, part, depth)
        nbrs = [g.adjncy[g.xadj[v]:g.xadj[v + 1]] for v in range(g.n)]
        boundary = [any(part[u] != part[v] for u in nbrs[v]) for v in range(g.n)]
        for v in range(g.n):
            seen, q, found = {v: 0}, deque([v]), -1
            while q:
                x = q.popleft()
                if boundary[x]:
                    found = seen[x]
                    break
                for y in nbrs[x]:
                    if part[y] == part[v] and y not in seen:
                        seen[y] = seen[x] + 1
                        q.append(y)
            want = found if 0 <= found <= depth else -1
            assert got[v] == want, (seed, v)
