"""The coarse relabelling of a level (Section 2: a matched pair becomes one
coarse node of weight c(u) + c(v); coarse ids by the rank of the pair's
representative, the smaller id) as the GPU computes it, on the CPU: the
element functions of the kernel's single-pass scan (RelabelOp::load and
::store), compiled by the host compiler and called around a sequential
prefix sum by tests/hostcc/relabel.cpp (CPU only).

Checked against the oracle's contraction of the same matching: the map, the
coarse node weights, the members of every coarse node, and the row bounds
(deg(u) + deg(v) - 2 per pair: the pair's own edge dropped) with their
exclusive prefix U.  Both record forms: Suitor offer records, where stale
non-mutual suitors must not form pairs, and the handshake match array,
where a node still free (after a wait that gave up) counts as single."""
import numpy as np
import pytest

import oracle as O
from paper_0910_2004_gb300 import inputs as I
from tests.test_exact_compare_host import host_program
from tests.test_gpa_round_scheme import random_cases


@pytest.fixture(scope="module")
def relabel(tmp_path_factory):
    return host_program("relabel.cpp", str(tmp_path_factory.mktemp("hostcc") / "relabel"))


def records(g, match, form, rng):
    """The GPU-side record of the matching: form 1 offer suitors (unmatched
    nodes get no suitor or a stale one that does not name them back), form 0
    the match array (unmatched nodes single or still free)."""
    n = g.n
    rec = [-1] * n
    for v in range(n):
        if match[v] != v:
            rec[v] = int(match[v])
        elif form == 0:
            rec[v] = v if rng.integers(2) else -1
    if form == 1:
        for v in range(n):
            deg = int(g.xadj[v + 1] - g.xadj[v])
            if match[v] == v and deg and rng.integers(2):
                u = int(g.adjncy[int(g.xadj[v]) + int(rng.integers(deg))])
                if rec[u] != v:
                    rec[v] = u
    return rec


def expected(g, match):
    coarse, mp = O.contract(g, match)
    cn = coarse.n
    members = [[] for _ in range(cn)]
    for v in range(g.n):
        members[int(mp[v])].append(v)
    first = [m[0] for m in members]
    second = [m[1] if len(m) > 1 else -1 for m in members]
    deg = np.diff(g.xadj.astype(np.int64))
    ub = [int(deg[a]) + (int(deg[b]) - 2 if b >= 0 else 0) for a, b in zip(first, second)]
    off = [0] + list(np.cumsum(ub[:-1])) if cn else []
    return [cn, sum(ub)] + [int(x) for x in mp] + first + second + [int(x) for x in coarse.vwgt] + [int(x) for x in off]


def run_case(relabel, g, match, form, rng):
    rec = records(g, match, form, rng)
    lines = [f"{form} {g.n}", " ".join(str(int(x)) for x in g.xadj), " ".join(str(int(x)) for x in g.vwgt),
             " ".join(str(x) for x in rec)]
    return relabel(lines) == expected(g, match)


@pytest.mark.parametrize("form", [1, 0])
def test_relabel_equals_the_oracle_contraction(relabel, form):
    for t, rng, g in random_cases(150, 19000):
        rating = ["expansion*2", "innerOuter", "weight", "expansion", "expansion*"][t % 5]
        match, _ = O.greedy_matching(g, rating, int(rng.integers(0, 2 ** 40)))
        assert run_case(relabel, g, match, form, rng), (t, form)


@pytest.mark.parametrize("form", [1, 0])
@pytest.mark.parametrize("g", [I.grid2d(24, 24), I.rgg2d(2000, 3), I.rmat(9, 2), I.star_graph(40),
                               I.path_graph(101)])
def test_structured_graphs(relabel, g, form):
    rng = np.random.default_rng(4)
    match, _ = O.greedy_matching(g, "expansion*2", 3)
    assert run_case(relabel, g, match, form, rng)
    unmatched = np.arange(g.n, dtype=np.int32)                 # nothing matched: cn = n
    assert run_case(relabel, g, unmatched, form, rng)
