"""The library's exact rating comparison, tie-break hash, strict edge order
and Suitor eligibility test, the functions every matching decision of the
GPU path goes through, compiled by the host compiler and run on the CPU (CPU
only).

cmp_frac compares two ratings num/den (Section 3.1; a zero denominator is
+infinity, two infinities are equal) by 128-bit cross products, with a
shortcut of single widening multiplies when all four terms fit 32 bits.  The
parity graphs keep weights small, so products beyond 64 bits and the switch
between the two forms are checked here instead: against Python's exact
fractions on random and boundary cases, in both builds of the function (with
the shortcut, and the 128-bit form alone as the persistent tail compiles it).
The hash is checked against the published splitmix64 vectors and the
oracle's independent implementation, and the order of two candidate edges
of a node (rating_ab and better) and the test whether an edge beats the
standing offer at its other end (eligible_at, which rebuilds the standing
edge from the 16-byte offer record and hashes it only on equal ratings)
against the oracle's edge order for all five ratings."""
import math
import os
import shutil
import subprocess
from fractions import Fraction

import numpy as np
import pytest

import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HERE = os.path.join(ROOT, "tests", "hostcc")
GAMMA = 0x9E3779B97F4A7C15


def _cuda_include():
    for d in (os.environ.get("CUDA_HOME", ""), "/usr/local/cuda"):
        if d and os.path.exists(os.path.join(d, "include", "cuda_runtime.h")):
            return os.path.join(d, "include")
    return None


def host_program(source: str, exe: str, defines=()):
    """Builds tests/hostcc/<source> with g++ against the library's headers
    and the stand-ins; returns run(lines) -> the integers it prints."""
    inc = _cuda_include()
    if shutil.which("g++") is None or inc is None:
        pytest.skip("needs g++ and the CUDA headers")
    cmd = ["g++", "-std=c++17", "-O1", "-Wno-attributes", *[f"-D{d}" for d in defines],
           "-include", os.path.join(HERE, "cuda_stubs.h"), "-I", os.path.join(ROOT, "include"),
           "-I", os.path.join(ROOT, "paper_0910_2004_gb300", "csrc"), "-I", inc, os.path.join(HERE, source),
           "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]

    def run(lines):
        out = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True, timeout=300)
        assert out.returncode == 0, out.stderr
        return [int(x) for x in out.stdout.split()]

    return run


@pytest.fixture(scope="module", params=["shortcut", "wide_only"])
def harness(request, tmp_path_factory):
    exe = str(tmp_path_factory.mktemp("hostcc") / f"exact_compare_{request.param}")
    return host_program("exact_compare.cpp", exe, ["KP_FRAC_WIDE_ONLY"] if request.param == "wide_only" else [])


def rating(num: int, den: int):
    return math.inf if den == 0 else Fraction(num, den)


def expected(a, b, c, d):
    x, y = rating(a, b), rating(c, d)
    return (x > y) - (x < y)


def cases(seed: int, count: int):
    """(num, den) pairs the ratings can produce: numerators in [1, 2^62]
    (expansion*2: omega^2 with omega < 2^31), denominators in [0, 2^62]
    (products of two node weights below 2^31), mixed with small values and
    the 32-bit boundary."""
    rng = np.random.default_rng(seed)
    edges = [1, 2, 3, (1 << 31) - 1, (1 << 32) - 1, 1 << 32, (1 << 32) + 1, (1 << 62) - 1, 1 << 62]
    out = []
    for _ in range(count):
        pick = []
        for lo in (1, 0):
            kind = int(rng.integers(4))
            if kind == 0:
                v = int(rng.integers(lo, 1 << 16))
            elif kind == 1:
                v = int(rng.integers(lo, 1 << 32))
            elif kind == 2:
                v = int(rng.integers(lo, (1 << 62) + 1, dtype=np.uint64))
            else:
                v = int(rng.choice(edges))
            pick.append(max(v, lo))
        out.append(tuple(pick))
    return out


def test_cmp_frac_equals_exact_fractions(harness):
    fr = cases(1, 4000)
    pairs = [(fr[i], fr[i + 1]) for i in range(0, len(fr) - 1, 2)]
    # equal fractions in other terms (a*k / b*k), near-equal ones, and infinities
    rng = np.random.default_rng(2)
    for _ in range(1000):
        a, b = int(rng.integers(1, 1 << 31)), int(rng.integers(1, 1 << 31))
        k = int(rng.integers(1, 1 << 31))
        pairs.append(((a, b), (a * k, b * k)))
        pairs.append(((a * k, b * k + 1), (a, b)))
        pairs.append(((a * k + 1, b * k), (a, b)))
    pairs += [((5, 0), (7, 0)), ((1, 0), ((1 << 62), 1)), (((1 << 62), (1 << 62)), (1, 1)),
              (((1 << 62), (1 << 62) - 1), ((1 << 62) - 1, (1 << 62) - 2)), (((1 << 32) - 1, 1), (1 << 32, 1))]
    lines = [f"c {a} {b} {c} {d}" for (a, b), (c, d) in pairs]
    got = harness(lines)
    want = [expected(a, b, c, d) for (a, b), (c, d) in pairs]
    bad = [(p, g, w) for p, g, w in zip(pairs, got, want) if g != w]
    assert not bad, bad[:5]
    # antisymmetric
    got_rev = harness([f"c {c} {d} {a} {b}" for (a, b), (c, d) in pairs])
    assert got_rev == [-x for x in got]


def test_hash_matches_the_published_vectors_and_the_oracle(harness):
    gold = [l.split() for l in open(os.path.join(ROOT, "tests", "golden", "splitmix64_seed0.txt"))
            if l.strip() and not l.startswith("#")]
    got = harness([f"s {(int(i) * GAMMA) % (1 << 64)}" for i, _ in gold])
    assert got == [int(h, 16) for _, h in gold]
    rng = np.random.default_rng(3)
    q = [(int(rng.integers(0, 1 << 63, dtype=np.uint64)) * 2 + int(rng.integers(2)),
          int(rng.integers(0, 1 << 31)), int(rng.integers(0, 1 << 31))) for _ in range(2000)]
    q += [(0, 0, 1), (0, 1, 0), ((1 << 64) - 1, (1 << 31) - 1, 0)]
    got = harness([f"h {s} {u} {v}" for s, u, v in q])
    assert got == [O.edge_hash(s, u, v) for s, u, v in q]


RATING_IDS = {"expansion*2": 0, "innerOuter": 1, "weight": 2, "expansion": 3, "expansion*": 4}


@pytest.mark.parametrize("rating", list(RATING_IDS))
def test_candidate_order_equals_the_oracle_edge_order(harness, rating):
    """Two edges {v,u1}, {v,u2} at a node v: the GPU's candidate order agrees
    with the oracle's strict order, both ways round.  Small weight, node
    weight and Out ranges make equal ratings common, so the hash decides many
    pairs; zero node weights give infinite ratings."""
    rng = np.random.default_rng(10 + RATING_IDS[rating])
    n = 64
    queries, expect = [], []
    for t in range(3000):
        wmax = [2, 5, 1 << 20, (1 << 31) - 1][t % 4]
        vw = rng.integers(0 if t % 3 == 0 else 1, [3, 50, 1 << 15, (1 << 31) - 1][t % 4], size=n).astype(np.int64)
        v, u1, u2 = (int(x) for x in rng.choice(n, size=3, replace=False))
        w1, w2 = int(rng.integers(1, wmax + 1)), int(rng.integers(1, wmax + 1))
        # Out(x) is at least the weight of any edge at x (innerOuter's denominator stays >= 0)
        out = (max(w1, w2) + rng.integers(0, [3, 50, 1 << 20, 1 << 20][t % 4], size=n)).astype(np.int64)
        if rating == "innerOuter":
            out = np.minimum(out, (1 << 31) - 1)
            attr = out
        else:
            attr = vw
        seed = int(rng.integers(0, 1 << 63, dtype=np.uint64))
        queries.append(f"b {RATING_IDS[rating]} {seed} {v} {u1} {w1} {u2} {w2} {attr[v]} {attr[u1]} {attr[u2]}")
        o = O.edge_order(rating, seed, vw.astype(np.int32), out, (v, u1, w1), (v, u2, w2))
        expect += [int(o == 1), int(o == -1)]
    assert harness(queries) == expect


@pytest.mark.parametrize("rating", list(RATING_IDS))
def test_suitor_eligibility_equals_the_oracle_edge_order(harness, rating):
    """cur may offer {cur,v} to v iff v holds no offer or {cur,v} comes before
    the standing edge {s,v} in the strict order."""
    rng = np.random.default_rng(20 + RATING_IDS[rating])
    n = 64
    queries, expect = [], []
    for t in range(3000):
        wmax = [2, 5, 1 << 20, (1 << 31) - 1][t % 4]
        vw = rng.integers(0 if t % 3 == 0 else 1, [3, 50, 1 << 15, (1 << 31) - 1][t % 4], size=n).astype(np.int64)
        cur, v, s = (int(x) for x in rng.choice(n, size=3, replace=False))
        w, ws = int(rng.integers(1, wmax + 1)), int(rng.integers(1, wmax + 1))
        out = np.minimum(max(w, ws) + rng.integers(0, [3, 50, 1 << 20, 1 << 20][t % 4], size=n),
                         (1 << 31) - 1).astype(np.int64)
        attr = out if rating == "innerOuter" else vw
        seed = int(rng.integers(0, 1 << 63, dtype=np.uint64))
        none = t % 10 == 0
        queries.append(f"e {RATING_IDS[rating]} {seed} {cur} {v} {w} {-1 if none else s} {ws} "
                       f"{attr[cur]} {attr[s]} {attr[v]}")
        if none:
            expect.append(1)
        else:
            o = O.edge_order(rating, seed, vw.astype(np.int32), out, (cur, v, w), (s, v, ws))
            expect.append(int(o == 1))
    assert harness(queries) == expect


@pytest.mark.parametrize("rating", list(RATING_IDS))
def test_gpa_edge_order_equals_the_oracle_edge_order(harness, rating):
    """The Global Path Algorithm compares edges that need not share a node
    (gedge_before): the same strict order, both ways round, and an edge is
    never before itself."""
    rng = np.random.default_rng(30 + RATING_IDS[rating])
    n = 40
    queries, expect = [], []
    for t in range(3000):
        wmax = [2, 5, 1 << 20, (1 << 31) - 1][t % 4]
        vw = rng.integers(0 if t % 3 == 0 else 1, [3, 50, 1 << 15, (1 << 31) - 1][t % 4], size=n).astype(np.int64)
        x1, y1 = (int(x) for x in rng.choice(n, size=2, replace=False))
        if t % 7 == 0:
            x2, y2 = y1, x1                                  # the same edge seen from its other end
        else:
            x2, y2 = (int(x) for x in rng.choice(n, size=2, replace=False))
        w1 = int(rng.integers(1, wmax + 1))
        w2 = w1 if {x1, y1} == {x2, y2} else int(rng.integers(1, wmax + 1))
        out = np.minimum(max(w1, w2) + rng.integers(0, [3, 50, 1 << 20, 1 << 20][t % 4], size=n),
                         (1 << 31) - 1).astype(np.int64)
        attr = out if rating == "innerOuter" else vw
        seed = int(rng.integers(0, 1 << 63, dtype=np.uint64))
        queries.append(f"g {RATING_IDS[rating]} {seed} {x1} {y1} {w1} {attr[x1]} {attr[y1]} "
                       f"{x2} {y2} {w2} {attr[x2]} {attr[y2]}")
        o = O.edge_order(rating, seed, vw.astype(np.int32), out, (x1, y1, w1), (x2, y2, w2))
        expect += [int(o == 1), int(o == -1)]
    assert harness(queries) == expect
