"""The library's one-thread contraction of a coarse row (Section 2: the
entries of a matched pair gathered, the pair's own edge dropped, parallel
edges summed into a sorted row), compiled by the host compiler and run on
the CPU (CPU only).  contract_thread<16> serves every coarse row of at most
16 gathered entries and contract_thread<32> those of 17..32, so together
they build most coarse rows of meshes and geometric graphs.

Its register sorting network is proven by the 0-1 principle (a comparator
network sorts every input if it sorts every sequence of 0s and 1s): every one
of the 2^16 patterns of two coarse ids over 16 entries is checked, which
covers each 0-1 input of the 16-entry network.  The 32-entry network is
checked on random rows, 0-1 patterns among them.  Expected rows follow the
definition: a sum per coarse neighbour, ascending ids, the row's own id
dropped, Out' the total kept weight."""
import numpy as np
import pytest

from tests.test_exact_compare_host import host_program


@pytest.fixture(scope="module")
def contract(tmp_path_factory):
    return host_program("contract_row.cpp", str(tmp_path_factory.mktemp("hostcc") / "contract_row"))


def query(T, x, keys, weights, da, gap):
    body = " ".join(f"{k} {w}" for k, w in zip(keys, weights))
    return f"{T} {x} {da} {len(keys) - da} {gap} {body}".strip()


def expected(x, keys, weights):
    sums = {}
    for k, w in zip(keys, weights):
        if k != x:
            sums[k] = sums.get(k, 0) + w
    row = sorted(sums.items())
    return [len(row), sum(s for _, s in row)] + [v for kv in row for v in kv]


def check(contract, rows):
    got = contract([query(*r) for r in rows])
    want = []
    for T, x, keys, weights, da, gap in rows:
        want += expected(x, keys, weights)
    if got != want:   # find the first row that differs
        pos = 0
        for r in rows:
            e = expected(r[1], r[2], r[3])
            if got[pos:pos + len(e)] != e:
                pytest.fail(f"row {r}: got {got[pos:pos + len(e)]}, want {e}")
            pos += len(e)
        pytest.fail("output length differs")


def test_every_two_id_pattern_of_16_entries(contract):
    """All 2^16 placements of coarse ids 10 and 11 over a full 16-entry row
    (weights distinct, the members split 7 + 9 with a gap between them)."""
    w = [i + 1 for i in range(16)]
    rows = [(16, 0, [10 + ((m >> i) & 1) for i in range(16)], w, 7, 5) for m in range(1 << 16)]
    check(contract, rows)


@pytest.mark.parametrize("T", [16, 32])
def test_random_rows(contract, T):
    """Rows of 0..T entries with few distinct ids (many parallel edges), some
    entries mapped to the row itself (the contracted edge), either member
    empty, weights up to 2^24 (sums stay in int32)."""
    rng = np.random.default_rng(T)
    rows = []
    for t in range(20000):
        n = int(rng.integers(0, T + 1))
        x = int(rng.integers(0, 40))
        ids = int(rng.choice([1, 2, 3, 8, 40]))
        keys = [int(k) for k in rng.integers(0, ids, size=n) + (x if t % 5 == 0 else 0)]
        if t % 3 == 0 and n:
            keys[int(rng.integers(n))] = x
        weights = [int(v) for v in rng.integers(1, 1 << int(rng.choice([1, 8, 24])), size=n)]
        da = int(rng.integers(0, n + 1))
        rows.append((T, x, keys, weights, da, int(rng.integers(0, 4))))
    check(contract, rows)


def test_random_two_id_patterns_of_32_entries(contract):
    rng = np.random.default_rng(5)
    rows = []
    for _ in range(30000):
        m = int(rng.integers(0, 1 << 32, dtype=np.uint64))
        rows.append((32, 3, [7 + ((m >> i) & 1) for i in range(32)], [i + 1 for i in range(32)], 16, 2))
    check(contract, rows)


def test_large_ids_and_the_sentinel_boundary(contract):
    """Coarse ids up to 2^31 - 2 (the sentinel is 2^31 - 1 and sorts last),
    empty rows and rows whose every entry is the contracted edge."""
    big = (1 << 31) - 2
    rows = [(16, 1, [big, 5, big, 0, big - 1], [1, 2, 3, 4, 5], 2, 0),
            (32, 7, [big] * 20 + [big - 1] * 11 + [7], list(range(1, 33)), 20, 1),
            (16, 4, [big - k for k in range(16)], [1] * 16, 8, 3),
            (16, 0, [], [], 0, 0), (32, 9, [9] * 32, [1] * 32, 0, 0), (16, 2, [2] * 5, [3] * 5, 5, 0)]
    check(contract, rows)
