"""Parity of the GPU Global Path Algorithm (matcher "gpa", Section 3.2) with
the oracle's sequential one: every level's CSR, node weights and map, the
projected partition and the cut/gain, exactly, for every rating; ragged,
degenerate and power-law graphs; batches (every graph as alone) and recorded
plans; the RGG 2^20 workload at full size."""
import numpy as np
import pytest

import oracle as O
from paper_0910_2004_gb300 import inputs as I

pytestmark = pytest.mark.gpu

RATINGS = ["expansion*2", "innerOuter", "weight", "expansion", "expansion*"]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


def B():
    from paper_0910_2004_gb300 import binding
    return binding


def gpu_levels(h):
    levels, maps = [], []
    for l in range(h.num_levels()):
        lv = h.level(l)
        levels.append(O.Level(lv["xadj"].cpu().numpy(), lv["adjncy"].cpu().numpy(), lv["ewgt"].cpu().numpy(),
                              lv["vwgt"].cpu().numpy()))
        if lv["map"] is not None:
            maps.append(lv["map"].cpu().numpy())
    return levels, maps


def assert_same(levels, maps, ref, where=""):
    assert len(levels) == len(ref.levels), (where, [l.n for l in levels], [l.n for l in ref.levels])
    for l, (a, b) in enumerate(zip(levels, ref.levels)):
        for key in ("xadj", "adjncy", "ewgt", "vwgt"):
            assert np.array_equal(getattr(a, key), getattr(b, key)), (where, l, key)
    for l, (a, b) in enumerate(zip(maps, ref.maps)):
        assert np.array_equal(a, b), (where, l, "map")


def gpa_path(g, rating, seed, stop, k=None, eps=0.03):
    import torch
    dg = B().DeviceGraph.from_csr(g)
    h = B().coarsen(dg, rating=rating, seed=seed, stop_size=stop, matcher="gpa")
    levels, maps = gpu_levels(h)
    ref = O.coarsen(g, rating, seed, stop, matcher="gpa")
    assert_same(levels, maps, ref, g.name)
    if k:
        cpart = I.random_balanced_partition(ref.levels[-1].n, k, seed=1)
        fine = h.project(torch.as_tensor(cpart).cuda()).cpu().numpy()
        want = O.project(ref.maps, cpart)
        assert np.array_equal(fine, want)
        got = B().cut_gain(dg, torch.as_tensor(want).cuda(), k, eps)
        exp = O.cut_gain(g, want, k, eps)
        for key in ("cut", "L_max", "imbalance"):
            assert got[key] == exp[key], key
        for key in ("block_w", "gain", "target"):
            assert np.array_equal(got[key].cpu().numpy(), exp[key]), key
    h.free()
    return ref


@pytest.mark.parametrize("rating", RATINGS)
def test_random_graphs(rating):
    for t in range(30):
        rng = np.random.default_rng(700 + t)
        n = int(rng.integers(2, 400))
        g = I.random_small_graph(n, float(rng.uniform(0.005, 0.25)), seed=900 + t,
                                 wmax=int(rng.choice([1, 5, 1000])), cmax=int(rng.choice([1, 4, 50])),
                                 allow_zero_c=(t % 5 == 0))
        gpa_path(g, rating, int(rng.integers(0, 2**63)), int(rng.choice([1, 10, 50])))


@pytest.mark.parametrize("rating", ["expansion*2", "innerOuter", "weight"])
def test_structured_graphs(rating):
    """Grids (many equal ratings: long paths and even cycles), RGG, R-MAT
    hubs, a long path with increasing weights, stars and odd cycles."""
    lo = np.arange(9)
    cycle9 = I.from_edges(9, lo, (lo + 1) % 9, np.arange(1, 10), name="cycle9")
    lo = np.arange(12)
    cycle12 = I.from_edges(12, lo, (lo + 1) % 12, np.array([3, 1, 4, 1, 5, 9, 2, 6, 5, 3, 5, 8]), name="cycle12")
    # R-MAT 2^15 and the star: rows above 2048 entries, rated by a block each
    for g in [I.grid2d(64, 64), I.grid3d(20, 17, 9), I.rgg2d(1 << 16, 3, wmax=16), I.rmat(13, 5), I.rmat(15, 3),
              I.path_graph(3000), I.star_graph(3000), cycle9, cycle12]:
        gpa_path(g, rating, 7, 20, k=5)


def test_tiny_and_degenerate():
    for g in [I.from_edges(1, np.zeros(0, np.int64), np.zeros(0, np.int64)),
              I.from_edges(30, np.zeros(0, np.int64), np.zeros(0, np.int64)),
              I.from_edges(2, np.array([0]), np.array([1])),
              I.from_edges(6, np.array([0, 2, 3]), np.array([1, 3, 4]), np.array([1, 50, 60]))]:
        for r in RATINGS:
            gpa_path(g, r, 1, 0)
    # zero node weights: +infinity ratings, whose double sums stay +infinity
    gpa_path(I.random_small_graph(300, 0.05, 9, cmax=2, allow_zero_c=True), "expansion*2", 5, 3, k=4)


def test_rgg_2pow20_full_size():
    """The RGG workload's graph (n = 2^20, mean degree 6), expansion*2, down
    to <= 20*64 nodes, k = 64."""
    gpa_path(I.rgg2d(1 << 20, 1), "expansion*2", 1, 20 * 64, k=64)


def test_batch_each_graph_as_alone():
    graphs = [I.rgg2d(3000 + 500 * i, 40 + i, wmax=16) for i in range(6)]
    graphs += [I.grid2d(17, 9), I.path_graph(200), I.star_graph(300), I.rmat(9, 2),
               I.from_edges(25, np.zeros(0, np.int64), np.zeros(0, np.int64))]
    U, off = I.union_graph(graphs)
    seeds = np.arange(len(graphs), dtype=np.uint64) * 13 + 1
    dg = B().DeviceGraph.from_csr(U)
    for rating in ["expansion*2", "innerOuter"]:
        h = B().coarsen_batch(dg, off, seeds, rating=rating, stop_size=6, matcher="gpa")
        levels = h.graph_levels()
        for gi, g in enumerate(graphs):
            ref = O.coarsen(g, rating, int(seeds[gi]), 6, matcher="gpa")
            assert levels[gi] == len(ref.levels), (gi, rating)
            for l, rl in enumerate(ref.levels):
                got = h.graph_level(gi, l)
                for key in ("xadj", "adjncy", "ewgt", "vwgt"):
                    assert np.array_equal(got[key], getattr(rl, key)), (gi, l, key)
                if l < len(ref.levels) - 1:
                    assert np.array_equal(got["map"], ref.maps[l]), (gi, l, "map")
        h.free()


def test_recorded_plan_equals_the_oracle():
    g = I.rgg2d(20000, 8, wmax=16)
    dg = B().DeviceGraph.from_csr(g)
    ref = O.coarsen(g, "expansion*2", 3, 40, matcher="gpa")
    with B().Plan(dg, rating="expansion*2", seed=3, stop_size=40, matcher="gpa") as plan:
        for _ in range(2):
            levels, maps = gpu_levels(plan.run())
            assert_same(levels, maps, ref, "plan")
