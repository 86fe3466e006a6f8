"""Captured plans (kp_plan_*): the whole hierarchy in one persistent launch
recorded into a CUDA graph; every replay equals the oracle, also after the
inputs' contents change in place and when the arena has to grow."""
import numpy as np
import pytest

import oracle as O
from paper_0910_2004_gb300 import inputs as I

pytestmark = pytest.mark.gpu


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


def check_graph(h, gi, g, ref):
    assert h.graph_levels()[gi] == len(ref.levels)
    for l, rl in enumerate(ref.levels):
        got = h.graph_level(gi, l)
        for key in ("xadj", "adjncy", "ewgt", "vwgt"):
            assert np.array_equal(got[key], getattr(rl, key)), (gi, l, key)
        if l < len(ref.levels) - 1:
            assert np.array_equal(got["map"], ref.maps[l]), (gi, l, "map")


@pytest.mark.parametrize("tail", [0, 0x7fffffff, -1, 2000])
@pytest.mark.parametrize("matcher", ["suitor", "handshake"])
@pytest.mark.parametrize("rating", ["expansion*2", "innerOuter"])
def test_batch_plan_replays_equal_oracle(rating, matcher, tail):
    import torch
    graphs = [I.rgg2d(int(n), 70 + i, wmax=16) for i, n in enumerate(I.batch_rgg_sizes(20, 3, 1024, 6000))]
    graphs += [I.rmat(10, 3), I.grid2d(17, 5), I.star_graph(200),
               I.from_edges(5, np.zeros(0, np.int64), np.zeros(0, np.int64))]
    U, off = I.union_graph(graphs)
    seeds = np.arange(len(graphs), dtype=np.uint64) * 3 + 1
    stops = np.where(np.arange(len(graphs)) % 3 == 0, 8, 40).astype(np.int32)
    dg = B().DeviceGraph.from_csr(U)
    refs = [O.coarsen(g, rating, int(seeds[i]), int(stops[i])) for i, g in enumerate(graphs)]
    with B().Plan(dg, off, seeds, stops, rating=rating, matcher=matcher, tail_nodes=tail) as plan:
        for rep in range(3):
            h = plan.run()
            for gi, g in enumerate(graphs):
                check_graph(h, gi, g, refs[gi])
        # new edge weights in place (same structure): the next replay reads them
        rng = np.random.default_rng(1)
        new_graphs = []
        for g in graphs:
            src = np.repeat(np.arange(g.n), np.diff(g.xadj))
            lo, hi = np.minimum(src, g.adjncy), np.maximum(src, g.adjncy)
            key = lo.astype(np.int64) * max(g.n, 1) + hi
            uniq, inv = np.unique(key, return_inverse=True)
            ew = rng.integers(1, 9, size=max(len(uniq), 1))[inv].astype(np.int32)
            new_graphs.append(I.CSRGraph(g.xadj, g.adjncy, ew, g.vwgt, g.name))
        U2, _ = I.union_graph(new_graphs)
        dg.ewgt.copy_(torch.as_tensor(U2.ewgt).cuda())
        h = plan.run()
        for gi, g in enumerate(new_graphs):
            check_graph(h, gi, g, O.coarsen(g, rating, int(seeds[gi]), int(stops[gi])))


def test_single_graph_plan_and_arena_growth():
    g = I.rgg2d(30000, 4, wmax=16)
    ref = O.coarsen(g, "innerOuter", 2, 40)
    dg = B().DeviceGraph.from_csr(g)
    # an arena far too small: the first replay grows it and runs again
    with B().Plan(dg, rating="innerOuter", seed=2, stop_size=40, arena_bytes=4096) as plan:
        for rep in range(2):
            h = plan.run()
            assert h.num_levels() == len(ref.levels)
            for l, rl in enumerate(ref.levels):
                lv = h.level(l)
                for key in ("xadj", "adjncy", "ewgt", "vwgt"):
                    assert np.array_equal(lv[key].cpu().numpy(), getattr(rl, key)), (l, key)
    small = I.grid2d(4, 4)     # below the stop size: the plan returns the input only
    with B().Plan(B().DeviceGraph.from_csr(small), stop_size=40) as plan:
        assert plan.run().num_levels() == 1
