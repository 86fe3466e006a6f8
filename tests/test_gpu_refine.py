"""Parity of the refinement helpers (Section 5) with the oracle: the quotient
graph of a partition and the bounded breadth-first search from the block
boundaries, bit-exact, on grids, RGGs, R-MAT graphs, random graphs, with
whole-graph and pair searches, at depths 0..20, and their error paths."""
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


def graphs():
    return [I.grid2d(37, 23), I.grid3d(9, 8, 7), I.rgg2d(4000, 3, wmax=9), I.rmat(11, 4), I.star_graph(500),
            I.path_graph(300), I.random_small_graph(90, 0.08, seed=3, wmax=5),
            I.from_edges(6, np.zeros(0, np.int64), np.zeros(0, np.int64))]


def partitions(g, seed):
    out = []
    for k in (1, 2, 5, 64):
        out.append((k, I.random_balanced_partition(g.n, k, seed=seed + k)))
    # a partition with spatial structure: contiguous id ranges
    k = 4
    out.append((k, np.minimum(np.arange(g.n) * k // max(g.n, 1), k - 1).astype(np.int32)))
    return out


def test_quotient_graph_equals_oracle():
    import torch
    for gi, g in enumerate(graphs()):
        dg = B().DeviceGraph.from_csr(g)
        for k, part in partitions(g, gi):
            q_xadj, q_adj, q_w = B().quotient_graph(dg, torch.as_tensor(part).cuda(), k)
            wx, wa, ww = O.quotient_graph(g, part, k)
            assert np.array_equal(q_xadj.cpu().numpy(), wx), (g.name, k)
            assert np.array_equal(q_adj.cpu().numpy(), wa), (g.name, k)
            assert np.array_equal(q_w.cpu().numpy(), ww), (g.name, k)


def test_quotient_graph_capacity_and_errors():
    import torch
    g = I.grid2d(20, 20)
    dg = B().DeviceGraph.from_csr(g)
    part = torch.as_tensor(I.random_partition(g.n, 30, seed=1)).cuda()
    want = O.quotient_graph(g, part.cpu().numpy(), 30)
    q_xadj = torch.empty(31, dtype=torch.int32, device="cuda")
    q_adj = torch.empty(4, dtype=torch.int32, device="cuda")
    q_w = torch.empty(4, dtype=torch.int64, device="cuda")
    got = B().kp_quotient_graph(dg.kp, part.data_ptr(), 30, q_xadj.data_ptr(), q_adj.data_ptr(), q_w.data_ptr(), 4,
                                B().current_stream())
    assert got == -len(want[1]) - 1            # overflow reports the size needed
    assert np.array_equal(q_xadj.cpu().numpy(), want[0])
    with pytest.raises(B().KpError) as e:
        B().quotient_graph(dg, torch.full((g.n,), 30, dtype=torch.int32, device="cuda"), 30)
    assert e.value.status == B().KP_ERR_INVALID
    with pytest.raises(B().KpError) as e:
        B().quotient_graph(dg, part, 5000)
    assert e.value.status == B().KP_ERR_UNSUPPORTED


@pytest.mark.parametrize("depth", [0, 1, 5, 20])
def test_boundary_band_equals_oracle(depth):
    import torch
    for gi, g in enumerate(graphs()):
        dg = B().DeviceGraph.from_csr(g)
        for k, part in partitions(g, 10 + gi):
            tp = torch.as_tensor(part).cuda()
            got = B().boundary_band(dg, tp, k, depth).cpu().numpy()
            assert np.array_equal(got, O.boundary_band(g, part, depth)), (g.name, k, depth)
            if k >= 2:
                pair = (0, k - 1)
                got = B().boundary_band(dg, tp, k, depth, pair=pair).cpu().numpy()
                assert np.array_equal(got, O.boundary_band(g, part, depth, pair=pair)), (g.name, k, depth, "pair")


def test_boundary_band_large_and_errors():
    import torch
    g = I.rgg2d(200000, 5)
    dg = B().DeviceGraph.from_csr(g)
    # a partition with real bands: a random 8-way partition of the coarsest
    # graph projected back (a random fine partition is boundary almost
    # everywhere)
    h = B().coarsen(dg, stop_size=160)
    top = B().kp_hierarchy_level(h.handle, h.num_levels() - 1)[0].n
    tp = h.project(torch.as_tensor(I.random_balanced_partition(top, 8, seed=2)).cuda())
    part = tp.cpu().numpy()
    h.free()
    want = O.boundary_band(g, part, 20)
    assert (want > 3).sum() > 1000   # a band, not only boundary nodes
    assert np.array_equal(B().boundary_band(dg, tp, 8, 20).cpu().numpy(), want)
    assert np.array_equal(B().boundary_band(dg, tp, 8, 5, pair=(1, 6)).cpu().numpy(),
                          O.boundary_band(g, part, 5, pair=(1, 6)))
    for depth, pair in [(-1, None), (3, (0, 0)), (3, (0, 9)), (3, (0, -1))]:
        with pytest.raises(B().KpError) as e:
            B().boundary_band(dg, tp, 8, depth, pair=pair)
        assert e.value.status == B().KP_ERR_INVALID, (depth, pair)
