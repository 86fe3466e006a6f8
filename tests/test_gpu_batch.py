"""Batches of independent graphs (kp_coarsen_batch): every graph of a batch
must come out exactly as the oracle coarsens it alone, with its own seed and
graph-local ids, whatever else is in the batch."""
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


def mixed_graphs(seed):
    rng = np.random.default_rng(seed)
    gs = []
    for t in range(14):
        gs.append(I.random_small_graph(int(rng.integers(2, 120)), float(rng.uniform(0.02, 0.3)), seed=seed * 100 + t,
                                       wmax=int(rng.choice([1, 7, 300])), cmax=int(rng.choice([1, 5])),
                                       allow_zero_c=(t % 4 == 0)))
    gs += [I.grid2d(17, 9), I.grid3d(6, 5, 4), I.rgg2d(3000, seed, wmax=16), I.star_graph(300),
           I.path_graph(200), I.rmat(9, seed)]
    gs.append(I.from_edges(0, np.zeros(0, np.int64), np.zeros(0, np.int64)))     # empty graph
    gs.append(I.from_edges(25, np.zeros(0, np.int64), np.zeros(0, np.int64)))    # isolated nodes only
    gs.append(I.from_edges(2, np.array([0]), np.array([1])))                      # a single edge
    order = rng.permutation(len(gs))
    return [gs[i] for i in order]


def check_batch(graphs, seeds, rating, stop, matcher, tail, max_levels=64, stops=None):
    import torch
    U, off = I.union_graph(graphs)
    dg = B().DeviceGraph.from_csr(U)
    h = B().coarsen_batch(dg, off, seeds, stop_sizes=stops, rating=rating, stop_size=stop, matcher=matcher,
                          tail_nodes=tail, max_levels=max_levels)
    levels = h.graph_levels()
    refs = []
    for gi, g in enumerate(graphs):
        ref = O.coarsen(g, rating, int(seeds[gi]), stop if stops is None else int(stops[gi]), max_levels=max_levels)
        refs.append(ref)
        assert levels[gi] == len(ref.levels), (gi, g.name, levels[gi], [l.n for l in ref.levels])
        for l, rl in enumerate(ref.levels):
            got = h.graph_level(gi, l)
            for key in ("xadj", "adjncy", "ewgt", "vwgt"):
                assert np.array_equal(got[key], getattr(rl, key)), (gi, g.name, l, key)
            if l < len(ref.levels) - 1:
                assert np.array_equal(got["map"], ref.maps[l]), (gi, g.name, l, "map")
    return h, dg, refs, off


@pytest.mark.parametrize("tail", [0, -1])
@pytest.mark.parametrize("matcher", ["suitor", "handshake"])
@pytest.mark.parametrize("rating", ["expansion*2", "innerOuter"])
def test_mixed_batch_equals_each_graph_alone(rating, matcher, tail):
    graphs = mixed_graphs(3)
    seeds = np.arange(len(graphs), dtype=np.uint64) * 7919 + 5
    check_batch(graphs, seeds, rating, 6, matcher, tail)


def test_placement_does_not_matter_and_level_cap():
    graphs = mixed_graphs(8)
    seeds = np.arange(len(graphs), dtype=np.uint64) + 100
    check_batch(graphs, seeds, "expansion*2", 2, "suitor", 0)
    rev = list(reversed(graphs))
    check_batch(rev, seeds[::-1].copy(), "expansion*2", 2, "suitor", 0)
    check_batch(graphs, seeds, "weight", 2, "suitor", 0, max_levels=2)


@pytest.mark.parametrize("matcher", ["suitor", "handshake"])
def test_per_graph_stop_sizes(matcher):
    graphs = mixed_graphs(11)
    seeds = np.arange(len(graphs), dtype=np.uint64) * 31 + 2
    stops = np.random.default_rng(4).choice([1, 2, 6, 40, 1000], size=len(graphs)).astype(np.int32)
    check_batch(graphs, seeds, "expansion*2", 6, matcher, 0, stops=stops)
    check_batch(graphs, seeds, "innerOuter", 6, matcher, -1, stops=stops)


def test_rgg_batch_log_uniform_sizes_and_projection():
    """The batched workload's shape at a smaller scale: RGGs with n
    log-uniform, mean degree 6, integer weights in [1,16], expansion*2,
    stop at <= 40 nodes; then per-graph random balanced 2-way partitions of
    the coarsest graphs projected back."""
    import torch
    sizes = I.batch_rgg_sizes(48, seed=1, nmin=1024, nmax=8192)
    graphs = [I.rgg2d(int(n), 1000 + i, wmax=16) for i, n in enumerate(sizes)]
    seeds = np.arange(len(graphs), dtype=np.uint64)
    h, dg, refs, off = check_batch(graphs, seeds, "expansion*2", 40, "suitor", 0)
    assert list(h.coarsest_sizes()) == [ref.levels[-1].n for ref in refs]
    parts, coarse_off = [], [0]
    for gi, ref in enumerate(refs):
        p = I.random_balanced_partition(ref.levels[-1].n, 2, seed=gi)
        parts.append(p)
        coarse_off.append(coarse_off[-1] + len(p))
    cp = torch.as_tensor(np.concatenate(parts).astype(np.int32)).cuda()
    co = torch.as_tensor(np.array(coarse_off, dtype=np.int32)).cuda()
    fine = h.project(cp, co).cpu().numpy()
    for gi, ref in enumerate(refs):
        want = O.project(ref.maps, parts[gi])
        assert np.array_equal(fine[off[gi]:off[gi + 1]], want), gi


def test_batch_rejects_bad_input():
    import torch
    a, b = I.grid2d(4, 4), I.grid2d(3, 3)
    U, off = I.union_graph([a, b])
    dg = B().DeviceGraph.from_csr(U)
    with pytest.raises(B().KpError) as e:
        B().coarsen_batch(dg, np.array([0, 20, 25], dtype=np.int32))     # does not end at n
    assert e.value.status == B().KP_ERR_INVALID
    with pytest.raises(B().KpError) as e:
        B().coarsen_batch(dg, np.array([0, 10, 25], dtype=np.int32))     # edges cross graphs
    assert e.value.status == B().KP_ERR_INVALID


def test_saved_and_loaded_batch_hierarchy_is_identical(tmp_path):
    import torch
    graphs = mixed_graphs(21)
    seeds = np.arange(len(graphs), dtype=np.uint64) + 3
    h, dg, refs, off = check_batch(graphs, seeds, "innerOuter", 6, "suitor", 0)
    path = str(tmp_path / "batch.kph")
    h.save(path)
    h2 = B().load_hierarchy(path)
    assert h2.graph_levels() == h.graph_levels()
    assert list(h2.coarsest_sizes()) == list(h.coarsest_sizes())
    for gi, ref in enumerate(refs):
        for l, rl in enumerate(ref.levels):
            got = h2.graph_level(gi, l)
            for key in ("xadj", "adjncy", "ewgt", "vwgt"):
                assert np.array_equal(got[key], getattr(rl, key)), (gi, l, key)
    cs = h.coarsest_sizes()
    cp, co = I.batch_partition(cs, 3, 5)
    a = h.project(torch.as_tensor(cp).cuda(), torch.as_tensor(co).cuda()).cpu().numpy()
    b = h2.project(torch.as_tensor(cp).cuda(), torch.as_tensor(co).cuda()).cpu().numpy()
    assert np.array_equal(a, b)
    h2.free()
    # a damaged file is refused
    data = open(path, "rb").read()
    for bad in (data[:len(data) // 2], b"XXXXXXXX" + data[8:], data + b"\0"):
        p2 = str(tmp_path / "bad.kph")
        open(p2, "wb").write(bad)
        with pytest.raises(B().KpError) as e:
            B().load_hierarchy(p2)
        assert e.value.status == B().KP_ERR_INVALID
