"""Tuning knobs and the autotuner: every knob setting gives exactly the
oracle's hierarchy (the knobs change the time, never a result), the tuner's
candidates all agree with each other, and its choice is cached per GPU and
shape class."""
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


def gpu_levels(h):
    out = []
    for l in range(h.num_levels()):
        lv = h.level(l)
        out.append({k: lv[k].cpu().numpy() for k in ("xadj", "adjncy", "ewgt", "vwgt")})
        if lv["map"] is not None:
            out[-1]["map"] = lv["map"].cpu().numpy()
    return out


def same_as_oracle(levels, ref):
    assert len(levels) == len(ref.levels)
    for l, (a, b) in enumerate(zip(levels, ref.levels)):
        for key in ("xadj", "adjncy", "ewgt", "vwgt"):
            assert np.array_equal(a[key], getattr(b, key)), (l, key)
        if l < len(ref.maps):
            assert np.array_equal(a["map"], ref.maps[l]), (l, "map")


HUBS = [(lambda: I.rmat(13, 21, edge_factor=64), "expansion*2"), (lambda: I.rmat(14, 22), "innerOuter")]


@pytest.mark.parametrize("knob,values", [
    ("suitor_lanes", [1, 2, 4, 8, 32]),
    ("suitor_blocks", [3, 4]),
    ("radix_bits", [4, 5, 6, 7]),
    ("sort_shared_max", [128, 512, 1024]),
    ("tail_block_nodes", [256, 16384]),
    ("tail_nodes", [0x7fffffff, 1 << 12]),
    ("cluster_nodes", [-1, 64, 5000, 1 << 20]),
])
def test_every_knob_value_gives_the_oracle_hierarchy(knob, values):
    for make, rating in HUBS:
        g = make()
        ref = O.coarsen(g, rating, 3, 40)
        dg = B().DeviceGraph.from_csr(g)
        for v in values:
            for tail in ([0, -1] if knob != "tail_nodes" else [v]):
                kw = {"tail_nodes": tail, knob: v}
                h = B().coarsen(dg, rating=rating, seed=3, stop_size=40, **kw)
                same_as_oracle(gpu_levels(h), ref)
                h.free()


def test_radix_widths_on_mid_length_rows():
    """With a low sort_shared_max the radix class (LSD passes through global
    memory) also holds rows of 129..2048 entries: every radix width gives the
    oracle's hierarchy."""
    for make, rating in HUBS:
        g = make()
        ref = O.coarsen(g, rating, 3, 40)
        dg = B().DeviceGraph.from_csr(g)
        for rb in (4, 5, 7, 8):
            h = B().coarsen(dg, rating=rating, seed=3, stop_size=40, tail_nodes=-1, sort_shared_max=128, radix_bits=rb)
            same_as_oracle(gpu_levels(h), ref)
            h.free()


def test_bad_knob_values_are_rejected():
    dg = B().DeviceGraph.from_csr(I.grid2d(8, 8))
    for kw in [dict(suitor_lanes=3), dict(suitor_lanes=16), dict(radix_bits=3), dict(radix_bits=9), dict(sort_shared_max=64),
               dict(sort_shared_max=4096), dict(tail_block_nodes=100), dict(suitor_blocks=5)]:
        with pytest.raises(B().KpError) as e:
            B().coarsen(dg, **kw)
        assert e.value.status == B().KP_ERR_INVALID, kw


def test_autotune_candidates_agree_and_choice_is_cached(tmp_path):
    # a batch of uneven graphs, as the batched workload has
    graphs = [I.rgg2d(int(n), 50 + i, wmax=16) for i, n in enumerate(I.batch_rgg_sizes(24, 5, 1024, 8192))]
    graphs += [I.rmat(11, 7), I.grid2d(30, 31)]
    U, off = I.union_graph(graphs)
    seeds = np.arange(len(graphs), dtype=np.uint64) + 9
    dg = B().DeviceGraph.from_csr(U)
    cache = str(tmp_path / "tune.json")
    knobs, trials, cached = B().autotune(dg, off, seeds, reps=1, cache=cache, stop_size=40)
    assert not cached and len(trials) >= 10
    ref = None
    for kn, ms in trials:
        assert ms > 0
        kn = dict(kn)
        h = B().coarsen_batch(dg, off, seeds, stop_size=40, **kn)
        got = [gpu_levels(h), list(h.graph_levels())]
        h.free()
        if ref is None:
            ref = got
            # and the first candidate against the oracle, graph by graph
            hb = B().coarsen_batch(dg, off, seeds, stop_size=40, **kn)
            for gi, gr in enumerate(graphs):
                o = O.coarsen(gr, "expansion*2", int(seeds[gi]), 40)
                assert got[1][gi] == len(o.levels)
                for l in range(len(o.levels)):
                    lv = hb.graph_level(gi, l)
                    for key in ("xadj", "adjncy", "ewgt", "vwgt"):
                        assert np.array_equal(lv[key], getattr(o.levels[l], key)), (gi, l, key)
            hb.free()
            continue
        assert got[1] == ref[1], kn
        assert len(got[0]) == len(ref[0]), kn
        for a, b in zip(got[0], ref[0]):
            for key in a:
                assert np.array_equal(a[key], b[key]), (kn, key)
    again, trials2, cached2 = B().autotune(dg, off, seeds, reps=1, cache=cache, stop_size=40)
    assert cached2 and again == knobs and trials2 == []
