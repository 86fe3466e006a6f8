"""Parity of the CUDA path (through the C ABI) with the oracle.

All arithmetic is integer, so every comparison is exact: each level's CSR,
node weights and map, the projected partition, the cut, block weights, L_max,
imbalance, gains and targets.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_0910_2004_gb300 import inputs as I

pytestmark = pytest.mark.gpu

RATINGS = ["expansion*2", "innerOuter", "weight", "expansion", "expansion*"]
MATCHERS = ["suitor", "handshake"]


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


def run_gpu(g, **opts):
    import torch
    dg = B().DeviceGraph.from_csr(g)
    h = B().coarsen(dg, **opts)
    levels, maps = [], []
    for l in range(h.num_levels()):
        lv = h.level(l)
        levels.append(O.Level(lv["xadj"].cpu().numpy(), lv["adjncy"].cpu().numpy(),
                              lv["ewgt"].cpu().numpy(), lv["vwgt"].cpu().numpy()))
        assert lv["nnz"] == levels[-1].nnz
        if lv["map"] is not None:
            maps.append(lv["map"].cpu().numpy())
    torch.cuda.synchronize()
    return h, dg, levels, maps


def assert_same(levels, maps, ref, where=""):
    assert len(levels) == len(ref.levels), (where, [l.n for l in levels], [l.n for l in ref.levels])
    for l, (a, b) in enumerate(zip(levels, ref.levels)):
        for key in ("xadj", "adjncy", "ewgt", "vwgt"):
            assert np.array_equal(getattr(a, key), getattr(b, key)), (where, l, key)
    for l, (a, b) in enumerate(zip(maps, ref.maps)):
        assert np.array_equal(a, b), (where, l, "map")


def check_eval(dg, g, part, k, eps):
    import torch
    got = B().cut_gain(dg, torch.as_tensor(part).cuda(), k, eps)
    want = O.cut_gain(g, part, k, eps)
    for key in ("cut", "L_max", "imbalance"):
        assert got[key] == want[key], key
    assert got["total_c"] == int(g.vwgt.astype(np.int64).sum())
    assert np.array_equal(got["block_w"].cpu().numpy(), want["block_w"])
    assert np.array_equal(got["gain"].cpu().numpy(), want["gain"])
    assert np.array_equal(got["target"].cpu().numpy(), want["target"])
    return got


def full_path(g, rating, seed, stop, k, eps=0.03, part_seed=1, matcher="suitor", tail=0):
    import torch
    h, dg, levels, maps = run_gpu(g, rating=rating, seed=seed, stop_size=stop, matcher=matcher, tail_nodes=tail)
    ref = O.coarsen(g, rating, seed, stop)
    assert_same(levels, maps, ref, g.name)
    cpart = I.random_balanced_partition(ref.levels[-1].n, k, seed=part_seed)
    fine = h.project(torch.as_tensor(cpart).cuda())
    want = O.project(ref.maps, cpart)
    assert np.array_equal(fine.cpu().numpy(), want)
    check_eval(dg, g, want, k, eps)
    h.free()
    return ref


# ---------------------------------------------------------------------------
# the measured workloads
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("matcher", MATCHERS)
def test_grid64_expansion_star2_k2(matcher):
    """2D 5-point grid 64x64, expansion*2, stop at <= 20k nodes, k=2."""
    ref = full_path(I.grid2d(64, 64), "expansion*2", 1, 40, 2, matcher=matcher)
    assert ref.levels[-1].n <= 40


@pytest.mark.parametrize("matcher", MATCHERS)
def test_rgg_2pow20_full_size(matcher):
    """2D RGG, n=2^20, mean degree 6, expansion*2, stop <= 20*64, k=64."""
    g = I.rgg2d(1 << 20, 1)
    full_path(g, "expansion*2", 1, 20 * 64, 64, matcher=matcher)


@pytest.mark.slow
def test_grid3d_256_full_size_levelwise():
    _grid3d_levelwise("suitor")


@pytest.mark.slow
def test_grid3d_256_full_size_levelwise_handshake():
    _grid3d_levelwise("handshake")


def _grid3d_levelwise(matcher):
    """3D 7-point grid 256^3, innerOuter, stop <= 20*256, k=256.  The oracle's
    Greedy sort is slow at this size, so every level is checked with the
    sort-free characterisation of the Greedy matching and the oracle's
    contraction, and the evaluation against the oracle's cut/gain."""
    import torch
    g = I.grid3d(256, 256, 256)
    h, dg, levels, maps = run_gpu(g, rating="innerOuter", seed=1, stop_size=20 * 256, validate=False,
                                  matcher=matcher)
    for l, mp in enumerate(maps):
        cur = levels[l]
        match = match_from_map(mp)
        assert O.check_greedy_matching(cur, "innerOuter", 1, match) == -1, l
        coarse, omap = O.contract(cur, match)
        assert np.array_equal(omap, mp)
        for key in ("xadj", "adjncy", "ewgt", "vwgt"):
            assert np.array_equal(getattr(coarse, key), getattr(levels[l + 1], key)), (l, key)
    top = levels[-1]
    assert top.n <= 20 * 256 or len(maps) == 64 or top.n * 1000 > levels[-2].n * 950
    cpart = I.random_balanced_partition(top.n, 256, seed=1)
    fine = h.project(torch.as_tensor(cpart).cuda()).cpu().numpy()
    want = O.project(maps, cpart)
    assert np.array_equal(fine, want)
    check_eval(dg, g, want, 256, 0.03)
    h.free()


def match_from_map(mp):
    n = mp.shape[0]
    order = np.argsort(mp, kind="stable")
    sm = mp[order]
    match = np.arange(n, dtype=np.int32)
    same = np.nonzero(sm[1:] == sm[:-1])[0]
    a, b = order[same], order[same + 1]
    match[a], match[b] = b, a
    return match


# ---------------------------------------------------------------------------
# many small and ragged graphs, every rating
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("tail", [0, -1])
@pytest.mark.parametrize("matcher", MATCHERS)
@pytest.mark.parametrize("rating", RATINGS)
def test_random_graphs(rating, matcher, tail):
    """tail 0: small graphs run in the persistent tail launch; -1: per-phase
    kernels only."""
    for t in range(24):
        rng = np.random.default_rng(t)
        n = int(rng.integers(2, 400))
        g = I.random_small_graph(n, float(rng.uniform(0.005, 0.2)), seed=100 + t,
                                 wmax=int(rng.choice([1, 5, 1000])), cmax=int(rng.choice([1, 4, 50])),
                                 allow_zero_c=(t % 5 == 0))
        seed = int(rng.integers(0, 2**63))
        stop = int(rng.choice([1, 10, 50]))
        h, dg, levels, maps = run_gpu(g, rating=rating, seed=seed, stop_size=stop, matcher=matcher,
                                      tail_nodes=tail)
        ref = O.coarsen(g, rating, seed, stop)
        assert_same(levels, maps, ref, f"{rating} {matcher} tail={tail} t={t}")
        h.free()


@pytest.mark.parametrize("make,rating", [
    (lambda: I.grid3d(23, 17, 9), "innerOuter"),
    (lambda: I.grid3d(48, 40, 32), "innerOuter"),   # thousands of 17..32-entry coarse rows
    (lambda: I.grid2d(301, 77), "expansion*2"),
    (lambda: I.rgg2d(20000, 5, wmax=16), "expansion*2"),
    (lambda: I.rgg2d(30000, 6, mean_degree=14), "innerOuter"),
    (lambda: I.rmat(12, 3), "expansion*2"),
    (lambda: I.rmat(13, 4), "innerOuter"),
    (lambda: I.rmat(11, 5, edge_factor=64), "weight"),
])
@pytest.mark.parametrize("matcher", MATCHERS)
def test_structured_graphs(make, rating, matcher):
    g = make()
    ref = full_path(g, rating, 7, 20, 5, matcher=matcher)
    assert len(ref.levels) >= 2


# ---------------------------------------------------------------------------
# edge cases
# ---------------------------------------------------------------------------

def test_star_hub_rows():
    """A hub row longer than any shared-memory tile takes the radix path."""
    full_path(I.star_graph(5000), "expansion*2", 3, 2, 2)
    # stars of stars: hubs survive several levels with long coarse rows
    lo, hi = [], []
    for hub in range(8):
        for leaf in range(3000):
            lo.append(hub)
            hi.append(8 + hub * 3000 + leaf)
    for hub in range(7):
        lo.append(hub)
        hi.append(hub + 1)
    g = I.from_edges(8 + 8 * 3000, np.array(lo), np.array(hi), name="stars")
    for r in ["expansion*2", "innerOuter", "weight"]:
        for m in MATCHERS:
            full_path(g, r, 11, 4, 3, matcher=m)


@pytest.mark.parametrize("tail", [0, -1])
@pytest.mark.parametrize("matcher", MATCHERS)
def test_power_law_hub_rows(matcher, tail):
    """R-MAT graphs: hub rows thousands of times longer than the mean take
    the block-per-search pass, at every mean degree (lanes per node 4 and
    32); with tail=-1 every level runs in separate launches."""
    for g, r in [(I.rmat(14, 8), "expansion*2"), (I.rmat(13, 6, edge_factor=256), "expansion*2"),
                 (I.rmat(13, 9, edge_factor=256), "innerOuter")]:
        d = np.diff(g.xadj)
        assert d.max() > 2048
        full_path(g, r, 5, 40, 4, matcher=matcher, tail=tail)


@pytest.mark.parametrize("matcher", MATCHERS)
def test_path_increasing_weights_many_rounds(matcher):
    """Worst case for rounds (one edge per round) and for proposal chains."""
    g = I.path_graph(3000)
    full_path(g, "weight", 0, 2, 2, matcher=matcher)


def test_tiny_and_degenerate():
    import torch
    # empty graph
    g = I.from_edges(0, np.zeros(0, np.int64), np.zeros(0, np.int64))
    h, dg, levels, maps = run_gpu(g)
    assert len(levels) == 1 and levels[0].n == 0
    h.free()
    # single node, isolated nodes, one isolated pair (innerOuter +infinity)
    for g in [I.from_edges(1, np.zeros(0, np.int64), np.zeros(0, np.int64)),
              I.from_edges(30, np.zeros(0, np.int64), np.zeros(0, np.int64)),
              I.from_edges(6, np.array([0, 2, 3]), np.array([1, 3, 4]), np.array([1, 50, 60]))]:
        for r in RATINGS:
            for m in MATCHERS:
                h, dg, levels, maps = run_gpu(g, rating=r, stop_size=0, matcher=m)
                assert_same(levels, maps, O.coarsen(g, r, 1, 0), f"deg {g.n} {r} {m}")
                h.free()
    # zero node weights: expansion*2 ratings become +infinity
    g = I.random_small_graph(200, 0.05, 9, cmax=2, allow_zero_c=True)
    full_path(g, "expansion*2", 5, 3, 4)
    # all ratings equal: the hash alone decides
    g = I.grid2d(50, 50)
    for seed in [0, 1, 2**63 + 5]:
        for m in MATCHERS:
            h, dg, levels, maps = run_gpu(g, seed=seed, stop_size=10, matcher=m)
            assert_same(levels, maps, O.coarsen(g, "expansion*2", seed, 10))
            h.free()


@pytest.mark.parametrize("tail", [0, -1, 2000])
@pytest.mark.parametrize("matcher", MATCHERS)
def test_arena_growth_resumes_exactly(matcher, tail):
    """A tiny initial arena overflows at several levels; the engine grows it
    and resumes at the level that did not fit, with the same results, in the
    per-phase path, the persistent tail, and a switch between them."""
    for g, r in [(I.rgg2d(30000, 9, wmax=5), "expansion*2"), (I.grid3d(20, 20, 20), "innerOuter")]:
        h, dg, levels, maps = run_gpu(g, rating=r, seed=3, stop_size=20, matcher=matcher, arena_bytes=4096,
                                      tail_nodes=tail)
        assert_same(levels, maps, O.coarsen(g, r, 3, 20), f"arena {g.name} {matcher}")
        h.free()


@pytest.mark.parametrize("tail", [0, -1])
def test_power_law_levels_continue_in_spare_arena(tail):
    """R-MAT graphs shrink by a few percent a level, so the initial arena runs
    low after a few levels; the engine continues in spare chunks supplied
    ahead of need (and restarts only if one comes too late), with the same
    results.  The hubs also take all three proposal passes."""
    for sc, seed in [(13, 3), (15, 4)]:
        g = I.rmat(sc, seed)
        for m in MATCHERS:
            h, dg, levels, maps = run_gpu(g, seed=5, stop_size=40, matcher=m, tail_nodes=tail)
            assert_same(levels, maps, O.coarsen(g, "expansion*2", 5, 40), f"{g.name} {m} tail={tail}")
            h.free()


def hub_graph(hubs, leaves, seed):
    """`hubs` nodes joined to every leaf plus a sparse random graph on the
    leaves, random weights: the hubs compete for the same leaves, so each is
    displaced many times."""
    rng = np.random.default_rng(seed)
    h = np.repeat(np.arange(hubs), leaves)
    lf = hubs + np.tile(np.arange(leaves), hubs)
    a = hubs + rng.integers(0, leaves, 3 * leaves)
    b = hubs + rng.integers(0, leaves, 3 * leaves)
    pairs = np.unique(np.stack([np.minimum(a, b), np.maximum(a, b)])[:, a != b], axis=1)
    lo = np.concatenate([h, pairs[0]])
    hi = np.concatenate([lf, pairs[1]])
    w = rng.integers(1, 10, len(lo))
    vw = rng.integers(1, 4, hubs + leaves)
    return I.from_edges(hubs + leaves, lo, hi, w, vwgt=vw, name=f"hubs{hubs}x{leaves}")


@pytest.mark.parametrize("rating", ["expansion*2", "innerOuter", "weight"])
def test_hub_rows_from_candidate_cache(rating):
    """Rows far longer than the cache threshold whose nodes are displaced
    again and again: proposals from the cached candidates reach the same
    matching as full scans (the oracle), in the per-level kernels."""
    for hubs, leaves, seed in [(12, 6000, 1), (40, 5000, 2), (3, 20000, 3)]:
        g = hub_graph(hubs, leaves, seed)
        assert np.diff(g.xadj).max() > 4096
        for stop in (20, 2000):
            h, dg, levels, maps = run_gpu(g, rating=rating, seed=7, stop_size=stop, tail_nodes=-1)
            assert_same(levels, maps, O.coarsen(g, rating, 7, stop), f"{g.name} {rating} stop={stop}")
            h.free()


@pytest.mark.parametrize("radix_bits", [0, 5, 8])
def test_huge_rows_by_cluster(radix_bits):
    """Gathered rows longer than 32768 entries are contracted by a thread-
    block cluster each (every radix pass split over the cluster's CTAs): the
    same sorted coarse rows as the oracle, for 1, 2 and more hubs, with the
    passes of 5 and 8 bits (0: the default)."""
    kw = dict(radix_bits=radix_bits) if radix_bits else {}
    for hubs, leaves, seed in [(1, 70000, 4), (2, 40000, 5), (5, 34000, 6)]:
        g = hub_graph(hubs, leaves, seed)
        for rating in ("expansion*2", "innerOuter"):
            h, dg, levels, maps = run_gpu(g, rating=rating, seed=3, stop_size=30, tail_nodes=-1, **kw)
            assert_same(levels, maps, O.coarsen(g, rating, 3, 30), f"{g.name} {rating} bits={radix_bits}")
            h.free()


def test_stop_rules():
    g = I.grid2d(64, 64)
    for kw in [dict(max_levels=2), dict(max_levels=0), dict(min_shrink_permille=600),
               dict(stop_size=5000)]:
        h, dg, levels, maps = run_gpu(g, stop_size=kw.get("stop_size", 2), **{k: v for k, v in kw.items() if k != "stop_size"})
        ref = O.coarsen(g, "expansion*2", 1, kw.get("stop_size", 2), max_levels=kw.get("max_levels", 64),
                        min_shrink_permille=kw.get("min_shrink_permille", 50))
        assert_same(levels, maps, ref, str(kw))
        h.free()


# ---------------------------------------------------------------------------
# evaluation
# ---------------------------------------------------------------------------

def test_cut_gain_many_k():
    # mean degree <= 12 takes the thread-per-row kernel (rows above 16
    # entries listed for the warp kernel): grids, RGGs, a star, a sparse R-MAT
    for g in [I.grid2d(40, 30), I.rmat(11, 2), I.rgg2d(5000, 3, wmax=9), I.star_graph(3000),
              I.rmat(12, 5, edge_factor=4), I.rgg2d(4000, 4, mean_degree=11, wmax=3)]:
        dg = B().DeviceGraph.from_csr(g)
        for k in [1, 2, 3, 64, 256, 3000]:
            check_eval(dg, g, I.random_partition(g.n, k, seed=k), k, 0.03)
            check_eval(dg, g, I.random_balanced_partition(g.n, k, seed=k + 1), k, 0.1)
        check_eval(dg, g, np.zeros(g.n, np.int32), 1, 0.0)


def test_cut_gain_hub_rows():
    """Rows far longer than a warp: with k <= 256 a warp sums the row's
    connections in shared memory in one pass, above that it visits the
    adjacent blocks one by one; rows above 4096 entries take a block each
    with shared-memory sums up to k = 4096; all give the oracle's gains and
    targets (largest connection, smallest block id on ties).  R-MAT's mean
    degree is above 20: the thread-per-row kernel lists its long rows."""
    for g in [I.rmat(13, 6), hub_graph(3, 20000, 3), hub_graph(40, 5000, 2)]:
        dg = B().DeviceGraph.from_csr(g)
        for k in [2, 64, 256, 257, 1000, 4096, 4097]:
            check_eval(dg, g, I.random_partition(g.n, k, seed=k), k, 0.03)
            check_eval(dg, g, I.random_balanced_partition(g.n, k, seed=k + 5), k, 0.1)


def test_cut_gain_closed_form_grid():
    g = I.grid2d(64, 64)
    dg = B().DeviceGraph.from_csr(g)
    part = np.array([0 if (v % 64) < 32 else 1 for v in range(4096)], dtype=np.int32)
    got = check_eval(dg, g, part, 2, 0.03)
    assert got["cut"] == 64 and got["L_max"] == 2110


# ---------------------------------------------------------------------------
# errors, timeouts, host-buffer entry, determinism
# ---------------------------------------------------------------------------

def test_error_statuses():
    import torch
    g = I.grid2d(8, 8)
    dg = B().DeviceGraph.from_csr(g)
    bad = torch.as_tensor(np.full(64, 2, np.int32)).cuda()
    with pytest.raises(B().KpError) as e:
        B().cut_gain(dg, bad, 2, 0.03)
    assert e.value.status == B().KP_ERR_INVALID
    ew = g.ewgt.copy()
    ew[0] = 7
    asym = B().DeviceGraph(g.xadj, g.adjncy, ew, g.vwgt)
    with pytest.raises(B().KpError) as e:
        B().coarsen(asym)
    assert e.value.status == B().KP_ERR_INVALID
    big = B().DeviceGraph(g.xadj, g.adjncy, g.ewgt, np.full(64, 2**26, np.int32))
    with pytest.raises(B().KpError) as e:
        B().coarsen(big)
    assert e.value.status == B().KP_ERR_OVERFLOW
    with pytest.raises(B().KpError) as e:
        B().coarsen(dg, rating=9)
    assert e.value.status == B().KP_ERR_UNSUPPORTED
    with pytest.raises(B().KpError) as e:
        B().coarsen(dg, matcher=7)
    assert e.value.status == B().KP_ERR_UNSUPPORTED


@pytest.mark.parametrize("matcher", MATCHERS)
def test_bounded_waits_report_status_and_context_survives(matcher):
    """With a bound of one step, a grid-barrier wait (handshake) or a proposal
    chain (suitor) runs out; the kernel sets the error flag and returns,
    kp_coarsen reports KP_ERR_TIMEOUT, and the next call on the same context
    succeeds."""
    g = I.grid2d(512, 512)
    dg = B().DeviceGraph.from_csr(g)
    with pytest.raises(B().KpError) as e:
        B().coarsen(dg, spin_limit=1, stop_size=10, matcher=matcher)
    assert e.value.status == B().KP_ERR_TIMEOUT
    h, _, levels, maps = run_gpu(I.grid2d(64, 64))
    assert_same(levels, maps, O.coarsen(I.grid2d(64, 64), "expansion*2", 1, 40))
    h.free()


def test_pipeline_host_matches_device_path():
    g = I.rgg2d(50000, 2, wmax=4)
    k = 16

    def ip(nc, cw, kk):
        return I.random_balanced_partition(nc, kk, seed=3)

    res = B().pipeline_host(g.xadj, g.adjncy, g.ewgt, g.vwgt, k, 0.03, ip, stop_size=20 * k, seed=4)
    ref = O.coarsen(g, "expansion*2", 4, 20 * k)
    assert res["num_levels"] == len(ref.levels)
    part = O.project(ref.maps, I.random_balanced_partition(ref.levels[-1].n, k, seed=3))
    want = O.cut_gain(g, part, k, 0.03)
    assert np.array_equal(res["part"], part)
    assert res["cut"] == want["cut"] and res["L_max"] == want["L_max"]
    assert res["imbalance"] == want["imbalance"]
    assert np.array_equal(res["gain"], want["gain"]) and np.array_equal(res["target"], want["target"])
    assert np.array_equal(res["block_w"], want["block_w"])


def test_deterministic_across_runs_and_streams():
    import torch
    g = I.rgg2d(100000, 8)
    h1, _, l1, m1 = run_gpu(g, stop_size=100)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        h2, _, l2, m2 = run_gpu(g, stop_size=100)
    torch.cuda.synchronize()
    assert len(l1) == len(l2)
    for a, b in zip(l1, l2):
        assert np.array_equal(a.adjncy, b.adjncy) and np.array_equal(a.ewgt, b.ewgt)
    for a, b in zip(m1, m2):
        assert np.array_equal(a, b)
    h1.free()
    h2.free()


def test_saved_and_loaded_hierarchy_is_identical(tmp_path):
    import torch
    g = I.rgg2d(20000, 9, wmax=16)
    h, dg, levels, maps = run_gpu(g, rating="expansion*2", seed=4, stop_size=40)
    path = str(tmp_path / "h.kph")
    h.save(path)
    h2 = B().load_hierarchy(path)
    assert h2.num_levels() == h.num_levels()
    for l in range(h.num_levels()):
        a, b = h.level(l), h2.level(l)
        for key in ("xadj", "adjncy", "ewgt", "vwgt"):
            assert np.array_equal(a[key].cpu().numpy(), b[key].cpu().numpy()), (l, key)
        if a["map"] is not None:
            assert np.array_equal(a["map"].cpu().numpy(), b["map"].cpu().numpy()), (l, "map")
    top = levels[-1].n
    cp = torch.as_tensor(I.random_balanced_partition(top, 4, seed=1)).cuda()
    assert np.array_equal(h.project(cp).cpu().numpy(), h2.project(cp).cpu().numpy())
    h2.free()
    h.free()
    # a map entry pointing past the next level is refused before any upload
    data = bytearray(open(path, "rb").read())
    n0, nnz0 = g.n, g.nnz
    if B().OFFSET_BITS == 64:   # file version 2: i32 n, i32 0, i64 nnz, int64 xadj
        map0 = 24 + 16 + 8 * (n0 + 1) + 8 * nnz0 + 4 * n0
    else:                       # version 1: i32 n, i32 nnz, int32 xadj
        map0 = 24 + 8 + 4 * (n0 + 1) + 8 * nnz0 + 4 * n0
    data[map0:map0 + 4] = np.int32(levels[1].n).tobytes()
    bad = str(tmp_path / "bad.kph")
    open(bad, "wb").write(bytes(data))
    with pytest.raises(B().KpError) as e:
        B().load_hierarchy(bad)
    assert e.value.status == B().KP_ERR_INVALID


def test_input_check_on_power_law_rows():
    """The entry-parallel input check: valid R-MAT graphs (hub rows of
    thousands of entries) pass; each kind of malformed row is refused, in a
    hub row as well as in a short one."""
    g = I.rmat(14, 8)
    d = np.diff(g.xadj)
    hub = int(np.argmax(d))
    short = int(np.nonzero((d[:-1] == 3) & (d[1:] > 0))[0][0])
    assert d[hub] > 2048
    h = B().coarsen(B().DeviceGraph.from_csr(g), stop_size=40)
    h.free()

    def refused(xadj, adj, ew, vw):
        dg = B().DeviceGraph(np.ascontiguousarray(xadj, np.int32), np.ascontiguousarray(adj, np.int32),
                             np.ascontiguousarray(ew, np.int32), np.ascontiguousarray(vw, np.int32))
        with pytest.raises(B().KpError) as e:
            B().coarsen(dg, stop_size=40)
        assert e.value.status == B().KP_ERR_INVALID

    for row in (hub, short):
        a, b = int(g.xadj[row]), int(g.xadj[row + 1])
        adj = g.adjncy.copy()
        adj[a], adj[a + 1] = adj[a + 1], adj[a]           # row not ascending
        refused(g.xadj, adj, g.ewgt, g.vwgt)
        adj = g.adjncy.copy()
        adj[b - 1] = row                                   # self loop
        refused(g.xadj, adj, g.ewgt, g.vwgt)
        ew = g.ewgt.copy()
        ew[a + 1] += 1                                     # reverse entry has another weight
        refused(g.xadj, g.adjncy, ew, g.vwgt)
        ew = g.ewgt.copy()
        ew[a] = 0                                          # omega must be positive
        refused(g.xadj, g.adjncy, ew, g.vwgt)
        adj = g.adjncy.copy()
        adj[b - 1] = g.n + 5                               # neighbour out of range
        refused(g.xadj, adj, g.ewgt, g.vwgt)
    vw = g.vwgt.copy()
    vw[hub] = -1                                           # c must be >= 0
    refused(g.xadj, g.adjncy, g.ewgt, vw)
    xadj = g.xadj.copy()
    xadj[short + 1], xadj[short + 2] = xadj[short + 2], xadj[short + 1]   # decreasing offsets (in range)
    refused(xadj, g.adjncy, g.ewgt, g.vwgt)
