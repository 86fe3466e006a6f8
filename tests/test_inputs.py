"""The seeded synthetic input generators that run with torch (R-MAT and RGG
graphs of the large workloads and the served pool, the device-drawn random
balanced partitions), checked on the CPU: valid symmetric sorted CSRs of the
stated structure, balanced partitions, determinism per seed."""
import numpy as np
import pytest

from paper_0910_2004_gb300 import inputs as I

torch = pytest.importorskip("torch")


def check_csr(g, weights_positive=True):
    n = g.n
    x, a, w = g.xadj.astype(np.int64), g.adjncy.astype(np.int64), g.ewgt.astype(np.int64)
    assert x[0] == 0 and x[-1] == len(a) and np.all(np.diff(x) >= 0)
    assert len(w) == len(a) and len(g.vwgt) == n
    rows = np.repeat(np.arange(n), np.diff(x))
    assert np.all((a >= 0) & (a < n))
    assert not np.any(rows == a), "self loop"
    # rows sorted strictly (no parallel entries)
    same_row = rows[1:] == rows[:-1]
    assert np.all(a[1:][same_row] > a[:-1][same_row])
    # symmetric with equal weights
    fwd = np.stack([rows, a, w], 1)
    bwd = np.stack([a, rows, w], 1)
    fwd = fwd[np.lexsort((fwd[:, 1], fwd[:, 0]))]
    bwd = bwd[np.lexsort((bwd[:, 1], bwd[:, 0]))]
    assert np.array_equal(fwd, bwd)
    if weights_positive:
        assert np.all(w >= 1)


@pytest.mark.parametrize("scale,seed", [(8, 1), (10, 2), (11, 7)])
def test_rmat_torch_structure(scale, seed):
    g = I.rmat_torch(scale, seed, device="cpu")
    assert g.n == 1 << scale
    check_csr(g)
    assert np.all(g.vwgt == 1)
    # every sample that is not a self loop lands in an edge weight: the
    # weights sum to the samples kept (at most edge_factor * n; self loops
    # need all scale bit pairs equal, probability (a + d)^scale)
    M = 16 * g.n
    kept = int(g.ewgt.astype(np.int64).sum()) // 2
    assert kept <= M
    assert kept >= M * (1 - 2 * 0.62 ** scale) - 4 * np.sqrt(M)
    # power law: hubs far above the mean degree
    deg = np.diff(g.xadj)
    assert deg.max() > 8 * deg.mean()
    # seeded
    h = I.rmat_torch(scale, seed, device="cpu")
    assert np.array_equal(g.xadj, h.xadj) and np.array_equal(g.adjncy, h.adjncy)
    assert np.array_equal(g.ewgt, h.ewgt)
    other = I.rmat_torch(scale, seed + 1, device="cpu")
    assert not (np.array_equal(g.xadj, other.xadj) and np.array_equal(g.adjncy, other.adjncy))


def test_rmat_torch_matches_the_numpy_generator_in_distribution():
    """Same distribution as rmat() (other draws): mean degree and largest
    degree of the same scale within a few percent over several seeds."""
    s = 11
    t = [I.rmat_torch(s, seed, device="cpu") for seed in range(4)]
    h = [I.rmat(s, seed) for seed in range(4)]
    mt = np.mean([len(g.adjncy) / g.n for g in t])
    mh = np.mean([len(g.adjncy) / g.n for g in h])
    assert abs(mt - mh) / mh < 0.03
    wt = np.mean([g.ewgt.astype(np.int64).sum() for g in t])
    wh = np.mean([g.ewgt.astype(np.int64).sum() for g in h])
    assert abs(wt - wh) / wh < 0.01


@pytest.mark.parametrize("n,seed", [(1000, 1), (4096, 3), (20000, 5)])
def test_rgg2d_torch_structure(n, seed):
    g = I.rgg2d_torch(n, seed, device="cpu")
    assert g.n == n
    check_csr(g)
    assert np.all(g.ewgt == 1) and np.all(g.vwgt == 1)
    mean = len(g.adjncy) / n
    assert 5.0 < mean < 7.0   # radius for mean degree 6 (fewer neighbours at the border)
    h = I.rgg2d_torch(n, seed, device="cpu")
    assert np.array_equal(g.adjncy, h.adjncy)


@pytest.mark.parametrize("k", [1, 2, 7, 64])
def test_batch_partition_torch_is_balanced_per_graph(k):
    sizes = [0, 1, 5, 64, 1000, 3, 4097]
    part, off = I.batch_partition_torch(sizes, k, seed=11, device="cpu")
    part, off = part.numpy(), off.numpy()
    assert np.array_equal(off, np.concatenate([[0], np.cumsum(sizes)]))
    assert len(part) == sum(sizes)
    assert np.all((part >= 0) & (part < k))
    for i, n in enumerate(sizes):
        p = part[off[i]:off[i + 1]]
        counts = np.bincount(p, minlength=k)
        assert counts.max() - counts.min() <= 1, (n, counts)
    again, _ = I.batch_partition_torch(sizes, k, seed=11, device="cpu")
    assert np.array_equal(part, again.numpy())
    if k > 1:
        other, _ = I.batch_partition_torch(sizes, k, seed=12, device="cpu")
        assert not np.array_equal(part, other.numpy())


def test_single_graph_device_partition_is_balanced():
    # the single-graph bench draws a large coarsest level's partition this way
    part, off = I.batch_partition_torch([70001], 64, seed=3, device="cpu")
    counts = np.bincount(part.numpy(), minlength=64)
    assert counts.max() - counts.min() <= 1 and counts.sum() == 70001


@pytest.mark.parametrize("n,count,seed", [(9, 4, 1), (101, 13, 2), (1000, 13, 3)])
def test_circulant_structure_and_torch_equals_numpy(n, count, seed):
    import oracle as O
    S = I.circulant_strides(n, count, seed)
    assert len(set(S.tolist())) == count and S.min() >= 1 and 2 * S.max() < n
    g = I.circulant(n, S)
    check_csr(g)
    assert np.all(np.diff(g.xadj) == 2 * count)
    assert O.validate(g) == 0
    x, a, w, v = I.circulant_torch(n, S, device="cpu", chunk=7)
    assert x.dtype == torch.int64
    assert np.array_equal(x.numpy(), g.xadj) and np.array_equal(a.numpy(), g.adjncy)
    assert np.array_equal(w.numpy(), g.ewgt) and np.array_equal(v.numpy(), g.vwgt)


def test_csr_container_refuses_wrapped_offsets():
    """xadj[n] must equal the number of entries: an offset that wrapped in a
    narrowing cast is caught where a generator builds the graph."""
    x = np.array([0, 1, 2], np.int32)
    I.CSRGraph(x, np.array([1, 0], np.int32), np.ones(2, np.int32), np.ones(2, np.int32))
    with pytest.raises(ValueError):
        I.CSRGraph(x, np.array([1, 0, 0], np.int32), np.ones(3, np.int32), np.ones(2, np.int32))
    with pytest.raises(ValueError):   # 2^26 nodes x 64 neighbours = 2^32 entries: the torch builder's size
        I.circulant(1 << 26, I.circulant_strides(1 << 26, 32, seed=1))
