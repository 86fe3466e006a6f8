"""The 64-bit offset build (libkp64.so) on the GPU, against the oracle:

- the parity suites again with every row offset and entry index 64-bit
  (random, structured, degenerate and power-law graphs, every rating and
  matcher, batches, refinement helpers), in a child process whose binding
  selects the wide library;
- a graph of more than 2^31 directed entries (a circulant graph, 26
  neighbours per node, 96M nodes, 2.5G entries: the input's offsets, the
  contraction's row slots and the coarse level's offsets all pass 2^31),
  contracted twice (Section 5.2's static adjacency array with 64-bit
  offsets).  A whole pass of the oracle over each level would take many
  minutes, so each level is checked on sampled nodes the oracle computes
  one by one -- 150,000 random ones, those whose rows straddle entry 2^31,
  and the last ones -- with its Greedy characterisation at those nodes and
  its coarse row of each sampled node's pair, plus what holds at any size
  (the map numbers the pairs' representatives in order, n' = n - |M|, the
  sum of c is kept, the coarse CSR is well formed).  The projection and the
  cut/gain of the input for k = 64 are checked whole.  All comparisons are
  exact."""
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle as O
from paper_0910_2004_gb300 import inputs as I

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def B():
    from paper_0910_2004_gb300 import binding
    return binding


def run_wide_pytest(args, timeout):
    env = dict(os.environ, KP_OFFSET_BITS="64")
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider"] + args, cwd=ROOT,
                       env=env, capture_output=True, text=True, timeout=timeout)
    assert r.returncode == 0, (r.stdout + r.stderr)[-6000:]
    return r.stdout


def test_parity_suites_through_64_bit_offsets():
    if B().OFFSET_BITS == 64:
        pytest.skip("runs the suites in a child with the wide library")
    out = run_wide_pytest(["tests/test_gpu_parity.py", "tests/test_gpu_gpa.py", "tests/test_gpu_batch.py",
                           "tests/test_gpu_refine.py", "-m", "gpu and not slow"], timeout=3600)
    assert " passed" in out and "skipped" not in out.splitlines()[-1], out[-2000:]


def _match_from_map(mp_):
    order = np.argsort(mp_, kind="stable")
    sm = mp_[order]
    match = np.arange(mp_.shape[0], dtype=np.int32)
    same = np.nonzero(sm[1:] == sm[:-1])[0]
    a, b = order[same], order[same + 1]
    match[a], match[b] = b, a
    return match


def _sample_nodes(xadj, count, seed):
    """Random nodes, the nodes whose rows hold entries next to 2^31, and the
    last nodes of the level."""
    n = xadj.shape[0] - 1
    rng = np.random.default_rng(seed)
    at = int(np.searchsorted(xadj, 2 ** 31, side="right")) - 1
    special = np.arange(max(0, at - 500), min(n, at + 500))
    last = np.arange(max(0, n - 1000), n)
    return np.unique(np.concatenate([rng.choice(n, size=min(count, n), replace=False), special, last])).astype(np.int32)


def _device_rows(lv, xs):
    """Rows xs of a device level, gathered on the device: (lengths, adjncy,
    ewgt) on the host."""
    import torch
    x = torch.as_tensor(xs, device="cuda").long()
    lo, hi = lv["xadj"][x], lv["xadj"][x + 1]
    ln = hi - lo
    start = torch.repeat_interleave(lo - torch.cumsum(ln, 0) + ln, ln)
    idx = start + torch.arange(int(ln.sum()), device="cuda")
    return ln.cpu().numpy(), lv["adjncy"][idx].cpu().numpy(), lv["ewgt"][idx].cpu().numpy()


def _host_memory_gb():
    try:
        for line in open("/proc/meminfo"):
            if line.startswith("MemAvailable:"):
                return int(line.split()[1]) / 2 ** 20
    except OSError:
        pass
    return 0.0


@pytest.mark.slow
def test_beyond_2pow31_entries():
    if B().OFFSET_BITS != 64:
        run_wide_pytest([f"{__file__}::test_beyond_2pow31_entries", "-m", "gpu"], timeout=3600)
        return
    import torch
    if torch.cuda.mem_get_info()[0] < 200 * 2 ** 30 or _host_memory_gb() < 48:
        pytest.skip("needs 200 GB free on the device and 48 GB of host memory")
    n, k, eps, rating, seed = 96_000_000, 64, 0.03, "expansion*2", 3
    S = I.circulant_strides(n, 13, 5)
    xadj, adj, ew, vw = I.circulant_torch(n, S)
    torch.cuda.synchronize()
    torch.cuda.empty_cache()   # the generator's blocks back to the device
    dg = B().DeviceGraph(xadj, adj, ew, vw)
    assert dg.nnz == 26 * n and dg.nnz > 2 ** 31
    h = B().coarsen(dg, rating=rating, seed=seed, stop_size=1000, max_levels=2, validate=True)
    assert h.num_levels() == 3
    lv = [h.level(l) for l in range(3)]
    assert int(lv[1]["nnz"]) > 2 ** 31, [int(x["nnz"]) for x in lv]   # coarse offsets past 2^31 too
    maps = [lv[l]["map"].cpu().numpy() for l in range(2)]

    # projection and cut/gain of the input, whole
    cur = O.Level(xadj.cpu().numpy(), adj.cpu().numpy(), ew.cpu().numpy(), vw.cpu().numpy())
    cpart = I.random_balanced_partition(int(lv[2]["n"]), k, seed=1)
    fine = h.project(torch.as_tensor(cpart).cuda()).cpu().numpy()
    want = O.project(maps, cpart)
    assert np.array_equal(fine, want)
    got = B().cut_gain(dg, torch.as_tensor(want).cuda(), k, eps)
    ref = O.cut_gain(cur, want, k, eps)
    for key in ("cut", "L_max", "imbalance"):
        assert got[key] == ref[key], key
    for key in ("block_w", "gain", "target"):
        assert np.array_equal(got[key].cpu().numpy(), ref[key]), key
    del fine, want, got, ref

    for l in range(2):
        mp_ = maps[l]
        nl = cur.n
        match = _match_from_map(mp_)
        v = np.arange(nl, dtype=np.int64)
        # what holds at any size: the map numbers the representatives (the
        # smaller end of each pair) in fine-id order, n' = n - |M|, sum c kept
        rep = match >= v
        assert np.array_equal(mp_[rep], np.arange(int(rep.sum()), dtype=np.int32)), l
        assert np.array_equal(mp_, mp_[np.minimum(match, v)]), l
        nxt = lv[l + 1]
        X1 = nxt["xadj"].cpu().numpy()
        c1 = nxt["vwgt"].cpu().numpy()
        assert X1.shape[0] - 1 == int(rep.sum()) and X1[0] == 0 and X1[-1] == int(nxt["nnz"])
        assert np.all(np.diff(X1) >= 0)
        assert int(c1.astype(np.int64).sum()) == int(cur.vwgt.astype(np.int64).sum())
        # sampled nodes: the Greedy characterisation and the coarse rows
        nodes = _sample_nodes(cur.xadj, 150_000, 10 + l)
        assert O.check_greedy_matching_at(cur, rating, seed, match, nodes) == -1, l
        rows = {}
        for u in nodes.tolist():
            p = int(match[u])
            rows[int(mp_[u])] = (min(u, p), max(u, p) if p != u else -1)
        xs = np.array(sorted(rows), dtype=np.int64)
        ln, gadj, gw = _device_rows(nxt, xs)
        want_rows = O.coarse_rows(cur, mp_, [(x,) + rows[x] for x in xs.tolist()])
        pos = 0
        for i, (x, (radj, rw, rc)) in enumerate(zip(xs.tolist(), want_rows)):
            assert int(ln[i]) == radj.shape[0], (l, x)
            assert np.array_equal(gadj[pos:pos + ln[i]], radj) and np.array_equal(gw[pos:pos + ln[i]], rw), (l, x)
            assert int(c1[x]) == rc, (l, x)
            pos += int(ln[i])
        del cur, match, rep, v
        if l == 0:
            cur = O.Level(X1, nxt["adjncy"].cpu().numpy(), nxt["ewgt"].cpu().numpy(), c1)
    h.free()
