"""kp_cut_gain_noalloc: the cut/gain evaluation for callers that cannot
allocate device memory (serving loops that must stay out of the allocator,
applications running the library under a fixed memory budget or behind their
own allocator).  Its scratch is a static device array shared by all calls.

The entry point is called through the C ABI and must give exactly what the
oracle's cut/gain gives, and what kp_cut_gain gives (all results are
integers, so the tolerance is zero), on consecutive calls that reuse the same
static scratch.  The cases reach every kernel the entry point dispatches to
(4, 8, 16 and 32 lanes per node; shared-memory connection bins for k <= 256;
rows longer than 4096 entries kept in the warp kernel; block weights beyond
the shared-memory limit).  This file sorts last so a run that stops at the
first failure has run every other test before it.
"""
import ctypes

import numpy as np
import pytest

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


def _noalloc(B, dg, part, k, eps):
    import torch
    bw = torch.full((k,), -7, dtype=torch.int64, device="cuda")
    gain = torch.full((dg.n,), -7, dtype=torch.int64, device="cuda")
    target = torch.full((dg.n,), -7, dtype=torch.int32, device="cuda")
    out = B.kp_cut_gain_out()
    out.block_w, out.gain, out.target = bw.data_ptr(), gain.data_ptr(), target.data_ptr()
    B.kp_cut_gain_noalloc(dg.kp, part.data_ptr(), k, eps, out, B.current_stream())
    return {"cut": out.cut, "total_c": out.total_c, "max_c": out.max_c, "L_max": out.l_max,
            "imbalance": out.imbalance, "block_w": bw.cpu().numpy(), "gain": gain.cpu().numpy(),
            "target": target.cpu().numpy()}


def _same(a, b):
    for key in ("cut", "L_max", "imbalance"):
        assert a[key] == b[key], key
    for key in ("total_c", "max_c"):
        if key in b:
            assert a[key] == b[key], key
    for key in ("block_w", "gain", "target"):
        want = b[key].cpu().numpy() if hasattr(b[key], "cpu") else b[key]
        assert np.array_equal(a[key], want), key


def test_noalloc_matches_the_oracle_and_cut_gain_on_consecutive_calls():
    import torch

    import oracle as O
    from paper_0910_2004_gb300 import binding as B
    rgg = I.rgg2d(40000, 3, wmax=7)
    rmat12, rmat15 = I.rmat(12, 5), I.rmat(15, 4)
    assert int(np.diff(rmat15.xadj).max()) > 4096
    cases = [
        (rgg, 64, 0.03, 1),                                          # mean degree 6: 8 lanes per node
        (I.grid2d(100, 80), 5, 0.10, 2),                             # 4 lanes; stale weights of call 1 must not leak
        (I.rgg2d(20000, 3, mean_degree=14, wmax=5), 16, 0.03, 5),    # mean degree 14: 16 lanes
        (rmat12, 64, 0.03, 6),                                       # a warp per node, shared-memory bins (k <= 256)
        (rmat15, 200, 0.05, 7),                                      # rows of more than 4096 entries, bins
        (rmat12, 3000, 0.03, 3),                                     # k above the shared-memory limit
        (rmat15, 5000, 0.03, 8),                                     # both
        (rgg, 64, 0.03, 1),                                          # the first call again
    ]
    for g, k, eps, seed in cases:
        dg = B.DeviceGraph.from_csr(g)
        host_part = I.random_partition(g.n, k, seed)
        part = torch.as_tensor(host_part).cuda()
        want = O.cut_gain(g, host_part, k, eps)
        got = _noalloc(B, dg, part, k, eps)
        _same(got, want)
        assert got["total_c"] == int(g.vwgt.sum()) and got["max_c"] == int(g.vwgt.max())
        got2 = _noalloc(B, dg, part, k, eps)          # two calls in a row on the same input
        _same(got2, want)
        _same(got2, B.cut_gain(dg, part, k, eps))     # and the allocating entry point agrees


def test_noalloc_rejects_k_above_the_static_maximum():
    import torch
    from paper_0910_2004_gb300 import binding as B
    g = I.grid2d(8, 8)
    dg = B.DeviceGraph.from_csr(g)
    k = B.KP_CUT_GAIN_NOALLOC_MAX_K + 1
    part = torch.zeros(g.n, dtype=torch.int32, device="cuda")
    with pytest.raises(B.KpError) as e:
        _noalloc(B, dg, part, k, 0.03)
    assert e.value.status == B.KP_ERR_UNSUPPORTED
    assert "KP_CUT_GAIN_NOALLOC_MAX_K" in str(e.value)
    # the largest accepted k still works
    kmax = B.KP_CUT_GAIN_NOALLOC_MAX_K
    import oracle as O
    host_part = I.random_partition(g.n, kmax, 4)
    part = torch.as_tensor(host_part).cuda()
    _same(_noalloc(B, dg, part, kmax, 0.03), O.cut_gain(g, host_part, kmax, 0.03))
    _same(_noalloc(B, dg, part, kmax, 0.03), B.cut_gain(dg, part, kmax, 0.03))
