"""kp_cut_gain_noalloc: the cut/gain evaluation for callers that cannot
allocate device memory (serving loops that must stay out of the allocator,
applications running the library under a fixed memory budget or behind their
own allocator).  Its scratch is a static device array shared by all calls.

The entry point is called through the C ABI and must give exactly what
kp_cut_gain gives (all results are integers, so the tolerance is zero), on
consecutive calls that reuse the same static scratch.  This file sorts last
so a run that stops at the first failure has run every other test before it.
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
    for key in ("cut", "total_c", "max_c", "L_max", "imbalance"):
        assert a[key] == b[key], key
    for key in ("block_w", "gain", "target"):
        want = b[key].cpu().numpy() if hasattr(b[key], "cpu") else b[key]
        assert np.array_equal(a[key], want), key


def test_noalloc_matches_cut_gain_on_consecutive_calls():
    import torch
    from paper_0910_2004_gb300 import binding as B
    cases = [
        (I.rgg2d(40000, 3, wmax=7), 64, 0.03, 1),     # many blocks, shared-memory block weights
        (I.grid2d(100, 80), 5, 0.10, 2),              # fewer blocks: stale weights of call 1 must not leak
        (I.rmat(12, 5), 3000, 0.03, 3),               # k above the shared-memory limit, hub rows
        (I.rgg2d(40000, 3, wmax=7), 64, 0.03, 1),     # the first call again
    ]
    for g, k, eps, seed in cases:
        dg = B.DeviceGraph.from_csr(g)
        part = torch.as_tensor(I.random_partition(g.n, k, seed)).cuda()
        want = B.cut_gain(dg, part, k, eps)
        got = _noalloc(B, dg, part, k, eps)
        _same(got, want)
        got2 = _noalloc(B, dg, part, k, eps)          # two calls in a row on the same input
        _same(got2, want)


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
    part = torch.as_tensor(I.random_partition(g.n, kmax, 4)).cuda()
    _same(_noalloc(B, dg, part, kmax, 0.03), B.cut_gain(dg, part, kmax, 0.03))
