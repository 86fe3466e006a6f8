"""Failure injection on the host (no GPU fault): every device allocation of
an entry point is made to fail in turn; the call must return KP_ERR_OOM, give
back every byte it took, and the next call must work and match the oracle."""
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


def sweep(call, check, limit=80):
    """call() under an injected failure of its i-th allocation, i = 0, 1, ...
    until it succeeds without one; check(result) on every success."""
    import torch
    torch.cuda.synchronize()
    base = B().kp_test_device_bytes_in_use()
    failures = 0
    for after in range(limit):
        B().kp_test_fail_allocation(after)
        try:
            res = call()
        except B().KpError as e:
            assert e.status == B().KP_ERR_OOM, str(e)
            assert "injected" in str(e)
            failures += 1
            torch.cuda.synchronize()
            assert B().kp_test_device_bytes_in_use() == base, after   # nothing leaked
            continue
        finally:
            B().kp_test_fail_allocation(-1)
        check(res)
        torch.cuda.synchronize()
        return failures
    raise AssertionError("no successful call within the limit")


def test_coarsen_and_batch_survive_every_allocation_failure():
    g = I.rgg2d(3000, 7, wmax=5)
    dg = B().DeviceGraph.from_csr(g)
    ref = O.coarsen(g, "innerOuter", 3, 20)

    def one():
        return B().coarsen(dg, rating="innerOuter", seed=3, stop_size=20, tail_nodes=-1)

    def check(h):
        assert h.num_levels() == len(ref.levels)
        lv = h.level(h.num_levels() - 1)
        assert np.array_equal(lv["adjncy"].cpu().numpy(), ref.levels[-1].adjncy)
        h.free()

    assert sweep(one, check) >= 5
    graphs = [I.grid2d(9, 7), I.rmat(8, 2), I.star_graph(40)]
    U, off = I.union_graph(graphs)
    du = B().DeviceGraph.from_csr(U)
    refs = [O.coarsen(gr, "expansion*2", 5, 6) for gr in graphs]

    def batch():
        return B().coarsen_batch(du, off, np.full(len(graphs), 5, np.uint64), stop_size=6)

    def check_batch(h):
        assert h.graph_levels() == [len(r.levels) for r in refs]
        h.free()

    assert sweep(batch, check_batch) >= 5


def test_evaluation_and_refinement_helpers_survive_allocation_failures():
    import torch
    g = I.grid2d(30, 20)
    dg = B().DeviceGraph.from_csr(g)
    part = I.random_balanced_partition(g.n, 4, seed=2)
    tp = torch.as_tensor(part).cuda()
    want = O.cut_gain(g, part, 4, 0.03)
    sweep(lambda: B().cut_gain(dg, tp, 4, 0.03), lambda r: r["cut"] == want["cut"])
    qw = O.quotient_graph(g, part, 4)
    sweep(lambda: B().quotient_graph(dg, tp, 4),
          lambda r: np.array_equal(r[2].cpu().numpy(), qw[2]) or pytest.fail("quotient differs"))
    bw = O.boundary_band(g, part, 5)
    sweep(lambda: B().boundary_band(dg, tp, 4, 5),
          lambda r: np.array_equal(r.cpu().numpy(), bw) or pytest.fail("band differs"))


def test_plan_survives_allocation_failures():
    g = I.rgg2d(2000, 8)
    dg = B().DeviceGraph.from_csr(g)
    ref = O.coarsen(g, "expansion*2", 1, 40)

    def make():
        return B().Plan(dg, stop_size=40)

    def check(plan):
        assert plan.run().num_levels() == len(ref.levels)
        plan.close()

    assert sweep(make, check) >= 3


def test_server_cancel_of_a_waiting_request():
    g = I.grid2d(30, 30)
    with B().Server(workers=1, max_batch=1, hbm_budget_bytes=1) as sv:
        ids = [sv.submit(g.xadj, g.adjncy, g.ewgt, g.vwgt, 2, 0.03, s, 40) for s in range(3)]
        first = sv.wait(ids[0])                 # resident: the others wait for budget
        sv.cancel(ids[2])
        with pytest.raises(B().KpError):
            sv.poll(ids[2])                     # forgotten
        with pytest.raises(B().KpError):
            sv.cancel(ids[0])                   # already started
        sv.release(ids[0])
        second = sv.wait(ids[1])
        assert second["status"] == 0 and first["status"] == 0
        sv.release(ids[1])


def test_server_cancel_wakes_a_thread_waiting_on_the_request():
    import threading
    import time
    g = I.grid2d(30, 30)
    with B().Server(workers=1, max_batch=1, hbm_budget_bytes=1) as sv:
        ids = [sv.submit(g.xadj, g.adjncy, g.ewgt, g.vwgt, 2, 0.03, s, 40) for s in range(2)]
        sv.wait(ids[0])                         # resident: ids[1] waits for budget
        box = {}

        def waiter():
            try:
                box["res"] = sv.wait(ids[1])
            except B().KpError as e:
                box["err"] = e

        t = threading.Thread(target=waiter)
        t.start()
        time.sleep(0.3)                         # the waiter blocks on the queued request
        sv.cancel(ids[1])
        t.join(timeout=60)
        assert not t.is_alive(), "a wait on a cancelled request must return"
        assert "err" in box and box["err"].status == B().KP_ERR_INVALID
        sv.release(ids[0])


def test_server_release_waits_for_a_fetch_in_progress():
    import threading
    g = I.grid2d(200, 200)
    with B().Server(workers=1, max_batch=1) as sv:
        for rep in range(3):
            rid = sv.submit(g.xadj, g.adjncy, g.ewgt, g.vwgt, 4, 0.03, rep, 80)
            res = sv.wait(rid)
            first = sv.fetch(rid, g.n, res["coarsest_n"])
            seen = []

            def reader():
                for _ in range(20):
                    try:
                        got = sv.fetch(rid, g.n, res["coarsest_n"])
                    except B().KpError as e:
                        seen.append(e.status)
                        return
                    seen.append(bool(np.array_equal(got["part"], first["part"])))

            t = threading.Thread(target=reader)
            t.start()
            sv.release(rid)
            t.join(timeout=60)
            assert not t.is_alive()
            # every fetch that ran saw the results intact, then the id was gone
            assert all(x is True or x == B().KP_ERR_INVALID for x in seen), seen
