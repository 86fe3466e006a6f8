"""The request server (kp_server_*): every request's result equals the oracle
run on that request alone (coarsening, projection of the coarsest partition,
cut/gain), whether the server ran it alone or merged into a batch with
others; admission is first in, first out under the device budget, and
resident results hold their budget until released."""
import time

import numpy as np
import pytest

import oracle as O
from paper_0910_2004_gb300 import inputs as I

pytestmark = pytest.mark.gpu

MASK = (1 << 64) - 1


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


def _mix(x):
    # splitmix64 (Steele, Lea, Flood 2014): advance by the golden-ratio
    # increment, then the two xor-shift-multiply rounds and a final xor-shift
    z = (x + 0x9E3779B97F4A7C15) & MASK
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK
    return z ^ (z >> 31)


def initial_partition(c, k, seed):
    """The server's documented initial partition: Fisher-Yates over 0..c-1
    with j = mix(state) mod (i+1), the state advanced by the golden-ratio
    increment before each draw, then block i mod k for the i-th node."""
    perm = list(range(c))
    state = seed & MASK
    for i in range(c - 1, 0, -1):
        state = (state + 0x9E3779B97F4A7C15) & MASK
        j = _mix(state) % (i + 1)
        perm[i], perm[j] = perm[j], perm[i]
    part = np.empty(c, np.int32)
    for i, v in enumerate(perm):
        part[v] = i % k
    return part


def request_pool(seed):
    rng = np.random.default_rng(seed)
    gs = [I.grid2d(17, 9), I.grid3d(6, 5, 4), I.rgg2d(3000, seed, wmax=16), I.star_graph(300), I.path_graph(200),
          I.rmat(9, seed), I.from_edges(0, np.zeros(0, np.int64), np.zeros(0, np.int64)),
          I.from_edges(25, np.zeros(0, np.int64), np.zeros(0, np.int64)),
          I.from_edges(2, np.array([0]), np.array([1]))]
    for t in range(9):
        gs.append(I.random_small_graph(int(rng.integers(2, 150)), float(rng.uniform(0.02, 0.3)),
                                       seed=seed * 100 + t, wmax=int(rng.choice([1, 7, 300])),
                                       cmax=int(rng.choice([1, 5])), allow_zero_c=(t % 3 == 0)))
    reqs = []
    for i, g in enumerate(gs):
        reqs.append(dict(g=g, k=int(rng.choice([1, 2, 3, 8])), eps=float(rng.choice([0.0, 0.03, 0.5])),
                         seed=int(rng.integers(0, 1 << 63)), stop=int(rng.choice([6, 40]))))
    return reqs


def submit_all(sv, reqs, borrow_every=0):
    return [sv.submit(r["g"].xadj, r["g"].adjncy, r["g"].ewgt, r["g"].vwgt, r["k"], r["eps"], r["seed"], r["stop"],
                      borrow=bool(borrow_every) and i % borrow_every == 0)
            for i, r in enumerate(reqs)]


def collect(sv, ids, reqs):
    out = []
    for rid, r in zip(ids, reqs):
        res = sv.wait(rid)
        assert res["status"] == 0
        res.update(sv.fetch(rid, r["g"].n, res["coarsest_n"]))
        out.append(res)
    for rid in ids:
        sv.release(rid)
    return out


def check_against_oracle(r, res):
    g = r["g"]
    ref = O.coarsen(g, "expansion*2", r["seed"], r["stop"])
    assert res["num_levels"] == len(ref.levels)
    c = ref.levels[-1].n
    assert res["coarsest_n"] == c
    cp = initial_partition(c, r["k"], r["seed"])
    assert np.array_equal(res["coarse_part"], cp)
    part = O.project(ref.maps, cp)
    assert np.array_equal(res["part"], part)
    want = O.cut_gain(g, part, r["k"], r["eps"])
    assert res["cut"] == want["cut"]
    assert res["l_max"] == want["L_max"]
    assert res["imbalance"] == want["imbalance"]
    assert res["total_c"] == int(g.vwgt.astype(np.int64).sum())
    assert np.array_equal(res["gain"], want["gain"])
    assert np.array_equal(res["target"], want["target"])


@pytest.mark.parametrize("matcher", ["suitor", "handshake"])
def test_requests_equal_oracle_alone_and_in_the_mix(matcher):
    reqs = request_pool(5)
    with B().Server(workers=1, max_batch=1, matcher=matcher) as alone:
        a = collect(alone, submit_all(alone, reqs), reqs)
    assert all(x["group_size"] == 1 for x in a)
    with B().Server(workers=3, max_batch=16, batch_max_nodes=4096, small_workers=1, matcher=matcher) as mix:
        m = collect(mix, submit_all(mix, reqs, borrow_every=2), reqs)
    assert max(x["group_size"] for x in m) > 1     # some requests did run merged
    for r, x, y in zip(reqs, a, m):
        for key in ("num_levels", "coarsest_n", "cut", "total_c", "l_max", "imbalance"):
            assert x[key] == y[key], (r["g"].name, key)
        for key in ("part", "gain", "target", "coarse_part"):
            assert np.array_equal(x[key], y[key]), (r["g"].name, key)
        check_against_oracle(r, y)


def test_large_requests_run_alone_and_match_oracle():
    reqs = [dict(g=I.rgg2d(20000, 3, wmax=16), k=4, eps=0.03, seed=11, stop=40),
            dict(g=I.grid2d(120, 90), k=2, eps=0.0, seed=12, stop=40),
            dict(g=I.grid2d(9, 9), k=2, eps=0.0, seed=13, stop=40)]
    with B().Server(workers=2, max_batch=8, batch_max_nodes=1000) as sv:
        res = collect(sv, submit_all(sv, reqs), reqs)
    assert res[0]["group_size"] == 1 and res[1]["group_size"] == 1
    for r, x in zip(reqs, res):
        check_against_oracle(r, x)


def test_admission_waits_for_released_budget():
    g = I.grid2d(40, 40)
    # a budget below one request's footprint: a request runs only when nothing
    # else is charged, and a resident result stays charged until released
    with B().Server(workers=2, max_batch=1, hbm_budget_bytes=1) as sv:
        ids = [sv.submit(g.xadj, g.adjncy, g.ewgt, g.vwgt, 2, 0.03, s, 40) for s in range(3)]
        first = sv.wait(ids[0])
        time.sleep(0.3)
        done, _ = sv.poll(ids[1])
        assert not done
        sv.release(ids[0])
        second = sv.wait(ids[1])
        assert second["t_admit_us"] >= first["t_done_us"]
        sv.release(ids[1])
        third = sv.wait(ids[2])
        assert third["t_admit_us"] >= second["t_done_us"]
        sv.release(ids[2])


def test_younger_results_do_not_hold_back_the_head():
    """A large request H waits behind an older resident result X; a small
    request Y (younger) runs past it on the small-request worker and stays
    resident.  Once X is released, H starts although Y is still resident (a
    client releasing in submission order waits for H before releasing Y)."""
    big = I.grid2d(40, 40)     # 1600 nodes: above batch_max_nodes
    small = I.grid2d(10, 10)
    res_x = 88 * big.n + 40 * big.nnz + (1 << 20)
    run_y = 148 * small.n + 57 * small.nnz + (2 << 20)
    budget = res_x + run_y      # X resident + Y running fit; X + H and Y + H do not
    with B().Server(workers=2, small_workers=1, max_batch=1, batch_max_nodes=1000, hbm_budget_bytes=budget,
                    tail_nodes=-1) as sv:
        ix = sv.submit(big.xadj, big.adjncy, big.ewgt, big.vwgt, 2, 0.03, 1, 40)
        sv.wait(ix)
        ih = sv.submit(big.xadj, big.adjncy, big.ewgt, big.vwgt, 2, 0.03, 2, 40)
        iy = sv.submit(small.xadj, small.adjncy, small.ewgt, small.vwgt, 2, 0.03, 3, 40)
        ry = sv.wait(iy)
        assert ry["status"] == 0
        done, _ = sv.poll(ih)
        assert not done          # X is older and still charged
        sv.release(ix)
        deadline = time.time() + 30
        while not sv.poll(ih)[0] and time.time() < deadline:
            time.sleep(0.01)
        assert sv.poll(ih)[0], "the head waited for a younger resident result"
        rh = sv.wait(ih)
        assert rh["status"] == 0 and rh["t_admit_us"] >= ry["t_done_us"]
        sv.release(ih)
        sv.release(iy)


def test_fifo_order_and_errors():
    g = I.grid2d(20, 20)
    with B().Server(workers=1, max_batch=1) as sv:
        ids = [sv.submit(g.xadj, g.adjncy, g.ewgt, g.vwgt, 2, 0.03, s, 40) for s in range(6)]
        res = [sv.wait(i) for i in ids]
        admits = [r["t_admit_us"] for r in res]
        assert admits == sorted(admits)
        with pytest.raises(B().KpError) as e:
            sv.submit(g.xadj, g.adjncy, g.ewgt, g.vwgt, 0, 0.03, 1, 40)      # k < 1
        assert e.value.status == B().KP_ERR_INVALID
        sv.release(ids[0])
        with pytest.raises(B().KpError) as e:
            sv.fetch(ids[0], g.n, 1)                                          # released
        assert e.value.status == B().KP_ERR_INVALID
        with pytest.raises(B().KpError):
            sv.wait(10 ** 9)                                                   # unknown id
        for i in ids[1:]:
            sv.release(i)
    with pytest.raises(B().KpError) as e:
        B().Server(workers=0)
    assert e.value.status == B().KP_ERR_INVALID
    with pytest.raises(B().KpError) as e:
        B().Server(workers=2, small_workers=2)        # nobody left for large requests
    assert e.value.status == B().KP_ERR_INVALID


def test_spare_arena_chunks_are_charged_until_release():
    """An R-MAT request shrinks slowly and takes spare arena chunks beyond its
    footprint estimate; they are charged to the budget as they are taken, so
    a request that fits the estimate but not the chunks waits for release."""
    a = I.rmat(15, 4)
    small = I.grid2d(20, 20)
    # every level launched on its own: the host supplies spare chunks ahead of need
    with B().Server(workers=1, max_batch=1, tail_nodes=-1) as sv:
        ra = sv.wait(sv.submit(a.xadj, a.adjncy, a.ewgt, a.vwgt, 4, 0.03, 5, 40))
    grown = ra["arena_grown_bytes"]
    assert grown > 0
    resident_a = 88 * a.n + 40 * a.nnz + (1 << 20)
    running_small = 148 * small.n + 57 * small.nnz + (2 << 20)
    budget = resident_a + running_small + grown // 2   # enough without the chunks, too little with them
    with B().Server(workers=2, max_batch=1, hbm_budget_bytes=budget, tail_nodes=-1) as sv:
        ia = sv.submit(a.xadj, a.adjncy, a.ewgt, a.vwgt, 4, 0.03, 5, 40)
        ra2 = sv.wait(ia)
        assert ra2["arena_grown_bytes"] == grown
        ib = sv.submit(small.xadj, small.adjncy, small.ewgt, small.vwgt, 2, 0.03, 1, 40)
        time.sleep(0.3)
        done, _ = sv.poll(ib)
        assert not done, "admitted although the spare chunks exhaust the budget"
        sv.release(ia)
        rb = sv.wait(ib)
        assert rb["status"] == 0 and rb["t_admit_us"] >= ra2["t_done_us"]
        sv.release(ib)
