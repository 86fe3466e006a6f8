"""The bench's reference arm (the oracle on the host cores) prints one JSON
line with the keys of the measurement contract; runs on the CPU."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_reference(workload, steps=1, warmup=0):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", workload,
                          "--steps", str(steps), "--warmup", str(warmup)],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1, out.stdout
    return json.loads(lines[0])


def test_reference_arm_json_line():
    d = run_reference("grid64", steps=2, warmup=1)
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference"
    assert d["steps"] == 2 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["value"] > 0 and d["ms_per_step"] > 0 and d["higher_is_better"] is True
    assert d["config"]["workload"] == "grid64"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0
    # edges/s of the workload's own graph: 64x64 grid, 8,064 undirected edges
    assert d["graph"]["m"] == 8064 and d["unit"] == "edges/s"
    assert d["config"] == {"workload": "grid64", "desc": d["config"]["desc"]}


class _FakeServer:
    """Stands in for binding.Server in the served phase's client logic: each
    request finishes after a scripted number of polls (None: never)."""

    def __init__(self, finish_after):
        self.finish_after = finish_after   # per request, in submission order
        self.polls, self.released, self.next = {}, [], 0
        self.t0 = 0.0

    def submit(self, *args, **kw):
        rid = self.next
        self.next += 1
        self.polls[rid] = 0
        return rid

    def poll(self, rid):
        self.polls[rid] += 1
        lim = self.finish_after[rid]
        return (1 if lim is not None and self.polls[rid] >= lim else 0), {}

    def wait(self, rid):
        assert self.poll(rid)[0], "waited on an unfinished request"
        return {"t_submit_us": 0.0, "t_done_us": 1000.0 * (rid + 1), "status": 0, "group_id": rid, "launches": 1,
                "group_size": 1}

    def release(self, rid):
        self.released.append(rid)


def _pool():
    import numpy as np
    from paper_0910_2004_gb300 import inputs as I
    g = I.grid2d(4, 4)
    return [("grid2d", 4, g)], np


def test_served_client_releases_in_completion_order():
    """A request that finishes early is released before an older one that is
    still running (a result left charged behind an unfinished request could
    hold back the server's queue head)."""
    import bench
    pool, np = _pool()
    sv = _FakeServer([40, 2, 2])     # the first request finishes last
    out = bench.serve_phase(sv, pool, [(0, 2, 0.03, s, 8) for s in range(3)], None)
    assert sv.released[-1] == 0 and sorted(sv.released) == [0, 1, 2]
    assert out["requests"] == 3 and out["edges"] == 3 * pool[0][2].m


def test_served_client_reports_a_stalled_phase():
    import bench
    import pytest
    pool, _ = _pool()
    sv = _FakeServer([1, None])       # the second request never finishes
    with pytest.raises(RuntimeError, match="stalled"):
        bench.serve_phase(sv, pool, [(0, 2, 0.03, s, 8) for s in range(2)], None, stall_s=0.3)
    assert sv.released == [0]
