#!/usr/bin/env python3
"""Benchmark of the whole data-parallel path on one synthetic workload.

A step is one pass of the path: coarsen the input level after level (rating,
handshake matching, contraction), partition the coarsest graph (a seeded
random balanced partition on the host, standing in for initial
partitioning), project it back to the input, and evaluate cut, block weights
and gains.  The metric is coarsened input edges per second (m_0 undirected
edges per step / step time), aggregated over all ranks.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload grid256]
  python bench.py --impl reference ...   (the CPU oracle, timed on the host)

Multi-GPU (torchrun): every rank coarsens its own replica of the workload
(independent problems, no collective on the data path), rank 0 prints one
JSON line with the max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_0910_2004_gb300 import inputs as I  # noqa: E402

L2_FLUSH_BYTES = 512 << 20   # > 129 MB L2

# DRAM bytes (read + write) per step of a workload's dominant phase, from ncu
# captures of the current kernels (dram__bytes_read.sum + dram__bytes_write.sum
# summed over the phase's launches); a phase without an entry reports traffic
# null.  The summaries under profiles/ give the commands and the scaling.
NCU_TRAFFIC = {("grid256", "match"): 4_235_000_000}
HBM_PEAK_FALLBACK = 6800.0


def workloads():
    return {
        "rgg20": dict(
            desc="2D random geometric graph, n=2^20 uniform points, radius for mean degree 6, unit int32 "
                 "weights, expansion*2 rating, full hierarchy to <= 20*64 nodes, cut/gain k=64 eps=0.03",
            make=lambda: I.rgg2d(1 << 20, 1), rating="expansion*2", k=64, eps=0.03),
        "rgg22": dict(
            desc="2D random geometric graph, n=2^22 uniform points, radius for mean degree 6, unit int32 "
                 "weights, expansion*2 rating, full hierarchy to <= 20*64 nodes, cut/gain k=64 eps=0.03",
            make=lambda: I.rgg2d(1 << 22, 1), rating="expansion*2", k=64, eps=0.03,
            sample=("the same generator at n=2^20", lambda: I.rgg2d(1 << 20, 1))),
        "rmat22": dict(
            desc="R-MAT graph, scale 22 (a=0.57, b=0.19, c=0.19, edge factor 16, self loops dropped, duplicates "
                 "merged into integer weights; the largest graph of the served mix), unit node weights, expansion*2, "
                 "hierarchy to <= 20*64 nodes or until a level shrinks by less than 5%, cut/gain k=64 eps=0.03",
            make=lambda: I.rmat_torch(22, 1022), rating="expansion*2", k=64, eps=0.03,
            sample=("the same generator at scale 17", lambda: I.rmat(17, 1017))),
        "batch4096": dict(
            desc="batched: 4,096 independent 2D random geometric graphs, n log-uniform in [1k, 64k], mean degree 6, "
                 "integer edge weights uniform in [1,16], expansion*2, each graph coarsened to <= 20*2 nodes in one "
                 "batch (union) call, per-graph seed = graph index, random balanced 2-way partitions projected back",
            make=None, rating="expansion*2", k=2, eps=0.03, batch=4096),
        "grid64": dict(
            desc="2D 5-point grid 64x64, unit weights, expansion*2, coarsen to <= 20*2 nodes, cut/gain k=2 eps=0.03",
            make=lambda: I.grid2d(64, 64), rating="expansion*2", k=2, eps=0.03),
        "served": dict(
            desc="served: Poisson stream of coarsen+partition+project+cut/gain requests drawn uniformly from a pool "
                 "of 2D/3D grids, 2D random geometric graphs and R-MAT graphs (a=0.57, b=0.19, c=0.19, edge factor "
                 "16, duplicates merged into weights) with 2^12..2^22 nodes, k = 2^U{1..6}, stop at 20k nodes, "
                 "eps=0.03; first saturated, then at 50% and 90% of the saturated request rate",
            make=None, rating="expansion*2", k=None, eps=0.03, served=True),
        "grid256": dict(
            desc="3D 7-point grid 256^3, unit weights, innerOuter, full hierarchy to <= 20*256 nodes, "
                 "cut/gain k=256 eps=0.03",
            make=lambda: I.grid3d(256, 256, 256), rating="innerOuter", k=256, eps=0.03,
            sample=("the same generator at 64^3", lambda: I.grid3d(64, 64, 64))),
        "grid256h": dict(
            desc="3D 7-point grid 256x256x128 (half of the 256^3 grid, for counter captures that must stay a few GB), "
                 "unit weights, innerOuter, full hierarchy to <= 20*256 nodes, cut/gain k=256 eps=0.03",
            make=lambda: I.grid3d(256, 256, 128), rating="innerOuter", k=256, eps=0.03,
            sample=("the same generator at 64^3", lambda: I.grid3d(64, 64, 64))),
    }


def ranks_max(x: float, dist, device) -> float:
    """The maximum of x over all ranks (x itself without a process group)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return HBM_PEAK_FALLBACK, "fallback"


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu_index = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.gpu_index), "-lms", "100"], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, val in zip(names, parts[5:9]):
                    if val.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# algorithmic bytes (int32 ids/weights), per phase, from the level sizes
# ---------------------------------------------------------------------------
def algorithmic_bytes(sizes, rating):
    """sizes: [(n_l, nnz_l)] for l = 0..L.  Bytes the method must move:
    match   read the fine CSR once (xadj, adjncy, ewgt), c (and Out), write match
    relabel read match, write map and c'
    contract read the fine CSR again, write the coarse rows
    csr     write the coarse xadj"""
    out = {"match": 0, "relabel": 0, "contract": 0, "csr": 0, "out": 0}
    if rating == "innerOuter" and sizes:
        n0, nnz0 = sizes[0]
        out["out"] = 4 * (n0 + 1) + 4 * nnz0 + 4 * n0
    for (n, nnz), (n2, nnz2) in zip(sizes, sizes[1:]):
        out["match"] += 4 * (n + 1) + 8 * nnz + 4 * n + 4 * n + (4 * n if rating == "innerOuter" else 0)
        out["relabel"] += 4 * n + 4 * n + 4 * n2
        out["contract"] += 4 * (n + 1) + 8 * nnz + 8 * nnz2 + (4 * n2 if rating == "innerOuter" else 0)
        out["csr"] += 4 * (n2 + 1) + 8 * nnz2
    return out


def eval_bytes(n, nnz, k):
    # cut/gain: xadj, adjncy, ewgt, part of the row ends (gathered), c, part; writes gain, target; block weights
    return 4 * (n + 1) + 8 * nnz + 4 * nnz + 4 * n + 4 * n + 12 * n + 8 * k


# ---------------------------------------------------------------------------
# reference arm: the oracle on the host cores
# ---------------------------------------------------------------------------
def oracle_step(g, wl, seed=1):
    import oracle as O
    k = wl["k"]
    h = O.coarsen(g, wl["rating"], 1, 20 * k)
    cpart = I.random_balanced_partition(h.levels[-1].n, k, seed)
    part = O.project(h.maps, cpart)
    r = O.cut_gain(g, part, k, wl["eps"])
    return h, r


def oracle_sample(wl, g):
    """The graph the oracle runs on: the workload's own, or for the largest
    workloads the same generator at a size the oracle finishes in seconds."""
    if "sample" in wl:
        what, make = wl["sample"]
        return make(), what
    return g, "the whole workload"


def run_reference(args, wl, g):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    g, what = oracle_sample(wl, g)
    for _ in range(max(0, min(args.warmup, 1))):
        oracle_step(g, wl)
    times = []
    for _ in range(args.steps):
        t = time.perf_counter()
        oracle_step(g, wl)
        times.append(time.perf_counter() - t)
    total = sum(times)
    value = g.m * args.steps / total
    line = {
        "impl": "reference", "metric": "coarsened edges/s (full hierarchy)", "value": value, "unit": "edges/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000 * total / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": args.workload, "desc": wl["desc"]},
        "graph": {"n": g.n, "m": g.m, "of": what},
        "cpu_baseline": {"value": value, "unit": "edges/s", "cores": 1, "kind": "oracle",
                         "sample": f"{what} per step ({args.steps} steps), single-threaded C/numpy oracle"},
        "e2e": {"value": value, "unit": "edges/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="grid256", choices=sorted(workloads()))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-matchers", action="store_true",
                    help="skip the side comparison of the matchers (kept out of launch-list captures)")
    ap.add_argument("--e2e-steps", type=int, default=None)
    ap.add_argument("--matcher", default="suitor", choices=["suitor", "handshake", "gpa"])
    ap.add_argument("--tail-nodes", type=int, default=0)
    ap.add_argument("--sort-shared-max", type=int, default=0, help="served: the server's sort_shared_max (0: built-in)")
    ap.add_argument("--no-tune", action="store_true", help="built-in knobs instead of the autotuner's")
    ap.add_argument("--requests", type=int, default=None, help="served: requests per load phase")
    ap.add_argument("--workers", type=int, default=4, help="served: server workers")
    ap.add_argument("--small-workers", type=int, default=1, help="served: workers kept for small requests")
    ap.add_argument("--repeats", type=int, default=3, help="served: repeats of each loaded phase")
    args = ap.parse_args()
    wl = workloads()[args.workload]
    if wl.get("batch"):
        return run_batch(args, wl)
    if wl.get("served"):
        return run_served(args, wl)
    if args.impl == "reference":
        # the oracle runs on the workload's sample where it has one: the full
        # graph is not built then
        return run_reference(args, wl, None if "sample" in wl else wl["make"]())
    g = wl["make"]()

    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    import __graft_entry__
    __graft_entry__.build()
    from paper_0910_2004_gb300 import binding as B

    k, eps, rating = wl["k"], wl["eps"], wl["rating"]
    stop = 20 * k
    dg = B.DeviceGraph.from_csr(g)
    fine = torch.empty(g.n, dtype=torch.int32, device="cuda")
    bw = torch.empty(k, dtype=torch.int64, device="cuda")
    gain = torch.empty(g.n, dtype=torch.int64, device="cuda")
    target = torch.empty(g.n, dtype=torch.int32, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    # the tuning knobs, measured on this graph (cached per GPU and shape class)
    knobs = {"matcher": args.matcher, "tail_nodes": args.tail_nodes}
    tuning = {"knobs": "built-in (--no-tune)"}
    if not args.no_tune:
        cache = os.path.join(os.path.expanduser("~"), ".cache", "paper_0910_2004_gb300", "tune.json")
        t_tune = time.perf_counter()
        knobs, trials, from_cache = B.autotune(dg, reps=2, cache=cache, rating=rating, stop_size=stop,
                                               matcher=args.matcher)
        tuning = {"knobs": knobs, "trials": len(trials), "from_cache": from_cache,
                  "seconds": time.perf_counter() - t_tune}

    def step(seed, validate=False, want_sizes=False):
        h = B.coarsen(dg, rating=rating, seed=1, stop_size=stop, validate=validate, profile=True, **knobs)
        L = h.num_levels()
        top, _ = B.kp_hierarchy_level(h.handle, L - 1)
        if top.n > (1 << 16):
            # a large coarsest level (power-law graphs stop while still large):
            # the same seeded random balanced partition, drawn on the device
            cpart = I.batch_partition_torch([top.n], k, seed)[0]
        else:
            cpart = torch.from_numpy(I.random_balanced_partition(top.n, k, seed)).to("cuda", non_blocking=False)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev2 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        h.project(cpart, fine)
        ev1.record(stream)
        res = B.cut_gain(dg, fine, k, eps, block_w=bw, gain=gain, target=target)
        ev2.record(stream)
        tot = h.profile()
        prof, launches = tot["phase_ms"], tot["launches"]
        sizes = None
        if want_sizes:
            sizes = []
            for l in range(L):
                gl, _ = B.kp_hierarchy_level(h.handle, l)
                sizes.append((gl.n, gl.nnz))
            per_level = []
            for l in range(L - 1):
                lp = h.profile(l)
                per_level.append({"n": lp["n"], "nnz": lp["nnz"], "searches": lp["searches"],
                                  "failed_cas": lp["failed_cas"], "rounds": lp["rounds"],
                                  **{kk + "_ms": round(v, 4) for kk, v in lp["phase_ms"].items() if v}})
            sizes = (sizes, per_level)
        h.free()
        return res, prof, launches + 3, sizes, (ev0, ev1, ev2)

    # warm-up; the first step also checks the input graph on the device (the
    # timed steps take it as checked)
    for w in range(max(args.warmup, 3)):
        step(w, validate=(w == 0))
    sizes, level_profile = step(0, want_sizes=True)[3]
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    sampler = ClockSampler(local)
    sampler.start()
    step_ms, phase_tot, launches_tot = [], {}, 0
    proj_ms = eval_ms = 0.0
    for s in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        res, prof, launches, _, evs = step(100 + s)
        e1.record(stream)
        torch.cuda.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        for kk, v in prof.items():
            phase_tot[kk] = phase_tot.get(kk, 0.0) + v
        proj_ms += evs[0].elapsed_time(evs[1])
        eval_ms += evs[1].elapsed_time(evs[2])
        launches_tot += launches
    clocks = sampler.stop()
    total_ms = ranks_max(sum(step_ms), dist, "cuda")
    if dist:
        dist.barrier()

    # the refinement-side helpers (Section 5) on the last projected partition:
    # quotient graph and the bounded boundary search at the strong setting's
    # depth 20 (not part of the step; reported beside it)
    refine = {}
    for name, fn, nbytes in [
            ("quotient_graph", lambda: B.quotient_graph(dg, fine, k), 8 * g.n + 12 * g.nnz + 16 * k * k),
            ("boundary_band_depth20", lambda: B.boundary_band(dg, fine, k, 20), 12 * g.n + 8 * g.nnz)]:
        fn()
        times = []
        for _ in range(5):
            flush.zero_()
            a0 = torch.cuda.Event(enable_timing=True)
            a1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a0.record(stream)
            fn()
            a1.record(stream)
            torch.cuda.synchronize()
            times.append(a0.elapsed_time(a1))
        ms = statistics.median(times)
        refine[name] = {"ms": ms, "algorithmic_bytes": nbytes,
                        "achieved_gbs": nbytes / (ms / 1000.0) / 1e9}

    # the other matchers on the same graph (not part of the step; reported
    # beside it): coarsening time, levels and matched pairs of the hierarchy
    matchers = {}
    for mname in (() if args.no_matchers else ("suitor", "gpa")):
        mopts = dict(knobs) if mname == args.matcher else {"matcher": mname}
        mopts["matcher"] = mname
        times, info = [], None
        for rep in range(3):
            flush.zero_()
            a0 = torch.cuda.Event(enable_timing=True)
            a1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a0.record(stream)
            hm = B.coarsen(dg, rating=rating, seed=1, stop_size=stop, validate=False, **mopts)
            a1.record(stream)
            torch.cuda.synchronize()
            times.append(a0.elapsed_time(a1))
            tot = hm.profile()
            info = {"levels": hm.num_levels(), "matched_pairs": int(tot["n"] - B.kp_hierarchy_level(
                hm.handle, hm.num_levels() - 1)[0].n), "rounds": tot["rounds"]}
            hm.free()
        ms = statistics.median(times)
        matchers[mname] = {"coarsen_ms": ms, "edges_per_s": g.m / (ms / 1000.0), **info}

    # end to end through the host-buffer entry point
    e2e_steps = args.e2e_steps if args.e2e_steps is not None else max(3, min(args.steps, 20))
    e2e_line = None
    if e2e_steps > 0:
        pin = {name: torch.from_numpy(np.ascontiguousarray(arr, dtype=np.int32)).pin_memory()
               for name, arr in (("xadj", g.xadj), ("adjncy", g.adjncy), ("ewgt", g.ewgt), ("vwgt", g.vwgt))}
        outs = {"part": torch.empty(g.n, dtype=torch.int32).pin_memory().numpy(),
                "gain": torch.empty(g.n, dtype=torch.int64).pin_memory().numpy(),
                "target": torch.empty(g.n, dtype=torch.int32).pin_memory().numpy(),
                "block_w": torch.empty(k, dtype=torch.int64).pin_memory().numpy()}
        coarse_n = []

        def ip(nc, cw, kk):
            coarse_n.append(nc)
            return I.random_balanced_partition(nc, kk, 7)

        arrs = [pin[x].numpy() for x in ("xadj", "adjncy", "ewgt", "vwgt")]
        B.pipeline_host(*arrs, k, eps, ip, outputs=outs, rating=rating, seed=1, stop_size=stop, **knobs)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        e2e_ms = []
        for s in range(e2e_steps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            B.pipeline_host(*arrs, k, eps, ip, outputs=outs, rating=rating, seed=1, stop_size=stop, **knobs)
            e2e_ms.append(1000 * (time.perf_counter() - t0))
        e2e_total = ranks_max(sum(e2e_ms), dist, "cuda")
        h2d = 4 * (g.n + 1) + 8 * g.nnz + 4 * g.n + 4 * coarse_n[-1]
        d2h = 4 * g.n + 8 * g.n + 4 * g.n + 8 * k + 4 * coarse_n[-1]
        e2e_line = {"value": world * g.m * e2e_steps / (e2e_total / 1000.0), "unit": "edges/s",
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "steps": e2e_steps,
                    "api": "kp_pipeline_host (host pinned buffers, copies inside)"}

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0

    steps = args.steps
    value = world * g.m * steps / (total_ms / 1000.0)
    peak, peak_kind = load_peaks()
    ab = algorithmic_bytes(sizes, rating)
    phase_ms = {kk: v / steps for kk, v in phase_tot.items()}
    cands = {kk: (ab.get(kk, 0), phase_ms.get(kk, 0.0)) for kk in ("match", "relabel", "contract", "csr")}
    # the persistent tail launch: every level from the first one it ran
    first_tail = next((i for i, lp in enumerate(level_profile) if lp.get("tail_ms")), None)
    if first_tail is not None and phase_ms.get("tail", 0.0) > 0:
        cands["tail"] = (sum(v for kk, v in algorithmic_bytes(sizes[first_tail:], rating).items() if kk != "out"),
                         phase_ms["tail"])
        for kk in ("match", "relabel", "contract", "csr"):   # the separate launches cover the levels before it
            cands[kk] = (algorithmic_bytes(sizes[:first_tail + 1], rating).get(kk, 0), phase_ms.get(kk, 0.0))
    cands["cut_gain"] = (eval_bytes(g.n, g.nnz, k), eval_ms / steps)
    dom = max(cands, key=lambda x: cands[x][1])
    dom_bytes, dom_ms = cands[dom]
    achieved = dom_bytes / (dom_ms / 1000.0) / 1e9 if dom_ms > 0 else 0.0
    path_bytes = sum(ab.values()) + eval_bytes(g.n, g.nnz, k) + 8 * g.n
    for v in refine.values():
        v["frac_of_measured_hbm"] = v["achieved_gbs"] / peak
    line = {
        "metric": "coarsened edges/s (full hierarchy)",
        "value": value, "unit": "edges/s", "n_gpus": world, "steps": steps, "warmup": max(args.warmup, 3),
        "ms_per_step": total_ms / steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "int32", "data": "synthetic",
        "config": {"workload": args.workload, "desc": wl["desc"]},
        "graph": {"n": g.n, "m": g.m, "levels": len(sizes), "coarsest_n": sizes[-1][0],
                  "level_n": [s[0] for s in sizes]},
        "run": {"l2": "flushed (512 MB write) before every timed step", "parallelism": f"replicas x{world}",
                "matcher": args.matcher, "input_check": "once before timing (kp_options.validate=0 in timed steps)"},
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_kind": peak_kind,
                     "traffic": NCU_TRAFFIC.get((args.workload, dom)),
                     "algorithmic_bytes_per_step": dom_bytes, "kernel_ms_per_step": dom_ms},
        "path_roofline": {"bytes_per_step": path_bytes, "achieved_gbs": path_bytes / (total_ms / steps / 1000) / 1e9,
                          "frac": path_bytes / (total_ms / steps / 1000) / 1e9 / peak},
        "phase_ms_per_step": {**phase_ms, "project": proj_ms / steps, "cut_gain": eval_ms / steps},
        "tuning": tuning,
        "level_profile": level_profile,
        "clocks": clocks,
        "e2e": e2e_line,
        "refinement_helpers": refine,
        "matchers": matchers,
        "gpu_launches": launches_tot,
    }
    if world == 1 and not args.no_cpu_baseline:
        go, what = oracle_sample(wl, g)
        t0 = time.perf_counter()
        oracle_step(go, wl)
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": go.m / dt, "unit": "edges/s", "cores": 1, "kind": "oracle",
                                "sample": f"one full step (coarsen + project + cut/gain) on {what}, "
                                          "single-threaded C/numpy oracle"}
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


# ---------------------------------------------------------------------------
# batched workload: many independent graphs in one call
# ---------------------------------------------------------------------------
def batch_slices(xadj, adj, ew, vw, off, idx):
    """Host CSRs of the graphs `idx` of a union (numpy)."""
    import numpy as _np
    x, a, w, v, o = [t.cpu().numpy() for t in (xadj, adj, ew, vw, off)]
    out = []
    for gi in idx:
        s0, e0 = int(o[gi]), int(o[gi + 1])
        X = (x[s0:e0 + 1].astype(_np.int64) - x[s0]).astype(_np.int32)
        out.append(I.CSRGraph(X, (a[x[s0]:x[e0]] - s0).astype(_np.int32), w[x[s0]:x[e0]].copy(), v[s0:e0].copy(),
                              f"batch_graph_{gi}"))
    return out


def run_batch(args, wl):
    G = wl["batch"]
    k, eps, rating = wl["k"], wl["eps"], wl["rating"]
    stop = 20 * k
    sizes = I.batch_rgg_sizes(G, seed=1, nmin=1024, nmax=65536)
    if args.impl == "reference":
        rank = int(os.environ.get("RANK", "0"))
        if rank != 0:
            return 0
        import oracle as O
        xadj, adj, ew, vw, off = I.rgg2d_batch(sizes, 1, wmax=16, device="cpu")
        sample = list(range(0, G, max(1, G // 64)))
        graphs = batch_slices(xadj, adj, ew, vw, off, sample)
        msum = sum(g.m for g in graphs)
        times = []
        for _ in range(args.steps):
            t0 = time.perf_counter()
            for gi, g in zip(sample, graphs):
                h = O.coarsen(g, rating, gi, stop)
                p = O.project(h.maps, I.random_balanced_partition(h.levels[-1].n, k, gi))
                O.cut_gain(g, p, k, eps)
            times.append(time.perf_counter() - t0)
        value = msum * args.steps / sum(times)
        print(json.dumps({
            "impl": "reference", "metric": "coarsened edges/s (full hierarchy)", "value": value, "unit": "edges/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000 * sum(times) / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": args.workload, "desc": wl["desc"]},
            "graph": {"graphs": G},
            "cpu_baseline": {"value": value, "unit": "edges/s", "cores": 1, "kind": "oracle",
                             "sample": f"{len(sample)} of the {G} graphs per step, single-threaded oracle"},
            "e2e": {"value": value, "unit": "edges/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}), flush=True)
        return 0

    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import __graft_entry__
    __graft_entry__.build()
    from paper_0910_2004_gb300 import binding as B

    xadj, adj, ew, vw, off = I.rgg2d_batch(sizes, 1, wmax=16, device="cuda")
    n, nnz = int(vw.numel()), int(adj.numel())
    m = nnz // 2
    dg = B.DeviceGraph(xadj, adj, ew, vw)
    seeds = np.arange(G, dtype=np.uint64)
    gidx = torch.repeat_interleave(torch.arange(G, device="cuda", dtype=torch.int32),
                                   (off[1:] - off[:-1]).long())
    fine = torch.empty(n, dtype=torch.int32, device="cuda")
    bw = torch.empty(k * G, dtype=torch.int64, device="cuda")
    gain = torch.empty(n, dtype=torch.int64, device="cuda")
    target = torch.empty(n, dtype=torch.int32, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()

    # the tuning knobs, measured on this batch (cached per GPU and shape class)
    cache = os.path.join(os.path.expanduser("~"), ".cache", "paper_0910_2004_gb300", "tune.json")
    t_tune = time.perf_counter()
    tuned, trials, from_cache = B.autotune(dg, off, seeds, reps=1, cache=cache, rating=rating, stop_size=stop,
                                           matcher=args.matcher)
    t_tune = time.perf_counter() - t_tune
    tuned_plan = dict(tuned)
    # the coarsening recorded into a CUDA graph with the tuned knobs (levels
    # above the tuned tail threshold as separate launches, the rest in one
    # persistent launch)
    plan = B.Plan(dg, off, seeds, rating=rating, stop_size=stop, validate=True, **tuned_plan)

    def step(seed, validate=False, want_profile=False):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        h = plan.run()
        e1.record(stream)
        cs = h.coarsest_sizes()
        cp, co = I.batch_partition_torch(cs, k, seed)
        cp += k * torch.repeat_interleave(torch.arange(G, device="cuda", dtype=torch.int32),
                                          torch.as_tensor(cs, device="cuda").long())   # block ids of the union
        h.project(cp, co, fine)
        res = B.cut_gain(dg, fine, k * G, eps, block_w=bw, gain=gain, target=target)
        tot = h.profile()
        levels = None
        if want_profile:
            levels = []
            for l in range(h.num_levels() - 1):
                lp = h.profile(l)
                levels.append({"n": lp["n"], "nnz": lp["nnz"], "searches": lp["searches"]})
            levels.append({"n": B.kp_hierarchy_level(h.handle, h.num_levels() - 1)[0].n,
                           "nnz": B.kp_hierarchy_level(h.handle, h.num_levels() - 1)[0].nnz})
        return res, tot, (e0, e1), levels

    for wi in range(max(args.warmup, 3)):
        step(wi, validate=(wi == 0))
    _, _, _, level_profile = step(0, want_profile=True)
    union_sizes = [(lp["n"], lp["nnz"]) for lp in level_profile]
    # the whole hierarchy as ONE persistent launch in a recorded graph
    one_ms = []
    with B.Plan(dg, off, seeds, rating=rating, stop_size=stop, validate=False,
                **{**tuned_plan, "tail_nodes": 0x7fffffff}) as plan1:
        for si in range(4):
            a0 = torch.cuda.Event(enable_timing=True)
            a1 = torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            plan1.run()
            a1.record(stream)
            torch.cuda.synchronize()
            one_ms.append(a0.elapsed_time(a1))
    # the same batch through the library's ordinary (non-recorded) call with
    # the tuned knobs, for context
    plain_ms = []
    for si in range(3):
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        hh = B.coarsen_batch(dg, off, seeds, rating=rating, stop_size=stop, validate=False, **tuned)
        a1.record(stream)
        torch.cuda.synchronize()
        hh.free()
        plain_ms.append(a0.elapsed_time(a1))
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    sampler = ClockSampler(local)
    sampler.start()
    step_ms, coarsen_ms, phase_tot, launches = [], [], {}, 0
    for si in range(args.steps):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        res, tot, ev, _ = step(100 + si)
        b.record(stream)
        torch.cuda.synchronize()
        step_ms.append(a.elapsed_time(b))
        coarsen_ms.append(ev[0].elapsed_time(ev[1]))
        launches += tot["launches"] + 4
    clocks = sampler.stop()
    total_ms = ranks_max(sum(step_ms), dist, "cuda")

    # the same graphs coarsened one call each (a sample), for comparison
    sample = list(range(0, G, max(1, G // 128)))
    graphs = batch_slices(xadj, adj, ew, vw, off, sample)
    dgs = [B.DeviceGraph.from_csr(g) for g in graphs]
    for d, gi in zip(dgs[:8], sample[:8]):
        B.coarsen(d, rating=rating, seed=gi, stop_size=stop, validate=False, matcher=args.matcher).free()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for d, gi in zip(dgs, sample):
        B.coarsen(d, rating=rating, seed=gi, stop_size=stop, validate=False, matcher=args.matcher).free()
    b.record(stream)
    torch.cuda.synchronize()
    loop_ms = a.elapsed_time(b)
    loop_m = sum(g.m for g in graphs)

    # end to end from pinned host buffers: copies in, the whole step, results out
    host = [t.cpu().pin_memory() for t in (xadj, adj, ew, vw, off)]
    dev = [torch.empty_like(t) for t in (xadj, adj, ew, vw, off)]
    outs = (torch.empty(n, dtype=torch.int32).pin_memory(), torch.empty(n, dtype=torch.int64).pin_memory())
    dge = B.DeviceGraph(dev[0], dev[1], dev[2], dev[3])
    for hst, d in zip(host, dev):
        d.copy_(hst, non_blocking=True)
    torch.cuda.synchronize()
    plan_e = B.Plan(dge, dev[4], seeds, rating=rating, stop_size=stop, validate=False, **tuned_plan)
    e2e_ms = []
    for si in range(3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for hst, d in zip(host, dev):
            d.copy_(hst, non_blocking=True)
        h = plan_e.run()
        cs = h.coarsest_sizes()
        cp, co = I.batch_partition_torch(cs, k, si)
        cp += k * torch.repeat_interleave(torch.arange(G, device="cuda", dtype=torch.int32),
                                          torch.as_tensor(cs, device="cuda").long())
        h.project(cp, co, fine)
        B.cut_gain(dge, fine, k * G, eps, block_w=bw, gain=gain, target=target)
        outs[0].copy_(fine, non_blocking=True)
        outs[1].copy_(gain, non_blocking=True)
        torch.cuda.synchronize()
        e2e_ms.append(1000 * (time.perf_counter() - t0))
    plan_e.close()
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0
    plan.close()
    steps = args.steps
    peak, peak_kind = load_peaks()
    ab = algorithmic_bytes(union_sizes, rating)
    coarsen_bytes = sum(ab.values())
    coarsen_ms_avg = sum(coarsen_ms) / steps
    achieved = coarsen_bytes / (coarsen_ms_avg / 1000.0) / 1e9
    line = {
        "metric": "coarsened edges/s (full hierarchy)",
        "value": world * m * steps / (total_ms / 1000.0), "unit": "edges/s", "n_gpus": world, "steps": steps,
        "warmup": max(args.warmup, 3), "ms_per_step": total_ms / steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": args.workload, "desc": wl["desc"]},
        "graph": {"graphs": G, "n": n, "m": m, "union_levels": len(level_profile) + 1},
        "run": {"l2": "inputs larger than L2; also flushed", "matcher": args.matcher,
                "parallelism": f"replicas x{world}"},
        "coarsen_only": {"recorded_plan_edges_per_s": m * steps / (sum(coarsen_ms) / 1000.0),
                         "recorded_plan_ms": coarsen_ms_avg,
                         "unrecorded_call_edges_per_s": m / (min(plain_ms) / 1000.0),
                         "one_persistent_launch_recorded_edges_per_s": m / (min(one_ms[1:]) / 1000.0),
                         "per_graph_loop_edges_per_s": loop_m / (loop_ms / 1000.0),
                         "per_graph_loop_sample_graphs": len(sample),
                         "speedup_vs_loop": (m * steps / sum(coarsen_ms)) / (loop_m / loop_ms)},
        "tuning": {"knobs": tuned, "trials": len(trials), "from_cache": from_cache, "seconds": t_tune},
        "roofline": {"bound": "hbm", "kernel": "the recorded coarsening (all its kernels, graph replay)",
                     "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "peak_kind": peak_kind, "traffic": None, "algorithmic_bytes_per_step": coarsen_bytes,
                     "kernel_ms_per_step": coarsen_ms_avg},
        "level_profile": level_profile,
        "clocks": clocks,
        "e2e": {"value": world * m * len(e2e_ms) / (sum(e2e_ms) / 1000.0), "unit": "edges/s",
                "h2d_bytes_per_step": sum(t.numel() * t.element_size() for t in host),
                "d2h_bytes_per_step": 12 * n, "steps": len(e2e_ms),
                "api": "kp_plan_run (recorded batch) + kp_project_batch + kp_cut_gain, inputs copied from pinned "
                       "host memory into the plan's input buffers every step"},
        "gpu_launches": launches,
    }
    if world == 1 and not args.no_cpu_baseline:
        import oracle as O
        osample = sample[:32]
        og = graphs[:32]
        t0 = time.perf_counter()
        for gi, g in zip(osample, og):
            h = O.coarsen(g, rating, gi, stop)
            p = O.project(h.maps, I.random_balanced_partition(h.levels[-1].n, k, gi))
            O.cut_gain(g, p, k, eps)
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": sum(g.m for g in og) / dt, "unit": "edges/s", "cores": 1, "kind": "oracle",
                                "sample": f"{len(og)} of the {G} graphs (every {G // 128}th), single-threaded oracle"}
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


# ---------------------------------------------------------------------------
# served workload: a request stream through the library's request server
# ---------------------------------------------------------------------------
def served_requests(pool, count, seed):
    """(pool index, k, eps, seed, stop size) of `count` requests: pool entry
    uniform, k = 2^U{1..6}, stop at 20k nodes."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for _ in range(count):
        pi = int(rng.integers(len(pool)))
        k = int(2 ** int(rng.integers(1, 7)))
        out.append((pi, k, 0.03, int(rng.integers(1, 1 << 62)), 20 * k))
    return out


def pin_pool(pool):
    """The pool's arrays in page-locked host memory, as a client that stages
    its requests in pinned buffers has them: the server's host-to-device
    copies then run at the host link's rate instead of through the driver's
    pageable path.  Returns the pool and the tensors that own the memory."""
    import torch
    keep, out = [], []
    for fam, sc, g in pool:
        arrs = []
        for a in (g.xadj, g.adjncy, g.ewgt, g.vwgt):
            t = torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
            keep.append(t)
            arrs.append(t.numpy())
        out.append((fam, sc, I.CSRGraph(*arrs, g.name)))
    return out, keep


def poisson_arrivals(count, rate, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.cumsum(rng.exponential(1.0 / rate, size=count))


def serve_phase(sv, pool, reqs, arrivals, borrow=True, stall_s=300.0):
    """Submits reqs at the given arrival offsets (seconds; None: all at once)
    while a second thread releases them as they finish (in any order, so no
    finished result stays charged behind an unfinished one).  Latency of a
    request: from its scheduled arrival to its completion (server clock for
    submit..done, plus the lag of the submit call behind the schedule).  A
    phase in which no request finishes for stall_s seconds is an error."""
    import queue
    import threading
    q = queue.Queue()
    results = [None] * len(reqs)
    failure = []

    def reaper():
        pending, closed, last = {}, False, time.perf_counter()
        while not (closed and not pending):
            try:
                while True:
                    item = q.get_nowait()
                    if item is None:
                        closed = True
                        break
                    i, rid, lag = item
                    pending[rid] = (i, lag)
            except queue.Empty:
                pass
            done = [rid for rid in pending if sv.poll(rid)[0]]
            for rid in done:
                i, lag = pending.pop(rid)
                res = sv.wait(rid)
                sv.release(rid)
                res["lag_s"] = lag
                results[i] = res
            now = time.perf_counter()
            if done:
                last = now
            elif pending and now - last > stall_s:
                failure.append(f"no request finished for {stall_s:.0f} s ({len(pending)} pending)")
                return
            if not done:
                time.sleep(0.0002)

    th = threading.Thread(target=reaper)
    th.start()
    t0 = time.perf_counter()
    for i, (pi, k, eps, seed, stop) in enumerate(reqs):
        g = pool[pi][2]
        if arrivals is not None:
            dt = t0 + arrivals[i] - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
        lag = 0.0 if arrivals is None else max(0.0, time.perf_counter() - (t0 + arrivals[i]))
        rid = sv.submit(g.xadj, g.adjncy, g.ewgt, g.vwgt, k, eps, seed, stop, borrow=borrow)
        q.put((i, rid, lag))
    q.put(None)
    th.join()
    if failure:
        raise RuntimeError("served phase stalled: " + failure[0])
    lat = np.array([(r["t_done_us"] - r["t_submit_us"]) / 1000.0 + 1000.0 * r["lag_s"] for r in results])
    span_s = (max(r["t_done_us"] for r in results) - min(r["t_submit_us"] for r in results)) / 1e6
    m = sum(pool[pi][2].m for pi, *_ in reqs)
    groups = {}
    for r in results:
        groups[r["group_id"]] = (r["launches"], r["group_size"])
    assert all(r["status"] == 0 for r in results)
    return {"requests": len(reqs), "edges": m, "span_s": span_s, "edges_per_s": m / span_s,
            "requests_per_s": len(reqs) / span_s, "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean()),
            "groups": len(groups), "mean_group_size": len(reqs) / max(1, len(groups)),
            "launches": sum(v[0] for v in groups.values())}


def replay_fifo(arrivals, service):
    """Latencies of a single FIFO server (the per-graph path, one request at
    a time) for given arrival times and service times (seconds)."""
    t, lat = 0.0, []
    for a, s in zip(arrivals, service):
        t = max(t, a) + s
        lat.append(t - a)
    return np.array(lat) * 1000.0


def run_served(args, wl):
    eps, rating = wl["eps"], wl["rating"]
    R = args.requests if args.requests is not None else max(200, 8 * args.steps)
    if args.impl == "reference":
        rank = int(os.environ.get("RANK", "0"))
        if rank != 0:
            return 0
        import oracle as O
        pool = I.served_mix(range(12, 17), seed=1, device="cpu")
        reqs = served_requests(pool, 64, seed=3)
        times, msum = [], 0
        for _ in range(args.steps):
            t0 = time.perf_counter()
            msum = 0
            for pi, k, e, sd, stop in reqs[:16]:
                g = pool[pi][2]
                h = O.coarsen(g, rating, sd, stop)
                O.cut_gain(g, O.project(h.maps, I.random_balanced_partition(h.levels[-1].n, k, 1)), k, e)
                msum += g.m
            times.append(time.perf_counter() - t0)
        value = msum * args.steps / sum(times)
        print(json.dumps({
            "impl": "reference", "metric": "served edges/s", "value": value, "unit": "edges/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000 * sum(times) / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": args.workload, "desc": wl["desc"]},
            "cpu_baseline": {"value": value, "unit": "edges/s", "cores": 1, "kind": "oracle",
                             "sample": "16 requests of the mix restricted to 2^12..2^16 nodes per step, "
                                       "one after another, single-threaded oracle"},
            "e2e": {"value": value, "unit": "edges/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}),
            flush=True)
        return 0

    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import __graft_entry__
    __graft_entry__.build()
    from paper_0910_2004_gb300 import binding as B

    pool, pinned = pin_pool(I.served_mix(range(12, 23), seed=1, device="cuda"))
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    free, _ = torch.cuda.mem_get_info()
    budget = int(free * 0.6)
    sat_reqs = served_requests(pool, R, seed=11)
    load_reqs = {0.5: served_requests(pool, R, seed=12), 0.9: served_requests(pool, R, seed=13)}

    sv = B.Server(workers=args.workers, max_batch=64, batch_max_nodes=1 << 16, hbm_budget_bytes=budget,
                  small_workers=args.small_workers, rating=rating, validate=False, matcher=args.matcher,
                  tail_nodes=args.tail_nodes, sort_shared_max=args.sort_shared_max)
    # warm-up: every pool graph once (allocator pool, library state)
    for _ in range(max(1, min(args.warmup, 2))):
        serve_phase(sv, pool, [(pi, 2, eps, 1, 40) for pi in range(len(pool))], None)
    if dist:
        dist.barrier()
    sampler = ClockSampler(local)
    sampler.start()
    sat = serve_phase(sv, pool, sat_reqs, None)
    loads = {}
    for load, reqs in load_reqs.items():
        # the loaded phases are repeated with other arrival draws; the line
        # reports every repeat and their medians
        rate = load * sat["requests_per_s"]
        reps = []
        for rep in range(max(1, args.repeats)):
            arr = poisson_arrivals(R, rate, seed=int(load * 100) + 1000 * rep)
            ph = serve_phase(sv, pool, reqs, arr)
            ph["arrivals"] = arr
            reps.append(ph)
        med = dict(reps[len(reps) // 2])
        for key in ("p50_ms", "p99_ms", "edges_per_s", "requests_per_s", "span_s", "mean_ms"):
            med[key] = float(np.median([r[key] for r in reps]))
        med["repeats"] = [{key: r[key] for key in ("p50_ms", "p99_ms", "edges_per_s", "span_s")} for r in reps]
        med["offered_requests_per_s"] = rate
        med["arrivals"] = reps[len(reps) // 2]["arrivals"]
        loads[load] = med
    clocks = sampler.stop()
    sv.close()
    # every rank served the same request sequence: the job's time is the
    # slowest rank's span
    for ph in [sat] + list(loads.values()):
        ph["span_s"] = ranks_max(ph["span_s"], dist, "cuda")
        ph["edges_per_s"] = world * ph["edges"] / ph["span_s"]
        ph["requests_per_s"] = world * ph["requests"] / ph["span_s"]

    # the plain per-graph GPU path: kp_pipeline_host, one request after the
    # other; its service times replayed through a FIFO queue at the same
    # arrivals
    def ip(nc, cw, kk):
        return I.random_balanced_partition(nc, kk, 1)

    service = {}
    for pi in sorted({r[0] for rs in [sat_reqs] + list(load_reqs.values()) for r in rs}):
        g = pool[pi][2]
        B.pipeline_host(g.xadj, g.adjncy, g.ewgt, g.vwgt, 2, eps, ip, rating=rating, seed=1, stop_size=40,
                        validate=False, matcher=args.matcher)
    for rs in [sat_reqs] + list(load_reqs.values()):
        for pi, k, e, sd, stop in rs:
            if (pi, k) in service:
                continue
            g = pool[pi][2]
            t0 = time.perf_counter()
            B.pipeline_host(g.xadj, g.adjncy, g.ewgt, g.vwgt, k, e, ip, rating=rating, seed=sd, stop_size=stop,
                            validate=False, matcher=args.matcher)
            service[(pi, k)] = time.perf_counter() - t0
    plain_sat_s = sum(service[(pi, k)] for pi, k, *_ in sat_reqs)
    plain = {"edges_per_s": sat["edges"] / plain_sat_s, "requests_per_s": R / plain_sat_s}
    for load, reqs in load_reqs.items():
        lat = replay_fifo(loads[load]["arrivals"], [service[(pi, k)] for pi, k, *_ in reqs])
        plain[f"load{int(load * 100)}"] = {"p50_ms": float(np.percentile(lat, 50)),
                                           "p99_ms": float(np.percentile(lat, 99))}

    # algorithmic bytes of the whole path per pool graph and k (level sizes
    # from one coarsening each)
    path_bytes = {}
    for pi, (fam, sc, g) in enumerate(pool):
        dg = B.DeviceGraph.from_csr(g)
        for k in (2, 4, 8, 16, 32, 64):
            h = B.coarsen(dg, rating=rating, seed=1, stop_size=20 * k, validate=False)
            sizes = [(B.kp_hierarchy_level(h.handle, l)[0].n, B.kp_hierarchy_level(h.handle, l)[0].nnz)
                     for l in range(h.num_levels())]
            h.free()
            path_bytes[(pi, k)] = (sum(algorithmic_bytes(sizes, rating).values()) + eval_bytes(g.n, g.nnz, k)
                                   + 8 * g.n)
        del dg
    sat_bytes = sum(path_bytes[(pi, k)] for pi, k, *_ in sat_reqs)
    peak, peak_kind = load_peaks()
    achieved = sat_bytes / sat["span_s"] / 1e9
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0
    for v in loads.values():
        v.pop("arrivals")
    h2d = sum(4 * (pool[pi][2].n + 1) + 8 * pool[pi][2].nnz + 4 * pool[pi][2].n for pi, *_ in sat_reqs) / R
    line = {
        "metric": "served edges/s at 90% load (p50/p99 ms beside)",
        "value": loads[0.9]["edges_per_s"], "unit": "edges/s", "n_gpus": world, "steps": R,
        "warmup": max(1, min(args.warmup, 2)), "ms_per_step": 1000.0 * loads[0.9]["span_s"] / R,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": args.workload, "desc": wl["desc"]},
        "run": {"pool_graphs": len(pool), "requests_per_phase": R, "workers": args.workers, "small_workers": args.small_workers,
                   "max_batch": 64,
                   "host_arrays": "page-locked numpy arrays of the pool, borrowed by the server (KP_REQUEST_BORROW: "
                                  "read by the worker's host-to-device copy, no copy at submit)",
                   "batch_max_nodes": 1 << 16, "hbm_budget_gb": budget / 1e9, "matcher": args.matcher,
                   "l2": "inputs of the large requests exceed L2; no flush between requests (a stream)",
                   "parallelism": f"replicas x{world}", "step": "one request"},
        "served": {"saturated": sat, "load50": loads[0.5], "load90": loads[0.9]},
        "p50_ms": loads[0.9]["p50_ms"], "p99_ms": loads[0.9]["p99_ms"],
        "plain_per_graph_path": {**plain, "api": "kp_pipeline_host per request, serial; latencies by FIFO replay "
                                                 "of measured service times at the same arrivals"},
        "roofline": {"bound": "hbm", "kernel": "whole path, saturated server", "achieved": achieved, "peak": peak,
                     "unit": "GB/s", "frac": achieved / peak, "peak_kind": peak_kind, "traffic": None,
                     "algorithmic_bytes_per_step": sat_bytes / R},
        "clocks": clocks,
        "e2e": {"value": sat["edges_per_s"], "unit": "edges/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": 32, "api": "kp_server_submit from host arrays .. kp_server_wait (saturated); "
                "results stay on the device"},
        "gpu_launches": sat["launches"] + sum(v["launches"] for v in loads.values()),
    }
    if world == 1 and not args.no_cpu_baseline:
        import oracle as O
        small = [r for r in sat_reqs if pool[r[0]][1] <= 16][:24]
        t0 = time.perf_counter()
        for pi, k, e, sd, stop in small:
            g = pool[pi][2]
            h = O.coarsen(g, rating, sd, stop)
            O.cut_gain(g, O.project(h.maps, I.random_balanced_partition(h.levels[-1].n, k, 1)), k, e)
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": sum(pool[r[0]][2].m for r in small) / dt, "unit": "edges/s", "cores": 1,
                                "kind": "oracle", "sample": f"{len(small)} requests of the saturated stream with "
                                                            "<= 2^16 nodes, one after another, single-threaded oracle"}
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
