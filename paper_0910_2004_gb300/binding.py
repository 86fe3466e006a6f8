"""Thin ctypes binding of the C ABI in include/kp.h (argument marshalling only).

Every computation runs in the CUDA library libkp.so, or libkp64.so when the
environment sets KP_OFFSET_BITS=64 before this module is imported (64-bit
entry offsets: graphs of 2^31 entries or more; kp_graph then holds an int64
nnz and int64 row offsets, as KP_WIDE_OFFSETS makes it in C).  The functions
named kp_* mirror the C entry points one to one; the helpers below them only
turn torch CUDA tensors into the plain pointers and sizes the ABI takes.  If
the library has not been built, every call raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
OFFSET_BITS = 64 if os.environ.get("KP_OFFSET_BITS", "32") == "64" else 32
LIB_PATH = os.path.join(HERE, "_build", "libkp64.so" if OFFSET_BITS == 64 else "libkp.so")
XADJ_NP = np.int64 if OFFSET_BITS == 64 else np.int32   # row offsets (kp_eoff)
XADJ_TYPESTR = "<i8" if OFFSET_BITS == 64 else "<i4"

KP_CUT_GAIN_NOALLOC_MAX_K = 16384
KP_REQUEST_BORROW = 1

KP_OK, KP_ERR_INVALID, KP_ERR_OVERFLOW, KP_ERR_OOM, KP_ERR_CUDA, KP_ERR_TIMEOUT, KP_ERR_UNSUPPORTED = range(7)
STATUS_NAMES = ["KP_OK", "KP_ERR_INVALID", "KP_ERR_OVERFLOW", "KP_ERR_OOM", "KP_ERR_CUDA",
                "KP_ERR_TIMEOUT", "KP_ERR_UNSUPPORTED"]
RATINGS = {"expansion*2": 0, "innerOuter": 1, "weight": 2, "expansion": 3, "expansion*": 4}
MATCHERS = {"suitor": 0, "handshake": 1, "gpa": 2}

PHASES = ["validate", "out", "match", "relabel", "contract", "csr", "tail"]

EXPORTED = ["kp_options_default", "kp_coarsen", "kp_hierarchy_num_levels", "kp_hierarchy_level",
            "kp_hierarchy_stats", "kp_hierarchy_profile", "kp_hierarchy_free", "kp_project", "kp_cut_gain", "kp_cut_gain_noalloc", "kp_pipeline_host",
            "kp_coarsen_batch", "kp_hierarchy_batch", "kp_hierarchy_level_offsets", "kp_project_batch",
            "kp_hierarchy_batch_coarsest",
            "kp_server_create", "kp_server_submit", "kp_server_poll", "kp_server_wait", "kp_server_fetch",
            "kp_server_release", "kp_server_cancel", "kp_server_destroy", "kp_autotune",
            "kp_test_fail_allocation", "kp_test_device_bytes_in_use", "kp_plan_create", "kp_plan_run",
            "kp_plan_destroy", "kp_quotient_graph", "kp_boundary_band", "kp_hierarchy_save", "kp_hierarchy_load",
            "kp_last_error", "kp_version", "kp_offset_bits"]


class KpError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{where}: {name}: {msg}")


_c_eoff = ctypes.c_int64 if OFFSET_BITS == 64 else ctypes.c_int32


def check_offset_width(nnz: int, where: str):
    """The 32-bit library's kp_graph holds nnz and the row offsets in int32:
    a graph of 2^31 entries or more is refused here, before ctypes or numpy
    would wrap the values into a smaller, consistent-looking graph."""
    if OFFSET_BITS == 32 and nnz >= 1 << 31:
        raise KpError(KP_ERR_OVERFLOW, where,
                      f"{nnz} entries: 2^31 or more need the 64-bit offsets library (KP_OFFSET_BITS=64)")


def host_offsets(xadj, where: str) -> np.ndarray:
    """Row offsets as a contiguous host array of the library's width; a value
    the width does not hold raises instead of wrapping."""
    a = np.asarray(xadj)
    if a.dtype != XADJ_NP and a.size:
        info = np.iinfo(XADJ_NP)
        if int(a.max()) > info.max or int(a.min()) < info.min:
            raise KpError(KP_ERR_OVERFLOW, where, f"row offsets beyond {OFFSET_BITS} bits")
    return np.ascontiguousarray(a, dtype=XADJ_NP)


class kp_graph(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("nnz", _c_eoff), ("xadj", ctypes.c_void_p),
                ("adjncy", ctypes.c_void_p), ("ewgt", ctypes.c_void_p), ("vwgt", ctypes.c_void_p)]


class kp_options(ctypes.Structure):
    _fields_ = [("rating", ctypes.c_int32), ("seed", ctypes.c_uint64), ("stop_size", ctypes.c_int32),
                ("max_levels", ctypes.c_int32), ("min_shrink_permille", ctypes.c_int32),
                ("spin_limit", ctypes.c_int64), ("validate", ctypes.c_int32), ("profile", ctypes.c_int32),
                ("matcher", ctypes.c_int32), ("arena_bytes", ctypes.c_int64), ("tail_nodes", ctypes.c_int32),
                ("suitor_lanes", ctypes.c_int32), ("tail_block_nodes", ctypes.c_int32),
                ("sort_shared_max", ctypes.c_int32), ("radix_bits", ctypes.c_int32),
                ("cluster_nodes", ctypes.c_int32), ("suitor_blocks", ctypes.c_int32)]

TUNING_KNOBS = ("suitor_lanes", "tail_block_nodes", "sort_shared_max", "radix_bits", "cluster_nodes", "tail_nodes",
                "suitor_blocks", "matcher")


class kp_cut_gain_out(ctypes.Structure):
    _fields_ = [("cut", ctypes.c_int64), ("total_c", ctypes.c_int64), ("max_c", ctypes.c_int64),
                ("l_max", ctypes.c_int64), ("imbalance", ctypes.c_int64), ("block_w", ctypes.c_void_p),
                ("gain", ctypes.c_void_p), ("target", ctypes.c_void_p)]


class kp_level_profile(ctypes.Structure):
    _fields_ = [("phase_ms", ctypes.c_double * 7), ("n", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("searches", ctypes.c_int64), ("failed_cas", ctypes.c_int64), ("launches", ctypes.c_int32),
                ("rounds", ctypes.c_int32)]


class kp_tune_trial(ctypes.Structure):
    _fields_ = [("options", kp_options), ("ms", ctypes.c_double)]


class kp_server_config(ctypes.Structure):
    _fields_ = [("workers", ctypes.c_int32), ("max_batch", ctypes.c_int32), ("batch_max_nodes", ctypes.c_int32),
                ("small_workers", ctypes.c_int32), ("hbm_budget_bytes", ctypes.c_int64), ("options", kp_options)]


class kp_request_params(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int32), ("stop_size", ctypes.c_int32), ("eps", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("flags", ctypes.c_int32), ("pad", ctypes.c_int32)]


class kp_request_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("num_levels", ctypes.c_int32), ("coarsest_n", ctypes.c_int32),
                ("group_size", ctypes.c_int32), ("launches", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("group_id", ctypes.c_int64), ("cut", ctypes.c_int64), ("total_c", ctypes.c_int64),
                ("l_max", ctypes.c_int64), ("imbalance", ctypes.c_int64), ("t_submit_us", ctypes.c_double),
                ("t_admit_us", ctypes.c_double), ("t_done_us", ctypes.c_double),
                ("arena_grown_bytes", ctypes.c_int64)]


kp_initial_partition_fn = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                                           ctypes.c_int32, ctypes.POINTER(ctypes.c_int32), ctypes.c_void_p)

_lib = None
_lock = threading.Lock()


def load(path: str = LIB_PATH):
    """Loads libkp.so; raises if it has not been built (no fallback)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library not built: {path} is missing "
                               "(run `python -c 'import __graft_entry__ as g; g.build()'`)")
        L = ctypes.CDLL(path)
        vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
        L.kp_options_default.argtypes = [ctypes.POINTER(kp_options)]
        L.kp_options_default.restype = None
        L.kp_coarsen.argtypes = [ctypes.POINTER(kp_graph), ctypes.POINTER(kp_options), vp, ctypes.POINTER(vp)]
        L.kp_coarsen.restype = ctypes.c_int
        L.kp_hierarchy_num_levels.argtypes = [vp, ctypes.POINTER(i32)]
        L.kp_hierarchy_num_levels.restype = ctypes.c_int
        L.kp_hierarchy_level.argtypes = [vp, i32, ctypes.POINTER(kp_graph), ctypes.POINTER(vp)]
        L.kp_hierarchy_level.restype = ctypes.c_int
        L.kp_hierarchy_stats.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i64)]
        L.kp_hierarchy_stats.restype = ctypes.c_int
        L.kp_hierarchy_profile.argtypes = [vp, i32, ctypes.POINTER(kp_level_profile)]
        L.kp_hierarchy_profile.restype = ctypes.c_int
        L.kp_hierarchy_free.argtypes = [vp]
        L.kp_hierarchy_free.restype = None
        L.kp_project.argtypes = [vp, vp, vp, vp]
        L.kp_project.restype = ctypes.c_int
        L.kp_cut_gain.argtypes = [ctypes.POINTER(kp_graph), vp, i32, ctypes.c_double,
                                  ctypes.POINTER(kp_cut_gain_out), vp]
        L.kp_cut_gain.restype = ctypes.c_int
        L.kp_cut_gain_noalloc.argtypes = [ctypes.POINTER(kp_graph), vp, i32, ctypes.c_double,
                                          ctypes.POINTER(kp_cut_gain_out), vp]
        L.kp_cut_gain_noalloc.restype = ctypes.c_int
        L.kp_pipeline_host.argtypes = [ctypes.POINTER(kp_graph), ctypes.POINTER(kp_options), i32, ctypes.c_double,
                                       kp_initial_partition_fn, vp, vp, vp, vp, vp,
                                       ctypes.POINTER(kp_cut_gain_out), ctypes.POINTER(i32), vp]
        L.kp_pipeline_host.restype = ctypes.c_int
        L.kp_coarsen_batch.argtypes = [ctypes.POINTER(kp_graph), i32, vp, vp, vp, ctypes.POINTER(kp_options), vp,
                                       ctypes.POINTER(vp)]
        L.kp_coarsen_batch.restype = ctypes.c_int
        L.kp_hierarchy_batch.argtypes = [vp, ctypes.POINTER(i32), vp]
        L.kp_hierarchy_batch.restype = ctypes.c_int
        L.kp_hierarchy_level_offsets.argtypes = [vp, i32, ctypes.POINTER(vp)]
        L.kp_hierarchy_level_offsets.restype = ctypes.c_int
        L.kp_hierarchy_batch_coarsest.argtypes = [vp, vp, vp]
        L.kp_hierarchy_batch_coarsest.restype = ctypes.c_int
        L.kp_project_batch.argtypes = [vp, vp, vp, vp, vp]
        L.kp_project_batch.restype = ctypes.c_int
        L.kp_server_create.argtypes = [ctypes.POINTER(kp_server_config), ctypes.POINTER(vp)]
        L.kp_server_create.restype = ctypes.c_int
        L.kp_server_submit.argtypes = [vp, ctypes.POINTER(kp_graph), ctypes.POINTER(kp_request_params),
                                       ctypes.POINTER(ctypes.c_uint64)]
        L.kp_server_submit.restype = ctypes.c_int
        L.kp_server_poll.argtypes = [vp, ctypes.c_uint64, ctypes.POINTER(i32), ctypes.POINTER(kp_request_result)]
        L.kp_server_poll.restype = ctypes.c_int
        L.kp_server_wait.argtypes = [vp, ctypes.c_uint64, ctypes.POINTER(kp_request_result)]
        L.kp_server_wait.restype = ctypes.c_int
        L.kp_server_fetch.argtypes = [vp, ctypes.c_uint64, vp, vp, vp, vp]
        L.kp_server_fetch.restype = ctypes.c_int
        L.kp_server_release.argtypes = [vp, ctypes.c_uint64]
        L.kp_server_release.restype = ctypes.c_int
        L.kp_server_cancel.argtypes = [vp, ctypes.c_uint64]
        L.kp_server_cancel.restype = ctypes.c_int
        L.kp_test_fail_allocation.argtypes = [i64]
        L.kp_test_fail_allocation.restype = None
        L.kp_test_device_bytes_in_use.argtypes = []
        L.kp_test_device_bytes_in_use.restype = i64
        L.kp_server_destroy.argtypes = [vp]
        L.kp_server_destroy.restype = None
        L.kp_autotune.argtypes = [ctypes.POINTER(kp_graph), i32, vp, vp, vp, ctypes.POINTER(kp_options), i32,
                                  ctypes.POINTER(kp_options), ctypes.POINTER(kp_tune_trial), i32,
                                  ctypes.POINTER(i32), vp]
        L.kp_autotune.restype = ctypes.c_int
        L.kp_plan_create.argtypes = [ctypes.POINTER(kp_graph), i32, vp, vp, vp, ctypes.POINTER(kp_options), vp,
                                     ctypes.POINTER(vp)]
        L.kp_plan_create.restype = ctypes.c_int
        L.kp_plan_run.argtypes = [vp, vp, ctypes.POINTER(vp)]
        L.kp_plan_run.restype = ctypes.c_int
        L.kp_plan_destroy.argtypes = [vp]
        L.kp_plan_destroy.restype = None
        L.kp_quotient_graph.argtypes = [ctypes.POINTER(kp_graph), vp, i32, vp, vp, vp, i64, ctypes.POINTER(i64), vp]
        L.kp_quotient_graph.restype = ctypes.c_int
        L.kp_boundary_band.argtypes = [ctypes.POINTER(kp_graph), vp, i32, i32, i32, i32, vp, vp]
        L.kp_boundary_band.restype = ctypes.c_int
        L.kp_hierarchy_save.argtypes = [vp, ctypes.c_char_p]
        L.kp_hierarchy_save.restype = ctypes.c_int
        L.kp_hierarchy_load.argtypes = [ctypes.c_char_p, vp, ctypes.POINTER(vp)]
        L.kp_hierarchy_load.restype = ctypes.c_int
        L.kp_last_error.argtypes = []
        L.kp_last_error.restype = ctypes.c_char_p
        L.kp_version.argtypes = []
        L.kp_version.restype = ctypes.c_char_p
        L.kp_offset_bits.argtypes = []
        L.kp_offset_bits.restype = ctypes.c_int32
        if L.kp_offset_bits() != OFFSET_BITS:
            raise RuntimeError(f"{path} has {L.kp_offset_bits()}-bit offsets, the binding {OFFSET_BITS}-bit")
        _lib = L
        return L


def _check(status: int, where: str):
    if status != KP_OK:
        raise KpError(status, where, load().kp_last_error().decode(errors="replace"))


# ---------------------------------------------------------------------------
# one wrapper per C entry point
# ---------------------------------------------------------------------------

def kp_options_default() -> kp_options:
    o = kp_options()
    load().kp_options_default(ctypes.byref(o))
    return o


def kp_coarsen(graph: kp_graph, options: kp_options, stream: int) -> int:
    h = ctypes.c_void_p()
    _check(load().kp_coarsen(ctypes.byref(graph), ctypes.byref(options), ctypes.c_void_p(stream),
                             ctypes.byref(h)), "kp_coarsen")
    return h.value


def kp_hierarchy_num_levels(h: int) -> int:
    n = ctypes.c_int32()
    _check(load().kp_hierarchy_num_levels(ctypes.c_void_p(h), ctypes.byref(n)), "kp_hierarchy_num_levels")
    return n.value


def kp_hierarchy_level(h: int, level: int):
    g = kp_graph()
    mp = ctypes.c_void_p()
    _check(load().kp_hierarchy_level(ctypes.c_void_p(h), level, ctypes.byref(g), ctypes.byref(mp)),
           "kp_hierarchy_level")
    return g, mp.value


def kp_hierarchy_stats(h: int):
    r, m = ctypes.c_int32(), ctypes.c_int64()
    _check(load().kp_hierarchy_stats(ctypes.c_void_p(h), ctypes.byref(r), ctypes.byref(m)), "kp_hierarchy_stats")
    return r.value, m.value


def kp_hierarchy_profile(h: int, level: int = -1) -> dict:
    p = kp_level_profile()
    _check(load().kp_hierarchy_profile(ctypes.c_void_p(h), level, ctypes.byref(p)), "kp_hierarchy_profile")
    return {"phase_ms": dict(zip(PHASES, list(p.phase_ms))), "n": p.n, "nnz": p.nnz, "searches": p.searches,
            "failed_cas": p.failed_cas, "launches": p.launches, "rounds": p.rounds}


def kp_hierarchy_free(h: int):
    if h:
        load().kp_hierarchy_free(ctypes.c_void_p(h))


def kp_project(h: int, coarse_part: int, fine_part: int, stream: int):
    _check(load().kp_project(ctypes.c_void_p(h), ctypes.c_void_p(coarse_part), ctypes.c_void_p(fine_part),
                             ctypes.c_void_p(stream)), "kp_project")


def kp_cut_gain(graph: kp_graph, part: int, k: int, eps: float, out: kp_cut_gain_out, stream: int):
    _check(load().kp_cut_gain(ctypes.byref(graph), ctypes.c_void_p(part), k, eps, ctypes.byref(out),
                              ctypes.c_void_p(stream)), "kp_cut_gain")


def kp_cut_gain_noalloc(graph: kp_graph, part: int, k: int, eps: float, out: kp_cut_gain_out, stream: int):
    """kp_cut_gain for callers that cannot allocate: scratch in a static device
    array (k <= KP_CUT_GAIN_NOALLOC_MAX_K); overlapping calls race."""
    _check(load().kp_cut_gain_noalloc(ctypes.byref(graph), ctypes.c_void_p(part), k, eps, ctypes.byref(out),
                                      ctypes.c_void_p(stream)), "kp_cut_gain_noalloc")


def kp_pipeline_host(graph: kp_graph, options: kp_options, k: int, eps: float, ip, user, fine_part: int,
                     gain: int, target: int, block_w: int, out: kp_cut_gain_out, stream: int) -> int:
    nl = ctypes.c_int32()
    _check(load().kp_pipeline_host(ctypes.byref(graph), ctypes.byref(options), k, eps, ip, user,
                                   ctypes.c_void_p(fine_part), ctypes.c_void_p(gain), ctypes.c_void_p(target),
                                   ctypes.c_void_p(block_w), ctypes.byref(out), ctypes.byref(nl),
                                   ctypes.c_void_p(stream)), "kp_pipeline_host")
    return nl.value


def kp_coarsen_batch(graph: kp_graph, num_graphs: int, node_offsets: int, seeds: int, stop_sizes: int,
                     options: kp_options, stream: int) -> int:
    h = ctypes.c_void_p()
    _check(load().kp_coarsen_batch(ctypes.byref(graph), num_graphs, ctypes.c_void_p(node_offsets),
                                   ctypes.c_void_p(seeds), ctypes.c_void_p(stop_sizes), ctypes.byref(options),
                                   ctypes.c_void_p(stream), ctypes.byref(h)), "kp_coarsen_batch")
    return h.value


def kp_hierarchy_batch(h: int):
    ng = ctypes.c_int32()
    _check(load().kp_hierarchy_batch(ctypes.c_void_p(h), ctypes.byref(ng), None), "kp_hierarchy_batch")
    levels = (ctypes.c_int32 * max(ng.value, 1))()
    _check(load().kp_hierarchy_batch(ctypes.c_void_p(h), ctypes.byref(ng), levels), "kp_hierarchy_batch")
    return ng.value, list(levels)[:ng.value]


def kp_hierarchy_level_offsets(h: int, level: int) -> int:
    p = ctypes.c_void_p()
    _check(load().kp_hierarchy_level_offsets(ctypes.c_void_p(h), level, ctypes.byref(p)),
           "kp_hierarchy_level_offsets")
    return p.value


def kp_hierarchy_batch_coarsest(h: int, num_graphs: int, stream: int) -> np.ndarray:
    out = np.empty(max(num_graphs, 1), dtype=np.int32)
    _check(load().kp_hierarchy_batch_coarsest(ctypes.c_void_p(h), ctypes.c_void_p(out.ctypes.data),
                                              ctypes.c_void_p(stream)), "kp_hierarchy_batch_coarsest")
    return out[:num_graphs]


def kp_project_batch(h: int, coarse_part: int, coarse_offsets: int, fine_part: int, stream: int):
    _check(load().kp_project_batch(ctypes.c_void_p(h), ctypes.c_void_p(coarse_part), ctypes.c_void_p(coarse_offsets),
                                   ctypes.c_void_p(fine_part), ctypes.c_void_p(stream)), "kp_project_batch")


def kp_server_create(config: kp_server_config) -> int:
    sv = ctypes.c_void_p()
    _check(load().kp_server_create(ctypes.byref(config), ctypes.byref(sv)), "kp_server_create")
    return sv.value


def kp_server_submit(sv: int, graph: kp_graph, params: kp_request_params) -> int:
    rid = ctypes.c_uint64()
    _check(load().kp_server_submit(sv, ctypes.byref(graph), ctypes.byref(params), ctypes.byref(rid)),
           "kp_server_submit")
    return rid.value


def kp_server_poll(sv: int, rid: int):
    done = ctypes.c_int32()
    res = kp_request_result()
    _check(load().kp_server_poll(sv, rid, ctypes.byref(done), ctypes.byref(res)), "kp_server_poll")
    return bool(done.value), res


def kp_server_wait(sv: int, rid: int) -> kp_request_result:
    res = kp_request_result()
    _check(load().kp_server_wait(sv, rid, ctypes.byref(res)), "kp_server_wait")
    return res


def kp_server_fetch(sv: int, rid: int, fine_part: int, gain: int, target: int, coarse_part: int):
    _check(load().kp_server_fetch(sv, rid, fine_part, gain, target, coarse_part), "kp_server_fetch")


def kp_server_release(sv: int, rid: int):
    _check(load().kp_server_release(sv, rid), "kp_server_release")


def kp_server_cancel(sv: int, rid: int):
    _check(load().kp_server_cancel(sv, rid), "kp_server_cancel")


def kp_test_fail_allocation(after: int):
    load().kp_test_fail_allocation(after)


def kp_test_device_bytes_in_use() -> int:
    return load().kp_test_device_bytes_in_use()


def kp_server_destroy(sv: int):
    load().kp_server_destroy(sv)


def kp_autotune(graph: kp_graph, num_graphs: int, node_offsets: int, seeds: int, stop_sizes: int,
                options: kp_options, reps: int, max_trials: int, stream: int):
    best = kp_options()
    trials = (kp_tune_trial * max(max_trials, 1))()
    nt = ctypes.c_int32()
    _check(load().kp_autotune(ctypes.byref(graph), num_graphs, ctypes.c_void_p(node_offsets), ctypes.c_void_p(seeds),
                              ctypes.c_void_p(stop_sizes), ctypes.byref(options), reps, ctypes.byref(best), trials,
                              max_trials, ctypes.byref(nt), ctypes.c_void_p(stream)), "kp_autotune")
    return best, [trials[i] for i in range(min(nt.value, max_trials))]


def kp_plan_create(graph: kp_graph, num_graphs: int, node_offsets: int, seeds: int, stop_sizes: int,
                   options: kp_options, stream: int) -> int:
    p = ctypes.c_void_p()
    _check(load().kp_plan_create(ctypes.byref(graph), num_graphs, ctypes.c_void_p(node_offsets),
                                 ctypes.c_void_p(seeds), ctypes.c_void_p(stop_sizes), ctypes.byref(options),
                                 ctypes.c_void_p(stream), ctypes.byref(p)), "kp_plan_create")
    return p.value


def kp_plan_run(plan: int, stream: int) -> int:
    h = ctypes.c_void_p()
    _check(load().kp_plan_run(ctypes.c_void_p(plan), ctypes.c_void_p(stream), ctypes.byref(h)), "kp_plan_run")
    return h.value


def kp_plan_destroy(plan: int):
    load().kp_plan_destroy(ctypes.c_void_p(plan))


def kp_quotient_graph(graph: kp_graph, part: int, k: int, q_xadj: int, q_adjncy: int, q_ewgt: int, capacity: int,
                      stream: int) -> int:
    nnz = ctypes.c_int64()
    st = load().kp_quotient_graph(ctypes.byref(graph), ctypes.c_void_p(part), k, ctypes.c_void_p(q_xadj),
                                  ctypes.c_void_p(q_adjncy), ctypes.c_void_p(q_ewgt), capacity, ctypes.byref(nnz),
                                  ctypes.c_void_p(stream))
    if st == KP_ERR_OVERFLOW:
        return -nnz.value - 1   # too small: -(needed) - 1
    _check(st, "kp_quotient_graph")
    return nnz.value


def kp_boundary_band(graph: kp_graph, part: int, k: int, depth: int, pair_a: int, pair_b: int, dist: int,
                     stream: int):
    _check(load().kp_boundary_band(ctypes.byref(graph), ctypes.c_void_p(part), k, depth, pair_a, pair_b,
                                   ctypes.c_void_p(dist), ctypes.c_void_p(stream)), "kp_boundary_band")


def kp_hierarchy_save(h: int, path: str):
    _check(load().kp_hierarchy_save(ctypes.c_void_p(h), os.fsencode(path)), "kp_hierarchy_save")


def kp_hierarchy_load(path: str, stream: int) -> int:
    h = ctypes.c_void_p()
    _check(load().kp_hierarchy_load(os.fsencode(path), ctypes.c_void_p(stream), ctypes.byref(h)),
           "kp_hierarchy_load")
    return h.value


def kp_last_error() -> str:
    return load().kp_last_error().decode(errors="replace")


def kp_version() -> str:
    return load().kp_version().decode()


# ---------------------------------------------------------------------------
# torch helpers (marshalling only)
# ---------------------------------------------------------------------------

def _torch():
    import torch
    return torch


def current_stream() -> int:
    return _torch().cuda.current_stream().cuda_stream


class _DevArray:
    """Zero-copy view of a library-owned device array (CUDA array interface)."""

    def __init__(self, ptr: int, n: int, typestr: str = "<i4"):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr, "data": (ptr or 0, False),
                                         "version": 3, "strides": None}


def device_view(ptr: int, n: int, dtype: str = "<i4"):
    torch = _torch()
    if n == 0:
        return torch.empty(0, dtype=torch.int32 if dtype == "<i4" else torch.int64, device="cuda")
    return torch.as_tensor(_DevArray(ptr, n, dtype), device="cuda")


class DeviceGraph:
    """A CSR graph held in torch CUDA tensors (int32; the row offsets in the
    library's offset width), with its kp_graph."""

    def __init__(self, xadj, adjncy, ewgt, vwgt):
        torch = _torch()
        dev = torch.device("cuda")
        xt = torch.int64 if OFFSET_BITS == 64 else torch.int32
        if torch.is_tensor(xadj):
            if xadj.dtype != xt and xadj.element_size() > 4 and xadj.numel() and int(xadj.max()) >= 1 << 31:
                raise KpError(KP_ERR_OVERFLOW, "DeviceGraph", f"row offsets beyond {OFFSET_BITS} bits")
            self.xadj = xadj if xadj.dtype == xt else xadj.to(xt).contiguous()
        else:
            self.xadj = torch.as_tensor(host_offsets(xadj, "DeviceGraph")).to(dev)
        self.adjncy = torch.as_tensor(np.asarray(adjncy, dtype=np.int32)).to(dev) if not torch.is_tensor(adjncy) else adjncy
        self.ewgt = torch.as_tensor(np.asarray(ewgt, dtype=np.int32)).to(dev) if not torch.is_tensor(ewgt) else ewgt
        self.vwgt = torch.as_tensor(np.asarray(vwgt, dtype=np.int32)).to(dev) if not torch.is_tensor(vwgt) else vwgt
        for t in (self.adjncy, self.ewgt, self.vwgt):
            assert t.dtype == torch.int32 and t.is_cuda and t.is_contiguous()
        assert self.xadj.dtype == xt and self.xadj.is_cuda and self.xadj.is_contiguous()
        self.n = int(self.xadj.numel() - 1)
        self.nnz = int(self.adjncy.numel())
        check_offset_width(self.nnz, "DeviceGraph")
        self.kp = kp_graph(self.n, self.nnz, self.xadj.data_ptr(), self.adjncy.data_ptr(),
                           self.ewgt.data_ptr(), self.vwgt.data_ptr())

    @classmethod
    def from_csr(cls, g):
        return cls(g.xadj, g.adjncy, g.ewgt, g.vwgt)


def make_options(rating="expansion*2", seed=1, stop_size=40, max_levels=64, min_shrink_permille=50,
                 spin_limit=1 << 22, validate=True, profile=False, matcher="suitor",
                 arena_bytes=0, tail_nodes=0, suitor_lanes=0, tail_block_nodes=0, sort_shared_max=0,
                 radix_bits=0, cluster_nodes=0, suitor_blocks=0) -> kp_options:
    o = kp_options_default()
    o.rating = RATINGS[rating] if isinstance(rating, str) else int(rating)
    o.seed = seed
    o.stop_size = stop_size
    o.max_levels = max_levels
    o.min_shrink_permille = min_shrink_permille
    o.spin_limit = spin_limit
    o.validate = 1 if validate else 0
    o.profile = 1 if profile else 0
    o.matcher = MATCHERS[matcher] if isinstance(matcher, str) else int(matcher)
    o.arena_bytes = arena_bytes
    o.tail_nodes = tail_nodes
    o.suitor_lanes = suitor_lanes
    o.tail_block_nodes = tail_block_nodes
    o.sort_shared_max = sort_shared_max
    o.radix_bits = radix_bits
    o.cluster_nodes = cluster_nodes
    o.suitor_blocks = suitor_blocks
    return o


class Hierarchy:
    """Owns a kp_hierarchy handle; level views are zero-copy tensors valid
    until free()."""

    def __init__(self, graph: DeviceGraph, handle: int):
        self.graph = graph            # level 0 is borrowed: keep it alive
        self.handle = handle

    def num_levels(self) -> int:
        return kp_hierarchy_num_levels(self.handle)

    def n0(self) -> int:
        return self.graph.n if self.graph is not None else kp_hierarchy_level(self.handle, 0)[0].n

    def save(self, path: str):
        """kp_hierarchy_save: every level, map and batch offset to a file."""
        kp_hierarchy_save(self.handle, path)

    def level(self, l: int):
        g, mp = kp_hierarchy_level(self.handle, l)
        out = {"n": g.n, "nnz": g.nnz, "xadj": device_view(g.xadj, g.n + 1, XADJ_TYPESTR),
               "adjncy": device_view(g.adjncy, g.nnz), "ewgt": device_view(g.ewgt, g.nnz),
               "vwgt": device_view(g.vwgt, g.n), "map": device_view(mp, g.n) if mp else None}
        out["graph"] = g
        return out

    def stats(self):
        return kp_hierarchy_stats(self.handle)

    def profile(self, level: int = -1) -> dict:
        return kp_hierarchy_profile(self.handle, level)

    def project(self, coarse_part, fine_part=None):
        torch = _torch()
        n0 = self.n0()
        if fine_part is None:
            fine_part = torch.empty(n0, dtype=torch.int32, device="cuda")
        kp_project(self.handle, coarse_part.data_ptr(), fine_part.data_ptr(), current_stream())
        return fine_part

    def free(self):
        if self.handle:
            kp_hierarchy_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def coarsen(graph: DeviceGraph, **opts) -> Hierarchy:
    h = kp_coarsen(graph.kp, make_options(**opts), current_stream())
    return Hierarchy(graph, h)


class BatchHierarchy(Hierarchy):
    """Hierarchy of a batch of independent graphs (kp_coarsen_batch)."""

    def __init__(self, graph: DeviceGraph, handle: int, offsets, seeds):
        super().__init__(graph, handle)
        self.offsets = offsets   # keep the borrowed arrays alive
        self.seeds = seeds

    def graph_levels(self):
        return kp_hierarchy_batch(self.handle)[1]

    def coarsest_sizes(self) -> np.ndarray:
        return kp_hierarchy_batch_coarsest(self.handle, self.offsets.numel() - 1, current_stream())

    def level_offsets(self, l: int):
        ng, _ = kp_hierarchy_batch(self.handle)
        return device_view(kp_hierarchy_level_offsets(self.handle, l), ng + 1)

    def graph_level(self, gi: int, l: int):
        """Graph gi at level l as host arrays with graph-local ids."""
        lv = self.level(l)
        off = self.level_offsets(l).cpu().numpy()
        a, b = int(off[gi]), int(off[gi + 1])
        X = lv["xadj"][a:b + 1].cpu().numpy().astype(np.int64)
        e0, e1 = int(X[0]), int(X[-1])
        out = {"n": b - a, "xadj": (X - e0).astype(XADJ_NP),
               "adjncy": (lv["adjncy"][e0:e1].cpu().numpy() - a).astype(np.int32),
               "ewgt": lv["ewgt"][e0:e1].cpu().numpy(), "vwgt": lv["vwgt"][a:b].cpu().numpy(), "map": None}
        levels = self.graph_levels()[gi]
        if l < levels - 1:
            nxt = self.level_offsets(l + 1).cpu().numpy()
            out["map"] = (lv["map"][a:b].cpu().numpy() - nxt[gi]).astype(np.int32)
        return out

    def project(self, coarse_part, coarse_offsets, fine_part=None):
        torch = _torch()
        if fine_part is None:
            fine_part = torch.empty(self.n0(), dtype=torch.int32, device="cuda")
        kp_project_batch(self.handle, coarse_part.data_ptr(), coarse_offsets.data_ptr(), fine_part.data_ptr(),
                         current_stream())
        return fine_part


def coarsen_batch(graph: DeviceGraph, offsets, seeds=None, stop_sizes=None, **opts) -> BatchHierarchy:
    """graph: the disjoint union (DeviceGraph); offsets: int32 node offsets
    [num_graphs+1] (array or CUDA tensor); seeds: per-graph uint64 or None;
    stop_sizes: per-graph int32 stop sizes or None (opts' stop_size for all)."""
    torch = _torch()
    off = offsets if torch.is_tensor(offsets) else torch.as_tensor(np.asarray(offsets, dtype=np.int32))
    off = off.to("cuda").contiguous()
    sd = None
    if seeds is not None:
        sd = torch.as_tensor(np.asarray(seeds, dtype=np.uint64).view(np.int64)).to("cuda").contiguous()
    ss = None
    if stop_sizes is not None:
        ss = stop_sizes if torch.is_tensor(stop_sizes) else torch.as_tensor(np.asarray(stop_sizes, dtype=np.int32))
        ss = ss.to("cuda").contiguous()
    h = kp_coarsen_batch(graph.kp, off.numel() - 1, off.data_ptr(), sd.data_ptr() if sd is not None else 0,
                         ss.data_ptr() if ss is not None else 0, make_options(**opts), current_stream())
    return BatchHierarchy(graph, h, off, (sd, ss))


def cut_gain(graph, part, k: int, eps: float, block_w=None, gain=None, target=None):
    """graph: DeviceGraph or kp_graph view; part: int32 CUDA tensor."""
    torch = _torch()
    kg = graph.kp if isinstance(graph, DeviceGraph) else graph
    n = kg.n
    block_w = torch.empty(max(k, 1), dtype=torch.int64, device="cuda") if block_w is None else block_w
    gain = torch.empty(max(n, 1), dtype=torch.int64, device="cuda") if gain is None else gain
    target = torch.empty(max(n, 1), dtype=torch.int32, device="cuda") if target is None else target
    out = kp_cut_gain_out()
    out.block_w, out.gain, out.target = block_w.data_ptr(), gain.data_ptr(), target.data_ptr()
    kp_cut_gain(kg, part.data_ptr() if n > 0 else 0, k, eps, out, current_stream())
    return {"cut": out.cut, "total_c": out.total_c, "max_c": out.max_c, "L_max": out.l_max,
            "imbalance": out.imbalance, "block_w": block_w[:k], "gain": gain[:n], "target": target[:n]}


def pipeline_host(xadj, adjncy, ewgt, vwgt, k: int, eps: float, initial_partition, outputs=None, **opts):
    """End to end from host arrays (numpy, ideally pinned): the whole path in
    one C call.  initial_partition(n_coarse, coarse_vwgt: np.ndarray, k) ->
    np.ndarray[int32] of block ids."""
    n = len(xadj) - 1
    nnz = len(adjncy)
    check_offset_width(nnz, "kp_pipeline_host")
    arrs = [host_offsets(xadj, "kp_pipeline_host")] + [np.ascontiguousarray(a, dtype=np.int32)
                                                         for a in (adjncy, ewgt, vwgt)]
    g = kp_graph(n, nnz, *[a.ctypes.data for a in arrs])
    if outputs is None:
        outputs = {"part": np.empty(n, np.int32), "gain": np.empty(n, np.int64),
                   "target": np.empty(n, np.int32), "block_w": np.empty(k, np.int64)}
    err = []

    def _ip(nc, cw_ptr, kk, part_ptr, user):
        try:
            cw = np.ctypeslib.as_array(cw_ptr, shape=(max(nc, 1),))[:nc].copy()
            p = np.asarray(initial_partition(nc, cw, kk), dtype=np.int32)
            np.ctypeslib.as_array(part_ptr, shape=(max(nc, 1),))[:nc] = p[:nc]
            return 0
        except Exception as e:   # reported through the C status
            err.append(e)
            return 1

    cb = kp_initial_partition_fn(_ip)
    out = kp_cut_gain_out()
    stream = current_stream()
    levels = kp_pipeline_host(g, make_options(**opts), k, eps, cb, None, outputs["part"].ctypes.data,
                              outputs["gain"].ctypes.data, outputs["target"].ctypes.data,
                              outputs["block_w"].ctypes.data, out, stream)
    if err:
        raise err[0]
    return {"cut": out.cut, "total_c": out.total_c, "max_c": out.max_c, "L_max": out.l_max,
            "imbalance": out.imbalance, "num_levels": levels, **outputs}


def _result_dict(res: kp_request_result) -> dict:
    return {name: getattr(res, name) for name, _ in kp_request_result._fields_}


class Server:
    """Request server of the library (kp_server_*): submit host graphs, wait,
    fetch the results, release.  Timestamps are microseconds since start."""

    def __init__(self, workers=4, max_batch=64, batch_max_nodes=1 << 16, hbm_budget_bytes=64 << 30,
                 small_workers=0, **opts):
        cfg = kp_server_config(workers, max_batch, batch_max_nodes, small_workers, hbm_budget_bytes,
                               make_options(**opts))
        self._sv = kp_server_create(cfg)
        self._borrowed = {}

    def submit(self, xadj, adjncy, ewgt, vwgt, k: int, eps: float, seed: int = 1, stop_size: int = 40,
               borrow: bool = False) -> int:
        """borrow=True: the server reads the arrays when the request runs (no
        copy at submit); they are kept referenced until release."""
        arrs = [host_offsets(xadj, "kp_server_submit")] + [np.ascontiguousarray(a, dtype=np.int32)
                                                             for a in (adjncy, ewgt, vwgt)]
        check_offset_width(len(arrs[1]), "kp_server_submit")
        g = kp_graph(len(arrs[0]) - 1, len(arrs[1]), *[a.ctypes.data for a in arrs])
        rid = kp_server_submit(self._sv, g, kp_request_params(k, stop_size, eps, seed,
                                                              KP_REQUEST_BORROW if borrow else 0, 0))
        if borrow:
            self._borrowed[rid] = arrs
        return rid

    def poll(self, rid: int):
        done, res = kp_server_poll(self._sv, rid)
        return done, _result_dict(res)

    def wait(self, rid: int) -> dict:
        return _result_dict(kp_server_wait(self._sv, rid))

    def fetch(self, rid: int, n: int, coarsest_n: int) -> dict:
        out = {"part": np.empty(max(n, 1), np.int32), "gain": np.empty(max(n, 1), np.int64),
               "target": np.empty(max(n, 1), np.int32), "coarse_part": np.empty(max(coarsest_n, 1), np.int32)}
        kp_server_fetch(self._sv, rid, out["part"].ctypes.data, out["gain"].ctypes.data,
                        out["target"].ctypes.data, out["coarse_part"].ctypes.data)
        return {"part": out["part"][:n], "gain": out["gain"][:n], "target": out["target"][:n],
                "coarse_part": out["coarse_part"][:coarsest_n]}

    def release(self, rid: int):
        kp_server_release(self._sv, rid)
        self._borrowed.pop(rid, None)

    def cancel(self, rid: int):
        kp_server_cancel(self._sv, rid)
        self._borrowed.pop(rid, None)

    def close(self):
        if self._sv:
            kp_server_destroy(self._sv)
            self._sv = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _knobs(o: kp_options) -> dict:
    return {k: int(getattr(o, k)) for k in TUNING_KNOBS}


def shape_key(graph, num_graphs: int = 0, rating="expansion*2", matcher="suitor") -> str:
    """Shape class of a tuning problem: powers of two of the node count and
    of the mean degree, the batch size class, rating and matcher."""
    import math
    n, nnz = max(graph.kp.n, 1), graph.kp.nnz
    return (f"n2^{round(math.log2(n))}|deg2^{round(math.log2(max(nnz / n, 1.0)))}|"
            f"graphs2^{round(math.log2(num_graphs)) if num_graphs > 0 else 'single'}|{rating}|{matcher}")


def autotune(graph: DeviceGraph, offsets=None, seeds=None, stop_sizes=None, reps: int = 2, cache: str | None = None,
             max_trials: int = 64, **opts):
    """Tuning knobs for this graph (or batch when offsets is given) by
    kp_autotune, cached in the JSON file `cache` under the GPU's name and the
    shape class.  Returns (knobs dict, trials [(knobs, ms)], from_cache)."""
    import json
    torch = _torch()
    key = f"{torch.cuda.get_device_name()}|" + shape_key(graph, 0 if offsets is None else len(offsets) - 1,
                                                            opts.get("rating", "expansion*2"),
                                                            opts.get("matcher", "suitor"))
    table = {}
    if cache and os.path.exists(cache):
        with open(cache) as f:
            table = json.load(f)
        if key in table:
            return table[key]["knobs"], [], True
    off = sd = ss = None
    if offsets is not None:
        off = offsets if torch.is_tensor(offsets) else torch.as_tensor(np.asarray(offsets, dtype=np.int32))
        off = off.to("cuda").contiguous()
        if seeds is not None:
            sd = torch.as_tensor(np.asarray(seeds, dtype=np.uint64).view(np.int64)).to("cuda").contiguous()
        if stop_sizes is not None:
            ss = torch.as_tensor(np.asarray(stop_sizes, dtype=np.int32)).to("cuda").contiguous()
    best, trials = kp_autotune(graph.kp, 0 if off is None else off.numel() - 1, 0 if off is None else off.data_ptr(),
                               0 if sd is None else sd.data_ptr(), 0 if ss is None else ss.data_ptr(),
                               make_options(**opts), reps, max_trials, current_stream())
    knobs = _knobs(best)
    if cache:
        table[key] = {"knobs": knobs, "best_ms": min(t.ms for t in trials) if trials else None}
        d = os.path.dirname(os.path.abspath(cache))
        os.makedirs(d, exist_ok=True)
        tmp = cache + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(table, f, indent=1, sort_keys=True)
        os.replace(tmp, cache)
    return knobs, [(_knobs(t.options), t.ms) for t in trials], False


class Plan:
    """A coarsening recorded once into a CUDA graph (kp_plan_*): one graph,
    or a batch when offsets is given.  run() replays it and returns a
    Hierarchy (BatchHierarchy for a batch) valid until the next run."""

    def __init__(self, graph: DeviceGraph, offsets=None, seeds=None, stop_sizes=None, **opts):
        torch = _torch()
        self.graph = graph
        self.off = self.sd = self.ss = None
        if offsets is not None:
            off = offsets if torch.is_tensor(offsets) else torch.as_tensor(np.asarray(offsets, dtype=np.int32))
            self.off = off.to("cuda").contiguous()
            if seeds is not None:
                self.sd = torch.as_tensor(np.asarray(seeds, dtype=np.uint64).view(np.int64)).to("cuda").contiguous()
            if stop_sizes is not None:
                self.ss = torch.as_tensor(np.asarray(stop_sizes, dtype=np.int32)).to("cuda").contiguous()
        G = 0 if self.off is None else self.off.numel() - 1
        self.handle = kp_plan_create(graph.kp, G, 0 if self.off is None else self.off.data_ptr(),
                                     0 if self.sd is None else self.sd.data_ptr(),
                                     0 if self.ss is None else self.ss.data_ptr(), make_options(**opts),
                                     current_stream())
        self._last = None

    def run(self):
        if self._last is not None:
            self._last.free()
        h = kp_plan_run(self.handle, current_stream())
        self._last = (BatchHierarchy(self.graph, h, self.off, (self.sd, self.ss)) if self.off is not None
                      else Hierarchy(self.graph, h))
        return self._last

    def close(self):
        if self._last is not None:
            self._last.free()
            self._last = None
        if self.handle:
            kp_plan_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def quotient_graph(graph, part, k: int):
    """Quotient graph of a partition (kp_quotient_graph): (q_xadj, q_adjncy,
    q_ewgt) CUDA tensors; buffers grow once if the first guess is small."""
    torch = _torch()
    kg = graph.kp if isinstance(graph, DeviceGraph) else graph
    q_xadj = torch.empty(k + 1, dtype=torch.int32, device="cuda")
    cap = max(16, min(k * (k - 1), 8 * k))
    for _ in range(2):
        q_adj = torch.empty(cap, dtype=torch.int32, device="cuda")
        q_w = torch.empty(cap, dtype=torch.int64, device="cuda")
        got = kp_quotient_graph(kg, part.data_ptr() if kg.n > 0 else 0, k, q_xadj.data_ptr(), q_adj.data_ptr(),
                                q_w.data_ptr(), cap, current_stream())
        if got >= 0:
            return q_xadj, q_adj[:got], q_w[:got]
        cap = -got - 1
    raise RuntimeError("quotient graph did not fit twice")


def boundary_band(graph, part, k: int, depth: int, pair=None, dist=None):
    """Bounded breadth-first search from the block boundaries
    (kp_boundary_band); returns dist (int32 CUDA tensor)."""
    torch = _torch()
    kg = graph.kp if isinstance(graph, DeviceGraph) else graph
    if dist is None:
        dist = torch.empty(max(kg.n, 1), dtype=torch.int32, device="cuda")
    a, b = pair if pair is not None else (-1, -1)
    kp_boundary_band(kg, part.data_ptr() if kg.n > 0 else 0, k, depth, a, b, dist.data_ptr(), current_stream())
    return dist[:kg.n]


def load_hierarchy(path: str):
    """kp_hierarchy_load: a saved hierarchy back on the device (it owns every
    level).  Returns a Hierarchy, or a BatchHierarchy for a batch."""
    h = kp_hierarchy_load(path, current_stream())
    G, _ = kp_hierarchy_batch(h)
    if G == 0:
        return Hierarchy(None, h)
    off = device_view(kp_hierarchy_level_offsets(h, 0), G + 1).clone()
    return BatchHierarchy(None, h, off, None)
