"""Oracle for the coarsening / projection / cut-gain path (TEST INFRASTRUCTURE).

A plain sequential CPU statement of what the partitioner's data-parallel path
computes, written from the paper ("Engineering a Scalable High Quality Graph
Partitioner", Sections 2, 3.1-3.3, 4, 5.2).  Only the tests, the smoke check
and the benchmark's CPU-baseline leg may import it; the product path never
does.  It shares no code with the CUDA library: the heavy loops are in
oracle.c (compiled here with gcc), the level loop, the stop rule, projection
and the balance bound are plain Python/numpy below.

Each function names the passage it follows.  All arithmetic is integer.
The refinement-side helpers at the end (quotient graph, bounded boundary
search, Section 5) are plain Python/numpy.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "RATINGS", "Level", "Hierarchy", "build", "lib", "validate", "out_weight",
    "frac_cmp", "splitmix64", "edge_hash", "edge_order", "greedy_matching",
    "handshake_matching", "gpa_matching", "check_greedy_matching", "contract", "coarsen",
    "project", "l_max", "cut_gain", "quotient_graph", "boundary_band",
]

RATINGS = {"expansion*2": 0, "innerOuter": 1, "weight": 2, "expansion": 3, "expansion*": 4}

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile oracle.c into a shared library (gcc, portable flags)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-Wall", "-shared", "-fPIC",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            i32, i64, u64, c_int = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_int
            L.or_validate.argtypes = [i32, i64, i64, _i64p, _i32p, _i32p, _i32p]
            L.or_validate.restype = c_int
            L.or_out_weight.argtypes = [i32, _i64p, _i32p, _i64p]
            L.or_out_weight.restype = None
            L.or_frac_cmp.argtypes = [u64, u64, u64, u64]
            L.or_frac_cmp.restype = c_int
            L.or_splitmix64.argtypes = [u64]
            L.or_splitmix64.restype = u64
            L.or_edge_hash.argtypes = [u64, i32, i32]
            L.or_edge_hash.restype = u64
            L.or_edge_order.argtypes = [c_int, u64, _i32p, _i64p, i32, i32, i32, i32, i32, i32]
            L.or_edge_order.restype = c_int
            L.or_greedy_matching.argtypes = [i32, _i64p, _i32p, _i32p, _i32p, c_int, u64, _i32p]
            L.or_greedy_matching.restype = i64
            L.or_handshake_matching.argtypes = [i32, _i64p, _i32p, _i32p, _i32p, c_int, u64, _i32p,
                                                ctypes.POINTER(i32), _i32p]
            L.or_handshake_matching.restype = i64
            L.or_gpa_matching.argtypes = [i32, _i64p, _i32p, _i32p, _i32p, c_int, u64, _i32p, _i32p]
            L.or_gpa_matching.restype = i64
            L.or_check_greedy_matching.argtypes = [i32, _i64p, _i32p, _i32p, _i32p, c_int, u64, _i32p]
            L.or_check_greedy_matching.restype = i64
            L.or_check_greedy_matching_at.argtypes = [i32, _i64p, _i32p, _i32p, _i32p, c_int, u64, _i32p,
                                                      i64, _i32p]
            L.or_check_greedy_matching_at.restype = i64
            L.or_coarse_row.argtypes = [_i64p, _i32p, _i32p, _i32p, _i32p, i32, i32, i32,
                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(i64)]
            L.or_coarse_row.restype = i32
            L.or_contract.argtypes = [i32, _i64p, _i32p, _i32p, _i32p, _i32p, _i32p,
                                      ctypes.POINTER(i64), _i64p, _i32p, _i32p, _i32p]
            L.or_contract.restype = i32
            L.or_project_level.argtypes = [i32, _i32p, _i32p, _i32p]
            L.or_project_level.restype = None
            L.or_cut_gain.argtypes = [i32, _i64p, _i32p, _i32p, _i32p, _i32p, i32,
                                      ctypes.POINTER(i64), _i64p, _i64p, _i32p]
            L.or_cut_gain.restype = c_int
            _lib = L
    return _lib


@dataclass
class Level:
    """One graph of the hierarchy as a symmetric sorted CSR (Section 5.2);
    row offsets int64 (graphs of 2^31 entries or more fit)."""
    xadj: np.ndarray
    adjncy: np.ndarray
    ewgt: np.ndarray
    vwgt: np.ndarray

    @property
    def n(self) -> int:
        return int(self.xadj.shape[0] - 1)

    @property
    def nnz(self) -> int:
        return int(self.adjncy.shape[0])


@dataclass
class Hierarchy:
    levels: list = field(default_factory=list)     # Level 0 (input) .. Level L (coarsest)
    maps: list = field(default_factory=list)       # maps[l]: node of level l -> node of level l+1
    matched: list = field(default_factory=list)    # |M_l| per contraction


def _as_level(g) -> Level:
    c = np.ascontiguousarray
    return Level(c(g.xadj, dtype=np.int64), c(g.adjncy, dtype=np.int32),
                 c(g.ewgt, dtype=np.int32), c(g.vwgt, dtype=np.int32))


def validate(g, nnz_limit: int = 1 << 31) -> int:
    """0 = valid, 1 = invalid (malformed/asymmetric/unsorted CSR, self loop,
    omega <= 0, c < 0: Section 2), 2 = outside the integer ranges (nnz must
    stay below nnz_limit: 2^31 with 32-bit offsets, 2^32 with 64-bit ones)."""
    g = _as_level(g)
    return lib().or_validate(g.n, g.nnz, nnz_limit, g.xadj, g.adjncy, g.ewgt, g.vwgt)


def out_weight(g) -> np.ndarray:
    """Out(v) (Section 3.1)."""
    g = _as_level(g)
    out = np.zeros(g.n, dtype=np.int64)
    lib().or_out_weight(g.n, g.xadj, g.ewgt, out)
    return out


def frac_cmp(a: int, b: int, c: int, d: int) -> int:
    return lib().or_frac_cmp(a, b, c, d)


def splitmix64(x: int) -> int:
    return lib().or_splitmix64(x)


def edge_hash(seed: int, u: int, v: int) -> int:
    return lib().or_edge_hash(seed, u, v)


def edge_order(rating: str, seed: int, vwgt, out, e1, e2) -> int:
    """+1 if edge e1=(u,v,w) comes before e2 in the strict order, -1 after, 0 same."""
    vw = np.ascontiguousarray(vwgt, dtype=np.int32)
    o = np.ascontiguousarray(out if out is not None else np.zeros(len(vw)), dtype=np.int64)
    return lib().or_edge_order(RATINGS[rating], seed, vw, o, *e1, *e2)


def greedy_matching(g, rating: str, seed: int):
    """Greedy matching (Section 3.2) under the strict edge order."""
    g = _as_level(g)
    match = np.empty(g.n, dtype=np.int32)
    size = lib().or_greedy_matching(g.n, g.xadj, g.adjncy, g.ewgt, g.vwgt, RATINGS[rating], seed, match)
    if size < 0:
        raise MemoryError("oracle greedy matching")
    return match, int(size)


def handshake_matching(g, rating: str, seed: int):
    """Round-by-round locally-heaviest matching (Section 3.3).
    Returns (match, |M|, rounds, first-round candidates)."""
    g = _as_level(g)
    match = np.empty(g.n, dtype=np.int32)
    cand1 = np.empty(g.n, dtype=np.int32)
    rounds = ctypes.c_int32(0)
    size = lib().or_handshake_matching(g.n, g.xadj, g.adjncy, g.ewgt, g.vwgt, RATINGS[rating], seed,
                                       match, ctypes.byref(rounds), cand1)
    if size < 0:
        raise MemoryError("oracle handshake matching")
    return match, int(size), int(rounds.value), cand1


def gpa_matching(g, rating: str, seed: int):
    """Global Path Algorithm (Section 3.2): paths and even cycles collected
    in the strict edge order, then an optimal matching of each by dynamic
    programming over the ratings in double precision (see oracle.c).
    Returns (match, |M|, nbr2) with nbr2[2v], nbr2[2v+1] the collected
    neighbours of v (-1 where fewer)."""
    g = _as_level(g)
    match = np.empty(g.n, dtype=np.int32)
    nbr2 = np.empty(max(2 * g.n, 1), dtype=np.int32)
    size = lib().or_gpa_matching(g.n, g.xadj, g.adjncy, g.ewgt, g.vwgt, RATINGS[rating], seed, match, nbr2)
    if size < 0:
        raise MemoryError("oracle GPA matching")
    return match, int(size), nbr2[:2 * g.n]


def check_greedy_matching(g, rating: str, seed: int, match) -> int:
    """-1 iff `match` is the Greedy matching of g (see oracle.c)."""
    g = _as_level(g)
    m = np.ascontiguousarray(match, dtype=np.int32)
    return int(lib().or_check_greedy_matching(g.n, g.xadj, g.adjncy, g.ewgt, g.vwgt,
                                              RATINGS[rating], seed, m))


def check_greedy_matching_at(g, rating: str, seed: int, match, nodes) -> int:
    """check_greedy_matching restricted to the listed nodes (large graphs):
    -1 iff every listed node passes."""
    g = _as_level(g)
    m = np.ascontiguousarray(match, dtype=np.int32)
    nd = np.ascontiguousarray(nodes, dtype=np.int32)
    return int(lib().or_check_greedy_matching_at(g.n, g.xadj, g.adjncy, g.ewgt, g.vwgt, RATINGS[rating], seed, m,
                                                 nd.shape[0], nd))


def coarse_rows(g, mp, rows):
    """Rows of the coarse nodes x with members a, b (b = -1: one member)
    under the map mp (Section 2), for rows = [(x, a, b), ...]: a list of
    (neighbours, weights, c)."""
    g = _as_level(g)
    mp = np.ascontiguousarray(mp, dtype=np.int32)
    res = []
    for x, a, b in rows:
        a, b = int(a), int(b)
        cap = int(g.xadj[a + 1] - g.xadj[a]) + (int(g.xadj[b + 1] - g.xadj[b]) if b >= 0 else 0)
        adj = np.empty(max(cap, 1), dtype=np.int32)
        w = np.empty(max(cap, 1), dtype=np.int32)
        c = ctypes.c_int64(0)
        k = lib().or_coarse_row(g.xadj, g.adjncy, g.ewgt, g.vwgt, mp, int(x), a, b, adj.ctypes.data,
                                w.ctypes.data, ctypes.byref(c))
        if k < 0:
            raise MemoryError("oracle coarse row")
        res.append((adj[:k], w[:k], int(c.value)))
    return res


def contract(g, match):
    """Contract all matched edges (Section 2).  Returns (coarse Level, map)."""
    g = _as_level(g)
    match = np.ascontiguousarray(match, dtype=np.int32)
    n = g.n
    mp = np.empty(n, dtype=np.int32)
    cxadj = np.empty(n + 1, dtype=np.int64)
    cadj = np.empty(max(g.nnz, 1), dtype=np.int32)
    cew = np.empty(max(g.nnz, 1), dtype=np.int32)
    cvw = np.empty(max(n, 1), dtype=np.int32)
    cnnz = ctypes.c_int64(0)
    cn = lib().or_contract(n, g.xadj, g.adjncy, g.ewgt, g.vwgt, match, mp, ctypes.byref(cnnz),
                           cxadj, cadj, cew, cvw)
    if cn < 0:
        raise MemoryError("oracle contraction")
    k = int(cnnz.value)
    # views of the first cn / k elements (no second copy of large levels)
    return Level(cxadj[:cn + 1], cadj[:k], cew[:k], cvw[:cn]), mp


def coarsen(g, rating: str, seed: int, stop_size: int, max_levels: int = 64,
            min_shrink_permille: int = 50, matcher: str = "greedy") -> Hierarchy:
    """The contraction phase (Section 2, multilevel scheme; Section 3).

    Level after level: compute the matching, contract it.  Stop before a level
    once the graph has at most `stop_size` nodes (Section 4 stops "when the
    graph is small enough"; the threshold is a parameter), or once
    `max_levels` contractions were made.  Stop after a contraction that
    matched nothing (that level is not kept) or that kept more than
    (1000 - min_shrink_permille)/1000 of the nodes (that level is kept)."""
    h = Hierarchy(levels=[_as_level(g)])
    while True:
        cur = h.levels[-1]
        if cur.n <= stop_size or len(h.maps) >= max_levels:
            break
        if matcher == "greedy":
            match, size = greedy_matching(cur, rating, seed)
        elif matcher == "gpa":
            match, size, _ = gpa_matching(cur, rating, seed)
        else:
            match, size, _, _ = handshake_matching(cur, rating, seed)
        if size == 0:
            break
        coarse, mp = contract(cur, match)
        h.levels.append(coarse)
        h.maps.append(mp)
        h.matched.append(size)
        if coarse.n * 1000 > cur.n * (1000 - min_shrink_permille):
            break
    return h


def project(maps, coarse_part) -> np.ndarray:
    """Uncontraction of the whole hierarchy (Section 2): a fine node takes the
    block of the coarse node it was contracted into, from the coarsest level
    down to the input graph."""
    part = np.ascontiguousarray(coarse_part, dtype=np.int32)
    for mp in reversed(maps):
        mp = np.ascontiguousarray(mp, dtype=np.int32)
        fine = np.empty(mp.shape[0], dtype=np.int32)
        lib().or_project_level(mp.shape[0], mp, part, fine)
        part = fine
    return part


def l_max(total_c: int, max_c: int, k: int, eps: float) -> int:
    """Balance bound L_max = (1+eps) c(V)/k + max_v c(v) (Section 2), with eps
    read in parts per million (rounded half up) and the result rounded down so
    that the integer test c(V_i) <= L_max is exact."""
    x = eps * 1_000_000          # the same double product as the C library's
    eps_ppm = math.floor(x) + (1 if x - math.floor(x) >= 0.5 else 0)   # round half up
    return ((1_000_000 + eps_ppm) * int(total_c) + k * 1_000_000 * int(max_c)) // (k * 1_000_000)


def cut_gain(g, part, k: int, eps: float) -> dict:
    """Cut (Section 2), block weights, L_max, imbalance (Section 5.2:
    max(0, max_i c(V_i) - L_max)) and per-node FM gains (Section 5.2)."""
    g = _as_level(g)
    part = np.ascontiguousarray(part, dtype=np.int32)
    cut = ctypes.c_int64(0)
    bw = np.zeros(max(k, 1), dtype=np.int64)
    gain = np.empty(g.n, dtype=np.int64)
    target = np.empty(g.n, dtype=np.int32)
    st = lib().or_cut_gain(g.n, g.xadj, g.adjncy, g.ewgt, g.vwgt, part, k, ctypes.byref(cut), bw, gain, target)
    if st != 0:
        raise ValueError(f"oracle cut_gain status {st}")
    total_c = int(g.vwgt.astype(np.int64).sum())
    max_c = int(g.vwgt.max()) if g.n else 0
    lm = l_max(total_c, max_c, k, eps)
    imb = max(0, int(bw[:k].max()) - lm) if k else 0
    return {"cut": int(cut.value), "block_w": bw[:k], "L_max": lm, "imbalance": imb,
            "gain": gain, "target": target}


def quotient_graph(g, part, k: int):
    """Quotient graph Q (Section 5): one node per block, an edge {a, b}
    whenever an edge of G joins blocks a and b, weighted by the total edge
    weight between them.  Returned as a symmetric CSR over the k blocks with
    ascending neighbour blocks: (xadj int32[k+1], adjncy int32[], ewgt
    int64[])."""
    g = _as_level(g)
    part = np.asarray(part, dtype=np.int64)
    acc = {}
    for u in range(g.n):
        pu = int(part[u])
        for e in range(int(g.xadj[u]), int(g.xadj[u + 1])):
            pv = int(part[int(g.adjncy[e])])
            if pv != pu:
                acc[(pu, pv)] = acc.get((pu, pv), 0) + int(g.ewgt[e])
    xadj = np.zeros(k + 1, dtype=np.int32)
    adj, w = [], []
    for a in range(k):
        row = sorted((b, c) for (aa, b), c in acc.items() if aa == a)
        for b, c in row:
            adj.append(b)
            w.append(c)
        xadj[a + 1] = len(adj)
    return xadj, np.asarray(adj, dtype=np.int32), np.asarray(w, dtype=np.int64)


def boundary_band(g, part, depth: int, pair=None) -> np.ndarray:
    """Bounded breadth-first search from the block boundaries (Section 5):
    dist[v] = length of a shortest path from v to a boundary node of its own
    block through nodes of that block, if at most `depth`, else -1.  A
    boundary node has a neighbour in another block.  With pair = (a, b) only
    blocks a and b take part: the boundary is the a-b boundary and nodes of
    other blocks get -2."""
    g = _as_level(g)
    part = np.asarray(part, dtype=np.int64)
    n = g.n
    dist = np.full(n, -1, dtype=np.int32)
    inside = np.ones(n, dtype=bool)
    if pair is not None:
        a, b = pair
        inside = (part == a) | (part == b)
        dist[~inside] = -2
    frontier = []
    for v in range(n):
        if not inside[v]:
            continue
        pv = int(part[v])
        for e in range(int(g.xadj[v]), int(g.xadj[v + 1])):
            pu = int(part[int(g.adjncy[e])])
            other = (pu != pv) if pair is None else (pu == (pair[1] if pv == pair[0] else pair[0]))
            if other and pu != pv:
                dist[v] = 0
                frontier.append(v)
                break
    for d in range(1, depth + 1):
        nxt = []
        for u in frontier:
            for e in range(int(g.xadj[u]), int(g.xadj[u + 1])):
                v = int(g.adjncy[e])
                if dist[v] == -1 and part[v] == part[u]:
                    dist[v] = d
                    nxt.append(v)
        frontier = nxt
    return dist
