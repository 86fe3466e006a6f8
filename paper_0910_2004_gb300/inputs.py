"""Seeded synthetic input generators (graphs and coarse partitions).

This module produces INPUTS only: CSR graphs with the shapes and weight
distributions of the workloads the partitioner is measured on, and the seeded
random coarse partition that stands in for initial partitioning.  It holds none
of the method's arithmetic (no rating, matching, contraction, cut or gain), so
both the CUDA path and the CPU oracle may consume what it returns.

Graph layout (shared by every consumer): an undirected graph is stored as a
symmetric CSR with int32 arrays
    xadj   [n+1]   row offsets
    adjncy [nnz]   neighbour ids, strictly increasing inside each row
    ewgt   [nnz]   edge weights (>0), equal for (u,v) and (v,u)
    vwgt   [n]     node weights (>=0)
nnz = 2m counts directed entries (Section 2: G=(V,E,c,omega), Section 5.2:
static adjacency array).

Random numbers come from numpy's PCG64 generator, whose bit stream is
platform independent, so the same seed gives the same graph on x86 and Arm.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

__all__ = [
    "CSRGraph", "from_edges", "grid2d", "grid3d", "rgg2d", "rmat",
    "random_small_graph", "path_graph", "star_graph", "batch_rgg_sizes",
    "random_balanced_partition", "random_partition", "union_graph", "rgg2d_batch", "batch_partition",
    "rmat_torch", "rgg2d_torch", "served_mix", "batch_partition_torch", "circulant_strides", "circulant",
    "circulant_torch",
]


@dataclass
class CSRGraph:
    xadj: np.ndarray
    adjncy: np.ndarray
    ewgt: np.ndarray
    vwgt: np.ndarray
    name: str = ""

    @property
    def n(self) -> int:
        return int(self.xadj.shape[0] - 1)

    @property
    def nnz(self) -> int:
        return int(self.adjncy.shape[0])

    @property
    def m(self) -> int:
        return self.nnz // 2

    def arrays(self):
        return self.xadj, self.adjncy, self.ewgt, self.vwgt

    def __post_init__(self):
        # a row offset that wrapped in a narrowing cast shows here
        if self.xadj.shape[0] and int(self.xadj[-1]) != self.adjncy.shape[0]:
            raise ValueError(f"{self.name}: xadj[n] = {int(self.xadj[-1])} but {self.adjncy.shape[0]} entries")


def from_edges(n: int, lo: np.ndarray, hi: np.ndarray, w: np.ndarray | None = None,
               vwgt: np.ndarray | None = None, name: str = "") -> CSRGraph:
    """Symmetric sorted CSR from an undirected edge list.

    (lo, hi) must be unique pairs with lo != hi (either orientation is fine).
    """
    lo = np.asarray(lo, dtype=np.int64)
    hi = np.asarray(hi, dtype=np.int64)
    if w is None:
        w = np.ones(lo.shape[0], dtype=np.int64)
    w = np.asarray(w, dtype=np.int64)
    src = np.concatenate([lo, hi])
    dst = np.concatenate([hi, lo])
    ww = np.concatenate([w, w])
    order = np.lexsort((dst, src))
    src, dst, ww = src[order], dst[order], ww[order]
    counts = np.bincount(src, minlength=n).astype(np.int64)
    xadj = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=xadj[1:])
    if vwgt is None:
        vwgt = np.ones(n, dtype=np.int32)
    return CSRGraph(xadj.astype(np.int32), dst.astype(np.int32), ww.astype(np.int32),
                    np.asarray(vwgt, dtype=np.int32), name)


def grid2d(nx: int, ny: int) -> CSRGraph:
    """5-point grid, id = x + nx*y, unit node and edge weights."""
    ids = np.arange(nx * ny, dtype=np.int64).reshape(ny, nx)
    lo = [ids[:, :-1].ravel(), ids[:-1, :].ravel()]
    hi = [ids[:, 1:].ravel(), ids[1:, :].ravel()]
    return from_edges(nx * ny, np.concatenate(lo), np.concatenate(hi),
                      name=f"grid2d_{nx}x{ny}")


def grid3d(nx: int, ny: int, nz: int) -> CSRGraph:
    """7-point grid, id = x + nx*(y + ny*z) (x fastest), unit weights.

    Built row by row in sorted order directly (no global sort), so the
    256^3 case (16.8M nodes, 100M directed entries) takes seconds.
    """
    n = nx * ny * nz
    v = np.arange(n, dtype=np.int64)
    x = v % nx
    y = (v // nx) % ny
    z = v // (nx * ny)
    # neighbour offsets in increasing id order: -nx*ny, -nx, -1, +1, +nx, +nx*ny
    offs = [(-nx * ny, z > 0), (-nx, y > 0), (-1, x > 0),
            (1, x < nx - 1), (nx, y < ny - 1), (nx * ny, z < nz - 1)]
    deg = np.zeros(n, dtype=np.int64)
    for _, ok in offs:
        deg += ok
    xadj = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(deg, out=xadj[1:])
    nnz = int(xadj[-1])
    adjncy = np.empty(nnz, dtype=np.int32)
    pos = xadj[:-1].copy()
    for off, ok in offs:
        idx = np.nonzero(ok)[0]
        adjncy[pos[idx]] = (idx + off).astype(np.int32)
        pos[idx] += 1
        del idx
    return CSRGraph(xadj.astype(np.int32), adjncy, np.ones(nnz, dtype=np.int32),
                    np.ones(n, dtype=np.int32), f"grid3d_{nx}x{ny}x{nz}")


def rgg2d(n: int, seed: int, mean_degree: float = 6.0, radius: float | None = None,
          wmax: int = 1) -> CSRGraph:
    """2D random geometric graph: n points uniform in [0,1)^2, edge iff the
    Euclidean distance is below r (Section 6, instances).  Default r gives
    expected mean degree `mean_degree` (pi r^2 n = mean_degree); ids follow
    generation order.  Edge weights are uniform in [1, wmax] (1 = unit)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    pts = rng.random((n, 2))
    if radius is None:
        radius = math.sqrt(mean_degree / (math.pi * n))
    r2 = radius * radius
    G = max(1, int(1.0 / radius))
    cx = np.minimum((pts[:, 0] * G).astype(np.int64), G - 1)
    cy = np.minimum((pts[:, 1] * G).astype(np.int64), G - 1)
    cell = cx + G * cy
    order = np.argsort(cell, kind="stable")
    cell_sorted = cell[order]
    start = np.searchsorted(cell_sorted, np.arange(G * G), side="left")
    count = np.searchsorted(cell_sorted, np.arange(G * G), side="right") - start
    maxc = int(count.max()) if n else 0
    los, his = [], []
    pid = np.arange(n, dtype=np.int64)
    for dx in (-1, 0, 1):
        for dy in (-1, 0, 1):
            ncx, ncy = cx + dx, cy + dy
            ok = (ncx >= 0) & (ncx < G) & (ncy >= 0) & (ncy < G)
            src = pid[ok]
            ncell = (ncx + G * ncy)[ok]
            s0, c0 = start[ncell], count[ncell]
            for j in range(maxc):
                has = c0 > j
                if not has.any():
                    break
                a = src[has]
                b = order[s0[has] + j]
                keep = a < b
                a, b = a[keep], b[keep]
                d = pts[a] - pts[b]
                close = (d * d).sum(axis=1) < r2
                los.append(a[close])
                his.append(b[close])
    lo = np.concatenate(los) if los else np.zeros(0, np.int64)
    hi = np.concatenate(his) if his else np.zeros(0, np.int64)
    if wmax > 1:
        w = rng.integers(1, wmax + 1, size=lo.shape[0])
    else:
        w = None
    return from_edges(n, lo, hi, w, name=f"rgg2d_n{n}_s{seed}")


def rmat(scale: int, seed: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19,
         c: float = 0.19) -> CSRGraph:
    """R-MAT graph (Chakrabarti et al. 2004): edge_factor * 2^scale samples,
    symmetrised, self loops dropped, duplicates merged into integer weights."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = 1 << scale
    M = edge_factor * n
    u = np.zeros(M, dtype=np.int64)
    v = np.zeros(M, dtype=np.int64)
    for bit in range(scale):
        r = rng.random(M)
        ubit = r >= a + b            # quadrants c, d -> lower half in u
        vbit = ((r >= a) & (r < a + b)) | (r >= a + b + c)
        u |= ubit.astype(np.int64) << bit
        v |= vbit.astype(np.int64) << bit
    keep = u != v
    u, v = u[keep], v[keep]
    lo, hi = np.minimum(u, v), np.maximum(u, v)
    key, cnt = np.unique(lo * n + hi, return_counts=True)
    return from_edges(n, key // n, key % n, cnt, name=f"rmat_s{scale}_seed{seed}")


def random_small_graph(n: int, p: float, seed: int, wmax: int = 4, cmax: int = 3,
                       allow_zero_c: bool = False) -> CSRGraph:
    """Erdos-Renyi G(n,p) with random integer edge weights in [1,wmax] and node
    weights in [1,cmax] (or [0,cmax])."""
    rng = np.random.Generator(np.random.PCG64(seed))
    iu, ju = np.triu_indices(n, 1)
    keep = rng.random(iu.shape[0]) < p
    lo, hi = iu[keep], ju[keep]
    w = rng.integers(1, wmax + 1, size=lo.shape[0])
    c = rng.integers(0 if allow_zero_c else 1, cmax + 1, size=n)
    return from_edges(n, lo, hi, w, c, name=f"gnp_n{n}_p{p}_s{seed}")


def path_graph(n: int, increasing: bool = True) -> CSRGraph:
    """Path 0-1-...-(n-1); edge (i,i+1) has weight i+1 (increasing) or 1."""
    lo = np.arange(n - 1)
    w = lo + 1 if increasing else np.ones(n - 1, dtype=np.int64)
    return from_edges(n, lo, lo + 1, w, name=f"path_{n}")


def star_graph(leaves: int) -> CSRGraph:
    """Hub 0 joined to leaves 1..leaves, unit weights."""
    return from_edges(leaves + 1, np.zeros(leaves, np.int64), np.arange(1, leaves + 1),
                      name=f"star_{leaves}")


def batch_rgg_sizes(count: int, seed: int, nmin: int = 1024, nmax: int = 65536) -> np.ndarray:
    """Node counts log-uniform in [nmin, nmax] for a batch of independent RGGs."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.floor(np.exp(rng.uniform(math.log(nmin), math.log(nmax), size=count))).astype(np.int64)


def union_graph(graphs) -> tuple:
    """Disjoint union of graphs in order: graph i's node v becomes node
    offsets[i] + v.  Returns (CSRGraph, offsets int32[len(graphs)+1])."""
    ns = np.array([g.n for g in graphs], dtype=np.int64)
    offsets = np.zeros(len(graphs) + 1, dtype=np.int64)
    np.cumsum(ns, out=offsets[1:])
    nnzs = np.array([g.nnz for g in graphs], dtype=np.int64)
    eoff = np.zeros(len(graphs) + 1, dtype=np.int64)
    np.cumsum(nnzs, out=eoff[1:])
    xadj = np.zeros(int(offsets[-1]) + 1, dtype=np.int64)
    adj = np.empty(int(eoff[-1]), dtype=np.int32)
    ew = np.empty(int(eoff[-1]), dtype=np.int32)
    vw = np.empty(int(offsets[-1]), dtype=np.int32)
    for i, g in enumerate(graphs):
        o, e = int(offsets[i]), int(eoff[i])
        xadj[o:o + g.n + 1] = g.xadj.astype(np.int64) + e
        adj[e:e + g.nnz] = g.adjncy + o
        ew[e:e + g.nnz] = g.ewgt
        vw[o:o + g.n] = g.vwgt
    return CSRGraph(xadj.astype(np.int32), adj, ew, vw, f"union_{len(graphs)}"), offsets.astype(np.int32)


def rgg2d_batch(sizes, seed: int, mean_degree: float = 6.0, wmax: int = 16, device: str = "cuda"):
    """Disjoint union of independent 2D random geometric graphs, built with
    torch on `device` (fast at tens of millions of nodes).  Graph i has
    sizes[i] points uniform in [0,1)^2 in generation order, an edge joins
    points closer than sqrt(mean_degree / (pi n_i)), and integer edge weights
    are uniform in [1, wmax].  Returns int32 tensors (xadj, adjncy, ewgt,
    vwgt, offsets); graph i owns nodes [offsets[i], offsets[i+1])."""
    import torch
    dev = torch.device(device)
    gen = torch.Generator(device=dev)
    gen.manual_seed(seed)
    sz = torch.as_tensor(np.asarray(sizes, dtype=np.int64), device=dev)
    G = int(sz.numel())
    P = int(sz.sum().item())
    offsets = torch.zeros(G + 1, dtype=torch.int64, device=dev)
    offsets[1:] = torch.cumsum(sz, 0)
    gid = torch.repeat_interleave(torch.arange(G, device=dev), sz)
    pts = torch.rand((P, 2), generator=gen, dtype=torch.float64, device=dev)
    r = torch.sqrt(mean_degree / (math.pi * sz.double()))
    cells = torch.clamp(torch.floor(1.0 / r).long(), min=1)
    cell_base = torch.zeros(G, dtype=torch.int64, device=dev)
    cell_base[1:] = torch.cumsum(cells * cells, 0)[:-1]
    gp = cells[gid]
    cx = torch.minimum((pts[:, 0] * gp).long(), gp - 1)
    cy = torch.minimum((pts[:, 1] * gp).long(), gp - 1)
    key = cell_base[gid] + cx + gp * cy
    order = torch.argsort(key)
    ncells = int((cell_base[-1] + cells[-1] * cells[-1]).item())
    count = torch.bincount(key, minlength=ncells)
    start = torch.cumsum(count, 0) - count
    maxc = int(count.max().item()) if P else 0
    r2 = (r * r)[gid]
    pid = torch.arange(P, device=dev)
    los, his = [], []
    for dx in (-1, 0, 1):
        for dy in (-1, 0, 1):
            ncx, ncy = cx + dx, cy + dy
            ok = (ncx >= 0) & (ncx < gp) & (ncy >= 0) & (ncy < gp)
            src = pid[ok]
            ncell = (cell_base[gid] + ncx + gp * ncy)[ok]
            s0, c0 = start[ncell], count[ncell]
            for j in range(maxc):
                has = c0 > j
                if not bool(has.any()):
                    break
                a = src[has]
                b = order[s0[has] + j]
                keep = a < b
                a, b = a[keep], b[keep]
                d = pts[a] - pts[b]
                close = (d * d).sum(dim=1) < r2[a]
                los.append(a[close])
                his.append(b[close])
    lo = torch.cat(los) if los else torch.zeros(0, dtype=torch.int64, device=dev)
    hi = torch.cat(his) if his else torch.zeros(0, dtype=torch.int64, device=dev)
    if wmax > 1:
        w = torch.randint(1, wmax + 1, (lo.numel(),), generator=gen, device=dev)
    else:
        w = torch.ones(lo.numel(), dtype=torch.int64, device=dev)
    src = torch.cat([lo, hi])
    dst = torch.cat([hi, lo])
    ww = torch.cat([w, w])
    perm = torch.argsort(src * max(P, 1) + dst)
    src, dst, ww = src[perm], dst[perm], ww[perm]
    xadj = torch.zeros(P + 1, dtype=torch.int64, device=dev)
    xadj[1:] = torch.cumsum(torch.bincount(src, minlength=P), 0)
    return (xadj.int(), dst.int(), ww.int(), torch.ones(P, dtype=torch.int32, device=dev), offsets.int())


def batch_partition(coarse_sizes, k: int, seed: int) -> tuple:
    """Seeded random balanced k-way partitions of many small graphs at once:
    within each graph a random order is dealt round-robin to blocks
    0..k-1 (block ids local to the graph).  Returns (part int32[sum], offsets
    int32[len+1])."""
    rng = np.random.Generator(np.random.PCG64(seed))
    sizes = np.asarray(coarse_sizes, dtype=np.int64)
    off = np.zeros(len(sizes) + 1, dtype=np.int64)
    np.cumsum(sizes, out=off[1:])
    g = np.repeat(np.arange(len(sizes)), sizes)
    order = np.lexsort((rng.random(int(off[-1])), g))
    rank = np.empty(int(off[-1]), dtype=np.int64)
    rank[order] = np.arange(int(off[-1])) - off[g[order]]
    return (rank % k).astype(np.int32), off.astype(np.int32)


def random_balanced_partition(n: int, k: int, seed: int) -> np.ndarray:
    """Seeded random balanced k-way partition of n nodes: a random permutation
    of the nodes is dealt round-robin to blocks 0..k-1, so block sizes differ
    by at most one.  Stands in for initial partitioning (Section 4)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    perm = rng.permutation(n)
    part = np.empty(n, dtype=np.int32)
    part[perm] = (np.arange(n) % k).astype(np.int32)
    return part


def random_partition(n: int, k: int, seed: int) -> np.ndarray:
    """Uniformly random block per node (not balanced)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.integers(0, k, size=n).astype(np.int32)


def _csr_from_edges_torch(n: int, lo, hi, w, name: str) -> CSRGraph:
    """Symmetric host CSR (int32, rows sorted) from undirected edges lo < hi
    held as torch tensors."""
    import torch
    src = torch.cat([lo, hi])
    dst = torch.cat([hi, lo])
    ww = torch.cat([w, w])
    perm = torch.argsort(src * max(n, 1) + dst)
    src, dst, ww = src[perm], dst[perm], ww[perm]
    xadj = torch.zeros(n + 1, dtype=torch.int64, device=src.device)
    xadj[1:] = torch.cumsum(torch.bincount(src, minlength=n), 0)
    return CSRGraph(xadj.int().cpu().numpy(), dst.int().cpu().numpy(), ww.int().cpu().numpy(),
                    np.ones(n, dtype=np.int32), name)


def rmat_torch(scale: int, seed: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
               device: str = "cuda") -> CSRGraph:
    """R-MAT graph as rmat() builds it (edge_factor * 2^scale quadrant-
    recursive samples, symmetrised, self loops dropped, duplicates merged
    into integer weights), drawn with torch on `device` for large scales;
    returned as host arrays.  Same distribution as rmat(), other draws."""
    import torch
    dev = torch.device(device)
    gen = torch.Generator(device=dev)
    gen.manual_seed(seed)
    n = 1 << scale
    M = edge_factor * n
    u = torch.zeros(M, dtype=torch.int64, device=dev)
    v = torch.zeros(M, dtype=torch.int64, device=dev)
    for bit in range(scale):
        r = torch.rand(M, generator=gen, device=dev)
        ubit = r >= a + b
        vbit = ((r >= a) & (r < a + b)) | (r >= a + b + c)
        u |= ubit.long() << bit
        v |= vbit.long() << bit
    keep = u != v
    u, v = u[keep], v[keep]
    key, cnt = torch.unique(torch.minimum(u, v) * n + torch.maximum(u, v), return_counts=True)
    return _csr_from_edges_torch(n, key // n, key % n, cnt, f"rmat_s{scale}_seed{seed}")


def rgg2d_torch(n: int, seed: int, mean_degree: float = 6.0, device: str = "cuda") -> CSRGraph:
    """2D random geometric graph with unit weights (as rgg2d), built with
    torch on `device`; returned as host arrays."""
    xadj, adj, ew, vw, _ = rgg2d_batch([n], seed, mean_degree=mean_degree, wmax=1, device=device)
    return CSRGraph(xadj.cpu().numpy(), adj.cpu().numpy(), ew.cpu().numpy(), vw.cpu().numpy(),
                    f"rgg2d_n{n}_s{seed}")


def served_mix(scales=range(12, 23), seed: int = 1, device: str = "cuda"):
    """The request pool of the serving workload: for every scale s, a 2D
    5-point grid and a 3D 7-point grid with about 2^s nodes, a 2D random
    geometric graph with 2^s nodes (mean degree 6) and an R-MAT graph of
    scale s (a=0.57, b=0.19, c=0.19, edge factor 16, duplicates merged into
    integer weights); unit node weights.  Returns a list of (family, scale,
    CSRGraph)."""
    pool = []
    for s in scales:
        side2 = int(round(2 ** (s / 2)))
        side3 = int(round(2 ** (s / 3)))
        pool.append(("grid2d", s, grid2d(side2, (1 << s) // side2)))
        pool.append(("grid3d", s, grid3d(side3, side3, max(1, (1 << s) // (side3 * side3)))))
        pool.append(("rgg2d", s, rgg2d_torch(1 << s, seed * 1000 + s, device=device)))
        pool.append(("rmat", s, rmat_torch(s, seed * 1000 + s, device=device)))
    return pool


def batch_partition_torch(coarse_sizes, k: int, seed: int, device: str = "cuda"):
    """batch_partition's distribution drawn with torch on `device` (other
    draws): within each graph a seeded random order dealt round-robin to
    blocks 0..k-1.  Returns (part int32 tensor of graph-local block ids,
    offsets int32 tensor [len+1])."""
    import torch
    dev = torch.device(device)
    sizes = torch.as_tensor(np.asarray(coarse_sizes, dtype=np.int64), device=dev)
    G = int(sizes.numel())
    N = int(sizes.sum().item()) if G else 0
    off = torch.zeros(G + 1, dtype=torch.int64, device=dev)
    if G:
        off[1:] = torch.cumsum(sizes, 0)
    gen = torch.Generator(device=dev)
    gen.manual_seed(seed)
    gid = torch.repeat_interleave(torch.arange(G, device=dev), sizes)
    r = torch.randint(0, 1 << 31, (N,), generator=gen, device=dev, dtype=torch.int64)
    order = torch.argsort((gid << 31) | r)
    rank = torch.empty(N, dtype=torch.int64, device=dev)
    rank[order] = torch.arange(N, device=dev) - off[gid[order]]
    return (rank % k).to(torch.int32), off.to(torch.int32)


def circulant_strides(n: int, count: int, seed: int) -> np.ndarray:
    """`count` distinct strides in [1, n/2) drawn with the seed (sorted)."""
    rng = np.random.default_rng(seed)
    hi = (n - 1) // 2   # s < n/2: v+s and v-s are different nodes
    if count > hi:
        raise ValueError("too many strides for n")
    return np.sort(rng.choice(np.arange(1, hi + 1, dtype=np.int64), size=count, replace=False))


def circulant(n: int, strides) -> CSRGraph:
    """Circulant graph: node v is joined to v+s and v-s (mod n) for every
    stride s; 2 * len(strides) neighbours per node, unit weights.  Pairs of a
    matching share few neighbours, so contraction keeps most entries (the
    sizes of a level barely fall while its nodes halve)."""
    S = np.asarray(strides, dtype=np.int64)
    D = np.concatenate([S, n - S])
    if n * D.size >= 1 << 31:
        raise ValueError("2^31 entries or more: circulant_torch builds those (int64 offsets)")
    v = np.arange(n, dtype=np.int64)[:, None]
    adj = np.sort((v + D[None, :]) % n, axis=1).astype(np.int32).reshape(-1)
    xadj = (np.arange(n + 1, dtype=np.int64) * D.size).astype(np.int32)
    return CSRGraph(xadj, adj, np.ones(adj.size, np.int32), np.ones(n, np.int32), f"circulant_n{n}_k{S.size}")


def circulant_torch(n: int, strides, device: str = "cuda", chunk: int = 1 << 23):
    """circulant() built with torch on `device`, rows in chunks (large n:
    more than 2^31 entries).  Returns device tensors (xadj int64, adjncy,
    ewgt, vwgt int32)."""
    import torch
    dev = torch.device(device)
    D = torch.as_tensor(np.concatenate([np.asarray(strides, np.int64), n - np.asarray(strides, np.int64)]),
                        device=dev)
    d = int(D.numel())
    adj = torch.empty(n * d, dtype=torch.int32, device=dev)
    for a in range(0, n, chunk):
        b = min(n, a + chunk)
        v = torch.arange(a, b, dtype=torch.int64, device=dev)
        nb, _ = torch.sort((v[:, None] + D[None, :]) % n, dim=1)
        adj[a * d:b * d] = nb.to(torch.int32).reshape(-1)
        del v, nb
    xadj = torch.arange(n + 1, dtype=torch.int64, device=dev) * d
    return (xadj, adj, torch.ones(n * d, dtype=torch.int32, device=dev),
            torch.ones(n, dtype=torch.int32, device=dev))
