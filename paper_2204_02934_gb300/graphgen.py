"""Seeded synthetic graph generators.

These build the inputs that both the CUDA path and the CPU oracle consume.
They hold none of the MIS-2 / aggregation arithmetic: only stencil
adjacency, R-MAT sampling and random geometric graphs.

Every generator returns a symmetric CSR graph with sorted, unique column
indices and no self-loops (the MIS-2 column step adds the vertex itself, so
the diagonal carries no information).  Random draws come from a
counter-based SplitMix64 stream (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), so a (seed, counter) pair
always yields the same value on every machine.

Workload shapes follow the paper's test matrices (Section VI: Laplace3D is a
7-point 100^3 grid, Elasticity3D a 27-point grid with 3 dof per point) and the
synthetic stand-ins used for its SuiteSparse graphs (R-MAT, random geometric
graphs, mixed-size batches).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

@dataclass
class CSRGraph:
    """Host CSR graph.  rowptr is int64[n+1] (or int32), colind int32[nnz]."""

    n: int
    rowptr: np.ndarray
    colind: np.ndarray
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.colind.shape[0])

    def degrees(self) -> np.ndarray:
        rp = self.rowptr.astype(np.int64)
        return rp[1:] - rp[:-1]

    def with_rowptr(self, dtype) -> "CSRGraph":
        return CSRGraph(self.n, self.rowptr.astype(dtype), self.colind, self.name)


# ---------------------------------------------------------------- randomness
def splitmix64(counters: np.ndarray, seed: int) -> np.ndarray:
    """SplitMix64 output for each counter (uint64 array) under `seed`."""
    with np.errstate(over="ignore"):
        z = (np.uint64(seed & 0xFFFFFFFFFFFFFFFF)
             + (counters.astype(np.uint64) + np.uint64(1)) * np.uint64(0x9E3779B97F4A7C15))
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(counters: np.ndarray, seed: int) -> np.ndarray:
    """Doubles in [0, 1) from the top 53 bits of SplitMix64."""
    return (splitmix64(counters, seed) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


# ---------------------------------------------------------------- CSR helpers
def csr_from_pairs(n: int, src: np.ndarray, dst: np.ndarray, name: str = "",
                   rowptr_dtype=np.int64) -> CSRGraph:
    """Symmetrise (src,dst) pairs, drop self-loops and duplicates, build CSR."""
    src = np.asarray(src, dtype=np.int64)
    dst = np.asarray(dst, dtype=np.int64)
    keep = src != dst
    src, dst = src[keep], dst[keep]
    keys = np.concatenate([src * n + dst, dst * n + src])
    keys.sort()
    if keys.shape[0] > 1:
        keys = keys[np.concatenate([[True], keys[1:] != keys[:-1]])]
    rows = keys // n
    cols = (keys - rows * n).astype(np.int32)
    counts = np.bincount(rows, minlength=n).astype(np.int64)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    return CSRGraph(n, rowptr.astype(rowptr_dtype), cols, name)


def _stencil_graph(dims, offsets, name, rowptr_dtype=np.int32) -> CSRGraph:
    """Grid graph whose neighbours are `offsets` (tuples over dims), no self."""
    dims = tuple(int(d) for d in dims)
    n = int(np.prod(dims))
    if n == 0:
        return CSRGraph(0, np.zeros(1, dtype=rowptr_dtype), np.zeros(0, dtype=np.int32), name)
    idx = np.arange(n, dtype=np.int64)
    coords = np.unravel_index(idx, dims)  # C order: last dim fastest
    strides = np.array([int(np.prod(dims[i + 1:])) for i in range(len(dims))], dtype=np.int64)
    # sort offsets by linear delta so every row comes out ascending
    offsets = sorted(offsets, key=lambda o: int(np.dot(o, strides)))
    cols = np.full((n, len(offsets)), -1, dtype=np.int64)
    for k, off in enumerate(offsets):
        ok = np.ones(n, dtype=bool)
        for d, o in enumerate(off):
            c = coords[d] + o
            ok &= (c >= 0) & (c < dims[d])
        cols[ok, k] = idx[ok] + int(np.dot(off, strides))
    valid = cols >= 0
    counts = valid.sum(axis=1)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    colind = cols[valid].astype(np.int32)
    return CSRGraph(n, rowptr.astype(rowptr_dtype), colind, name)


def _offsets(ndim: int, full: bool):
    rng = (-1, 0, 1)
    out = []
    if full:
        for o in np.ndindex(*(3,) * ndim):
            off = tuple(rng[i] for i in o)
            if any(off):
                out.append(off)
    else:
        for d in range(ndim):
            for s in (-1, 1):
                off = [0] * ndim
                off[d] = s
                out.append(tuple(off))
    return out


def grid2d_5pt(nx: int, ny: int, rowptr_dtype=np.int32) -> CSRGraph:
    """2D 5-point Laplacian grid graph (4 neighbours in the interior)."""
    return _stencil_graph((ny, nx), _offsets(2, False), f"grid2d_5pt_{nx}x{ny}", rowptr_dtype)


def grid3d_7pt(nx: int, ny: int, nz: int, rowptr_dtype=np.int32) -> CSRGraph:
    """3D 7-point Laplacian grid graph (Laplace3D in the paper's Section VI)."""
    return _stencil_graph((nz, ny, nx), _offsets(3, False), f"grid3d_7pt_{nx}x{ny}x{nz}", rowptr_dtype)


def grid3d_27pt(nx: int, ny: int, nz: int, rowptr_dtype=np.int32) -> CSRGraph:
    """3D 27-point stencil grid graph (26 neighbours in the interior)."""
    return _stencil_graph((nz, ny, nx), _offsets(3, True), f"grid3d_27pt_{nx}x{ny}x{nz}", rowptr_dtype)


def elasticity3d(nx: int, ny: int, nz: int, dof: int = 3, rowptr_dtype=np.int32) -> CSRGraph:
    """27-point grid with `dof` fully coupled unknowns per point (Elasticity3D).

    Vertex p*dof+i couples to every dof of every point in the closed 27-point
    neighbourhood of p, so interior rows hold 27*dof - 1 off-diagonal entries
    (81 stored entries with the diagonal, the paper's max degree).
    """
    g = grid3d_27pt(nx, ny, nz, np.int64)
    npts = g.n
    prow = np.concatenate([np.repeat(np.arange(npts, dtype=np.int64), g.degrees()),
                           np.arange(npts, dtype=np.int64)])
    pcol = np.concatenate([g.colind.astype(np.int64), np.arange(npts, dtype=np.int64)])
    src = (prow[:, None, None] * dof + np.arange(dof)[None, :, None]) + 0 * np.arange(dof)[None, None, :]
    dst = (pcol[:, None, None] * dof + np.arange(dof)[None, None, :]) + 0 * np.arange(dof)[None, :, None]
    out = csr_from_pairs(npts * dof, src.reshape(-1), dst.reshape(-1),
                         f"elasticity3d_{nx}x{ny}x{nz}x{dof}", np.int64)
    return out.with_rowptr(rowptr_dtype)


def rmat(scale: int, pairs_per_vertex: int = 8, a: float = 0.57, b: float = 0.19,
         c: float = 0.19, seed: int = 42, rowptr_dtype=np.int64) -> CSRGraph:
    """R-MAT graph (Chakrabarti, Zhan & Faloutsos, SDM 2004).

    Samples pairs_per_vertex * 2^scale (row, col) pairs by recursive quadrant
    choice with probabilities (a, b, c, 1-a-b-c), no noise and no relabelling,
    then symmetrises and drops self-loops and duplicates.  With 8 pairs per
    vertex the symmetrised average degree is close to 16.
    """
    n = 1 << scale
    m = pairs_per_vertex * n
    ta = np.uint32(min(int(a * 4294967296.0), 0xFFFFFFFF))
    tab = np.uint32(min(int((a + b) * 4294967296.0), 0xFFFFFFFF))
    tabc = np.uint32(min(int((a + b + c) * 4294967296.0), 0xFFFFFFFF))
    src = np.zeros(m, dtype=np.int64)
    dst = np.zeros(m, dtype=np.int64)
    words = (scale + 1) // 2
    base = np.arange(m, dtype=np.uint64) * np.uint64(words)
    for w in range(words):
        r = splitmix64(base + np.uint64(w), seed)
        for half in range(2):
            lvl = 2 * w + half
            if lvl >= scale:
                break
            u = (r >> np.uint64(32 * half)).astype(np.uint32)
            rbit = (u >= tab).astype(np.int64)               # quadrants c, d -> lower half
            cbit = (((u >= ta) & (u < tab)) | (u >= tabc)).astype(np.int64)  # b, d -> right half
            src = (src << 1) | rbit
            dst = (dst << 1) | cbit
        del r
    return csr_from_pairs(n, src, dst, f"rmat_s{scale}", rowptr_dtype)


def rgg2d(n: int, avg_degree: float = 10.0, seed: int = 7, rowptr_dtype=np.int32) -> CSRGraph:
    """2D random geometric graph: n uniform points in [0,1)^2, radius
    sqrt(avg_degree / (pi n)), built by spatial binning (scipy cKDTree)."""
    from scipy.spatial import cKDTree

    if n <= 1:
        return CSRGraph(n, np.zeros(n + 1, dtype=rowptr_dtype), np.zeros(0, dtype=np.int32), f"rgg2d_{n}")
    cnt = np.arange(2 * n, dtype=np.uint64)
    u = uniform01(cnt, seed)
    pts = np.stack([u[0::2], u[1::2]], axis=1)
    r = math.sqrt(avg_degree / (math.pi * n))
    pairs = cKDTree(pts).query_pairs(r, output_type="ndarray")
    g = csr_from_pairs(n, pairs[:, 0], pairs[:, 1], f"rgg2d_{n}", rowptr_dtype)
    return g


# ---------------------------------------------------------------- workloads
def workload_small(rowptr_dtype=np.int32) -> CSRGraph:
    """100x100 2D 5-point grid: 10,000 vertices, 39,600 off-diagonal entries."""
    return grid2d_5pt(100, 100, rowptr_dtype)


def workload_27pt(side: int = 100, rowptr_dtype=np.int32) -> CSRGraph:
    """side^3 27-point grid: 10^6 vertices and 25,463,592 entries at side 100."""
    return grid3d_27pt(side, side, side, rowptr_dtype)


def workload_rmat(scale: int = 22, seed: int = 42) -> CSRGraph:
    """R-MAT scale 22, (0.57, 0.19, 0.19, 0.05), 8n pairs, int64 rowptr."""
    return rmat(scale, 8, 0.57, 0.19, 0.19, seed, np.int64)


def batch_sizes(n_graphs: int = 512, lo: float = 1e3, hi: float = 2e5, seed: int = 7):
    """Log-uniform sizes and uniform types (0: 2D 5-pt, 1: 3D 7-pt, 2: RGG)."""
    u = uniform01(np.arange(2 * n_graphs, dtype=np.uint64), seed ^ 0x5EED)
    sizes = np.rint(np.exp(math.log(lo) + u[0::2] * (math.log(hi) - math.log(lo)))).astype(np.int64)
    types = np.minimum((u[1::2] * 3).astype(np.int64), 2)
    return sizes, types


def mixed_batch(n_graphs: int = 512, lo: float = 1e3, hi: float = 2e5, seed: int = 7):
    """Mixed-size batch of 2D 5-pt grids, 3D 7-pt grids and 2D RGGs."""
    sizes, types = batch_sizes(n_graphs, lo, hi, seed)
    out = []
    for i, (nv, t) in enumerate(zip(sizes.tolist(), types.tolist())):
        if t == 0:
            s = max(1, int(round(math.sqrt(nv))))
            out.append(grid2d_5pt(s, s))
        elif t == 1:
            s = max(1, int(round(nv ** (1.0 / 3.0))))
            out.append(grid3d_7pt(s, s, s))
        else:
            out.append(rgg2d(int(nv), 10.0, seed * 1000003 + i))
    return out


def serving_graph(i: int, n_graphs: int = 64, seed: int = 11, max_side: int = 160, max_scale: int = 20) -> CSRGraph:
    """Graph i of the request pool: a 3D 7-pt grid (side log-uniform in
    [20, max_side]) or an R-MAT graph (scale uniform in [14, max_scale],
    average degree 16), each with probability 1/2; int32 rowptr."""
    u = uniform01(np.arange(3 * i, 3 * i + 3, dtype=np.uint64), seed)
    if u[0] < 0.5:
        side = int(round(math.exp(math.log(20) + u[1] * (math.log(max_side) - math.log(20)))))
        return grid3d_7pt(side, side, side)
    sc = 14 + min(int(u[2] * (max_scale - 13)), max_scale - 14)
    return rmat(sc, 8, 0.57, 0.19, 0.19, seed * 7919 + i, np.int32)


def _serving_graph_star(args):
    return serving_graph(*args)


def serving_pool(n_graphs: int = 64, seed: int = 11, max_side: int = 160, max_scale: int = 20,
                 processes: int = 1) -> list:
    """The request pool (serving_graph 0..n_graphs-1).  processes > 1 builds
    the graphs in a spawned process pool (safe after CUDA is initialised)."""
    jobs = [(i, n_graphs, seed, max_side, max_scale) for i in range(n_graphs)]
    if processes <= 1:
        return [serving_graph(*j) for j in jobs]
    import multiprocessing as mp

    with mp.get_context("spawn").Pool(processes) as pool:
        return pool.map(_serving_graph_star, jobs, chunksize=1)


def poisson_arrivals(n_requests: int, rate_per_s: float, seed: int = 13) -> np.ndarray:
    """Arrival times (s) of a Poisson process: exponential inter-arrival gaps."""
    u = uniform01(np.arange(n_requests, dtype=np.uint64), seed)
    gaps = -np.log1p(-u) / rate_per_s
    return np.cumsum(gaps)


def random_graph(n: int, p: float, seed: int) -> CSRGraph:
    """Erdos-Renyi G(n, p) (small n only: draws one number per vertex pair)."""
    iu, ju = np.triu_indices(n, 1)
    u = uniform01(np.arange(iu.shape[0], dtype=np.uint64), seed)
    keep = u < p
    return csr_from_pairs(n, iu[keep], ju[keep], f"gnp_{n}_{p}", np.int64)


def graph_from_edges(n: int, edges, rowptr_dtype=np.int64) -> CSRGraph:
    """CSR from an explicit undirected edge list (tests, worked examples)."""
    if len(edges) == 0:
        return CSRGraph(n, np.zeros(n + 1, dtype=rowptr_dtype), np.zeros(0, dtype=np.int32))
    e = np.asarray(edges, dtype=np.int64)
    return csr_from_pairs(n, e[:, 0], e[:, 1], "edges", rowptr_dtype)
