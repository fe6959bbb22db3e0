"""CPU oracle for MIS-2, MIS-2 aggregation and the coarse graph.

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's
CPU-baseline and reference legs may import this package; the CUDA library
never calls it and shares no code with it.

The arithmetic lives in plain single-threaded C (mis2_oracle.c), which follows
the paper's Algorithm 1 (MIS-2), Algorithm 3 (aggregation; Algorithm 2 as the
BASIC mode), the coarse graph of Algorithm 4's setup, and the two Galerkin
pieces that follow it in a multilevel method (Section III-B): the coarse
edge weights and the tentative prolongator; distance-k MIS, Algorithm 1 with
unpacked tuples, and the colouring of Algorithm 4's setup (the colour sets
and cluster lists are stable groupings written here in numpy).  This module only
compiles it with gcc, marshals numpy arrays through ctypes and chains the
calls into one coarsening level and a recursive hierarchy (Section I: coarsen
recursively until the graph is below a threshold).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mis2_oracle.c")
_LIB = os.path.join(_HERE, "liboracle_mis2.so")
_lock = threading.Lock()
_lib = None

IN = 0
OUT = 0xFFFFFFFF
HASH_XORSHIFT_STAR, HASH_XORSHIFT, HASH_FIXED = 0, 1, 2
MODE_AGG, MODE_BASIC = 0, 1


class OracleError(RuntimeError):
    pass


def build(force: bool = False) -> str:
    """Compile the C oracle into liboracle_mis2.so (gcc -O2, no -march)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC],
                       check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P = ctypes.c_void_p
            i64, u64, i32 = ctypes.c_int64, ctypes.c_uint64, ctypes.c_int
            lib.oracle_mis2.argtypes = [i64, P, P, u64, i32, P, P, i64, P, P, P, i64]
            lib.oracle_mis2.restype = i32
            lib.oracle_mis2_snap.argtypes = [i64, P, P, u64, i32, P, P, i64, P, P, P, i64, P, i64]
            lib.oracle_mis2_snap.restype = i32
            lib.oracle_aggregate.argtypes = [i64, P, P, P, u64, i32, i32, P, P, P, P, P, i64]
            lib.oracle_aggregate.restype = i32
            lib.oracle_coarsen.argtypes = [i64, P, P, P, i64, P, P, P]
            lib.oracle_coarsen.restype = i32
            lib.oracle_misk.argtypes = [i64, P, P, i32, u64, i32, P, P]
            lib.oracle_misk.restype = i32
            lib.oracle_mis2_unpacked.argtypes = [i64, P, P, u64, i32, P, P]
            lib.oracle_mis2_unpacked.restype = i32
            lib.oracle_color_greedy.argtypes = [i64, P, P, u64, i32, P, P]
            lib.oracle_color_greedy.restype = i32
            lib.oracle_coarse_weights.argtypes = [i64, P, P, P, i64, P, P, P]
            lib.oracle_coarse_weights.restype = i32
            lib.oracle_prolongator.argtypes = [i64, P, i64, i32, P, P]
            lib.oracle_prolongator.restype = i32
            lib.oracle_id_bits.argtypes = [i64]
            lib.oracle_id_bits.restype = i32
            lib.oracle_pack.argtypes = [u64, i64, i32]
            lib.oracle_pack.restype = ctypes.c_uint32
            lib.oracle_hash.argtypes = [i32, u64, i64, u64]
            lib.oracle_hash.restype = ctypes.c_uint64
            lib.oracle_priority_tuple.argtypes = [i32, u64, i64, i64, u64]
            lib.oracle_priority_tuple.restype = ctypes.c_uint32
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _csr(g):
    rp = np.ascontiguousarray(g.rowptr, dtype=np.int64)
    ci = np.ascontiguousarray(g.colind, dtype=np.int32)
    return int(g.n), rp, ci


def _check(rc, what):
    if rc != 0:
        raise OracleError(f"{what} failed with status {rc}")


def id_bits(n: int) -> int:
    return int(_load().oracle_id_bits(n))


def pack(hash64: int, v: int, b: int) -> int:
    return int(_load().oracle_pack(hash64, v, b))


def hash64(iter_: int, v: int, seed: int = 0, hash_variant: int = 0) -> int:
    """h(iter, v) = f(f(iter) ^ f(v) ^ seed) of Section V-A, all 64 bits."""
    return int(_load().oracle_hash(hash_variant, iter_, v, seed))


def priority_tuple(iter_: int, v: int, n: int, seed: int = 0, hash_variant: int = 0) -> int:
    return int(_load().oracle_priority_tuple(hash_variant, iter_, v, n, seed))


def mis2(g, seed: int = 0, hash_variant: int = HASH_XORSHIFT_STAR, member=None,
         prio_table=None, trace_cap: int = 0, snap_cap: int = 0):
    """Algorithm 1.  Returns (in_set uint8[n], roots int32 ascending, rounds,
    trace int64[rounds, 4] of (W1, W2, D1, D2) or None).  With snap_cap > 0
    a fifth item holds uint32[rounds, 3, n]: T after refresh, M after the
    column step and T after decide, per round."""
    lib = _load()
    n, rp, ci = _csr(g)
    in_set = np.zeros(max(n, 1), dtype=np.uint8)
    rounds = ctypes.c_int32(0)
    mem = None if member is None else np.ascontiguousarray(member, dtype=np.uint8)
    tab, trounds = None, 0
    if prio_table is not None:
        tab = np.ascontiguousarray(prio_table, dtype=np.uint32)
        trounds = tab.shape[0]
        tab = tab.reshape(-1)
    trace = np.zeros((trace_cap, 4), dtype=np.int64) if trace_cap else None
    snaps = np.full((snap_cap, 3, max(n, 1)), OUT, dtype=np.uint32) if snap_cap else None
    rc = lib.oracle_mis2_snap(n, _ptr(rp), _ptr(ci), seed, hash_variant, _ptr(mem), _ptr(tab),
                              trounds, _ptr(in_set), ctypes.byref(rounds), _ptr(trace), trace_cap,
                              _ptr(snaps), snap_cap)
    _check(rc, "oracle_mis2")
    in_set = in_set[:n]
    roots = np.flatnonzero(in_set).astype(np.int32)
    r = int(rounds.value)
    out = (in_set, roots, r, (trace[:min(r, trace_cap)] if trace is not None else None))
    if snap_cap:
        out = out + (snaps[:min(r, snap_cap), :, :n],)
    return out


def aggregate(g, in_set, seed: int = 0, mode: int = MODE_AGG,
              hash_variant: int = HASH_XORSHIFT_STAR, trace_cap: int = 0):
    """Algorithm 3 (mode 0) or Algorithm 2 (mode 1).  Returns (labels int32[n],
    n_aggs, n_phase1, phase-2 rounds, phase-2 trace or None)."""
    lib = _load()
    n, rp, ci = _csr(g)
    flags = np.ascontiguousarray(in_set, dtype=np.uint8)
    labels = np.zeros(max(n, 1), dtype=np.int32)
    n_aggs, n1 = ctypes.c_int64(0), ctypes.c_int64(0)
    r2 = ctypes.c_int32(0)
    trace = np.zeros((trace_cap, 4), dtype=np.int64) if trace_cap else None
    rc = lib.oracle_aggregate(n, _ptr(rp), _ptr(ci), _ptr(flags), seed, hash_variant, mode,
                              _ptr(labels), ctypes.byref(n_aggs), ctypes.byref(n1),
                              ctypes.byref(r2), _ptr(trace), trace_cap)
    _check(rc, "oracle_aggregate")
    r = int(r2.value)
    return (labels[:n], int(n_aggs.value), int(n1.value), r,
            (trace[:min(r, trace_cap)] if trace is not None else None))


def coarsen(g, labels, n_aggs: int):
    """Coarse graph of an aggregation: returns (c_rowptr int64, c_colind int32)."""
    lib = _load()
    n, rp, ci = _csr(g)
    lab = np.ascontiguousarray(labels, dtype=np.int32)
    c_rowptr = np.zeros(n_aggs + 1, dtype=np.int64)
    c_nnz = ctypes.c_int64(0)
    rc = lib.oracle_coarsen(n, _ptr(rp), _ptr(ci), _ptr(lab), n_aggs, _ptr(c_rowptr), None,
                            ctypes.byref(c_nnz))
    _check(rc, "oracle_coarsen")
    c_colind = np.zeros(max(int(c_nnz.value), 1), dtype=np.int32)
    rc = lib.oracle_coarsen(n, _ptr(rp), _ptr(ci), _ptr(lab), n_aggs, _ptr(c_rowptr),
                            _ptr(c_colind), ctypes.byref(c_nnz))
    _check(rc, "oracle_coarsen")
    return c_rowptr, c_colind[:int(c_nnz.value)]


def misk(g, k: int, seed: int = 0, hash_variant: int = HASH_XORSHIFT_STAR):
    """Distance-k MIS (k = 2: Algorithm 1).  Returns (in_set uint8[n], roots
    int32 ascending, rounds)."""
    lib = _load()
    n, rp, ci = _csr(g)
    in_set = np.zeros(max(n, 1), dtype=np.uint8)
    rounds = ctypes.c_int32(0)
    rc = lib.oracle_misk(n, _ptr(rp), _ptr(ci), k, seed, hash_variant, _ptr(in_set), ctypes.byref(rounds))
    _check(rc, "oracle_misk")
    in_set = in_set[:n]
    return in_set, np.flatnonzero(in_set).astype(np.int32), int(rounds.value)


def mis2_unpacked(g, seed: int = 0, hash_variant: int = HASH_XORSHIFT_STAR):
    """Algorithm 1 with unpacked (status, priority, id) tuples, priority =
    the 32-b bits Eq. 1 packs.  Returns (in_set uint8[n], roots int32,
    rounds)."""
    lib = _load()
    n, rp, ci = _csr(g)
    in_set = np.zeros(max(n, 1), dtype=np.uint8)
    rounds = ctypes.c_int32(0)
    rc = lib.oracle_mis2_unpacked(n, _ptr(rp), _ptr(ci), seed, hash_variant, _ptr(in_set), ctypes.byref(rounds))
    _check(rc, "oracle_mis2_unpacked")
    in_set = in_set[:n]
    return in_set, np.flatnonzero(in_set).astype(np.int32), int(rounds.value)


def color_greedy(g, seed: int = 0, hash_variant: int = HASH_XORSHIFT_STAR):
    """First-fit coloring in ascending round-0 tuple order: (colors int32[n],
    n_colors)."""
    lib = _load()
    n, rp, ci = _csr(g)
    colors = np.zeros(max(n, 1), dtype=np.int32)
    nc = ctypes.c_int32(0)
    rc = lib.oracle_color_greedy(n, _ptr(rp), _ptr(ci), seed, hash_variant, _ptr(colors), ctypes.byref(nc))
    _check(rc, "oracle_color_greedy")
    return colors[:n], int(nc.value)


def group_by(keys, n_keys: int):
    """Indices 0..n-1 grouped by key, ascending within a key: (ptr int64
    [n_keys+1], list int32); key k owns list[ptr[k]:ptr[k+1]]."""
    keys = np.asarray(keys)
    ptr = np.zeros(n_keys + 1, dtype=np.int64)
    np.add.at(ptr, keys.astype(np.int64) + 1, 1)
    ptr = np.cumsum(ptr)
    order = np.argsort(keys, kind="stable").astype(np.int32)
    return ptr, order


def color_sets(colors, n_colors: int):
    """The colour sets of Algorithm 4 (vertices of each colour, ascending)."""
    return group_by(colors, n_colors)


def cluster_lists(labels, n_aggs: int):
    """The clusters of Algorithm 4 (fine vertices of each aggregate,
    ascending)."""
    return group_by(labels, n_aggs)


def coarse_weights(g, labels, n_aggs: int, c_rowptr, c_colind):
    """Number of fine entries behind each coarse entry (int64, aligned with
    c_colind): the off-diagonal of P^T A P for 0/1 A and P."""
    lib = _load()
    n, rp, ci = _csr(g)
    lab = np.ascontiguousarray(labels, dtype=np.int32)
    crp = np.ascontiguousarray(c_rowptr, dtype=np.int64)
    cci = np.ascontiguousarray(c_colind, dtype=np.int32)
    w = np.zeros(max(int(crp[-1]), 1), dtype=np.int64)
    rc = lib.oracle_coarse_weights(n, _ptr(rp), _ptr(ci), _ptr(lab), n_aggs, _ptr(crp), _ptr(cci), _ptr(w))
    _check(rc, "oracle_coarse_weights")
    return w[:int(crp[-1])]


def prolongator(labels, n_aggs: int, normalize: bool = True):
    """Tentative prolongator, one entry per row: (p_colind int32, p_values
    float64); the row pointer is 0, 1, ..., n."""
    lib = _load()
    lab = np.ascontiguousarray(labels, dtype=np.int32)
    n = lab.shape[0]
    pc = np.zeros(max(n, 1), dtype=np.int32)
    pv = np.zeros(max(n, 1), dtype=np.float64)
    rc = lib.oracle_prolongator(n, _ptr(lab), n_aggs, 1 if normalize else 0, _ptr(pc), _ptr(pv))
    _check(rc, "oracle_prolongator")
    return pc[:n], pv[:n]


class Level:
    """One coarsening level: MIS-2, aggregation and the coarse graph."""

    def __init__(self, in_set, roots, rounds, labels, n_aggs, n_phase1, rounds2, c_rowptr,
                 c_colind, trace=None, trace2=None):
        self.in_set, self.roots, self.rounds = in_set, roots, rounds
        self.labels, self.n_aggs, self.n_phase1, self.rounds2 = labels, n_aggs, n_phase1, rounds2
        self.c_rowptr, self.c_colind = c_rowptr, c_colind
        self.trace, self.trace2 = trace, trace2


def coarsen_level(g, seed: int = 0, mode: int = MODE_AGG, hash_variant: int = HASH_XORSHIFT_STAR,
                  trace_cap: int = 0) -> Level:
    in_set, roots, rounds, trace = mis2(g, seed, hash_variant, trace_cap=trace_cap)
    labels, n_aggs, n1, r2, trace2 = aggregate(g, in_set, seed, mode, hash_variant, trace_cap)
    c_rowptr, c_colind = coarsen(g, labels, n_aggs)
    return Level(in_set, roots, rounds, labels, n_aggs, n1, r2, c_rowptr, c_colind, trace, trace2)


def hierarchy(g, min_n: int = 1000, max_levels: int = 32, seed: int = 0,
              mode: int = MODE_AGG):
    """Recursive coarsening: coarsen while n >= min_n, the graph still
    shrinks, and fewer than max_levels levels were built.  Returns the list
    of Levels (level k maps the level-k graph onto the level-(k+1) graph)."""
    from types import SimpleNamespace

    levels = []
    cur = g
    while cur.n >= min_n and len(levels) < max_levels:
        lv = coarsen_level(cur, seed, mode)
        levels.append(lv)
        if lv.n_aggs >= cur.n:
            break
        cur = SimpleNamespace(n=lv.n_aggs, rowptr=lv.c_rowptr, colind=lv.c_colind)
    return levels
