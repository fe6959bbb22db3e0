"""Python binding of the C ABI in include/mis2.h (argument marshalling only).

Every function named mis2_* here calls the C function of the same name in
libmis2_gb300.so through ctypes; all computation runs in the library's CUDA
kernels.  There is no CPU fallback: if the library is missing or fails to
load, importing the binding raises.

Device buffers come from torch (CUDA tensors); streams are torch streams.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import _build

MIS2_OK = 0
STATUS = {
    0: "MIS2_OK", -1: "MIS2_ERR_INVALID_ARG", -2: "MIS2_ERR_OUT_OF_MEMORY", -3: "MIS2_ERR_CUDA",
    -4: "MIS2_ERR_BAD_GRAPH", -5: "MIS2_ERR_TIMEOUT", -6: "MIS2_ERR_NO_PROGRESS", -7: "MIS2_ERR_CANCELLED",
}
MIS2_AGG_ALG3, MIS2_AGG_BASIC = 0, 1
MIS2_HASH_XORSHIFT_STAR, MIS2_HASH_XORSHIFT, MIS2_HASH_FIXED = 0, 1, 2
MIS2_LOOP_HOST, MIS2_LOOP_DEVICE = 0, 1
MIS2_TIMING_OFF, MIS2_TIMING_ALL, MIS2_TIMING_LOOP = 0, 1, 2
MIS2_DEBUG_VALIDATE, MIS2_DEBUG_FORCE_TIMEOUT = 0x1, 0x100
MIS2_ABLATE_NO_WORKLISTS, MIS2_ABLATE_TUPLE_ENGINE, MIS2_ABLATE_UNPACKED_TUPLES = 0x1, 0x2, 0x4
MIS2_TRACE_CAP = 64
MIS2_NUM_KERNEL_CLASSES = 8
KERNEL_CLASSES = ["init", "column", "decide", "compact", "aggregate", "coarse", "device_loop", "other"]

# C function names the header declares (checked by the CPU tests).
EXPORTS = [
    "mis2_config_default", "mis2_ctx_create", "mis2_ctx_destroy", "mis2_ctx_set_config", "mis2_get_stats",
    "mis2_run", "mis2_run_with_priorities", "mis2_run_snapshots", "mis2_aggregate", "mis2_coarsen", "mis2_coarsen_level",
    "mis2_coarsen_level_host", "mis2_status_string", "mis2_last_error", "mis2_version", "mis2_run_noalloc",
    "mis2_batch_create", "mis2_batch_destroy", "mis2_batch_coarsen", "mis2_batch_level_sizes", "mis2_batch_labels",
    "mis2_batch_coarse", "mis2_batch_stats",
    "mis2_server_config_default", "mis2_server_create", "mis2_server_destroy", "mis2_server_submit",
    "mis2_server_submit_out",
    "mis2_server_wait", "mis2_server_cancel", "mis2_server_replay", "mis2_coarse_weights", "mis2_tentative_prolongator",
    "mis2_run_k", "mis2_color", "mis2_cluster_lists",
]
MIS2_NOALLOC_MAX_N = 262144


class Mis2Error(RuntimeError):
    def __init__(self, status: int, where: str):
        detail = ""
        if status == -3:
            try:
                detail = ": " + _lib().mis2_last_error().decode()
            except Exception:  # pragma: no cover
                pass
        super().__init__(f"{where} returned {STATUS.get(status, status)}{detail}")
        self.status = status


class mis2_csr(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz", ctypes.c_int64), ("rowptr_is_64", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("rowptr", ctypes.c_void_p), ("colind", ctypes.c_void_p)]


class mis2_config(ctypes.Structure):
    _fields_ = [("hash_variant", ctypes.c_int32), ("agg_mode", ctypes.c_int32), ("group_lanes", ctypes.c_int32),
                ("warp_degree", ctypes.c_int32), ("block_degree", ctypes.c_int32), ("block_size", ctypes.c_int32),
                ("loop", ctypes.c_int32), ("debug_checks", ctypes.c_int32), ("timing", ctypes.c_int32),
                ("loop_blocks_per_sm", ctypes.c_int32), ("ablation", ctypes.c_int32),
                ("serial_launches", ctypes.c_int32), ("spin_limit", ctypes.c_int64)]


class mis2_server_config(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_int32), ("batch_max", ctypes.c_int32), ("mem_budget", ctypes.c_int64),
                ("slot_max_n", ctypes.c_int64), ("slot_max_nnz", ctypes.c_int64), ("cfg", mis2_config)]


class mis2_request_out(ctypes.Structure):
    _fields_ = [("in_set", ctypes.c_void_p), ("roots", ctypes.c_void_p), ("labels", ctypes.c_void_p),
                ("c_rowptr", ctypes.c_void_p), ("c_colind", ctypes.c_void_p), ("c_colind_cap", ctypes.c_int64)]


class mis2_result(ctypes.Structure):
    _fields_ = [("ticket", ctypes.c_int64), ("n", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("n_roots", ctypes.c_int64), ("n_aggs", ctypes.c_int64), ("c_nnz", ctypes.c_int64),
                ("checksum", ctypes.c_uint64), ("t_arrive", ctypes.c_double), ("t_start", ctypes.c_double),
                ("t_done", ctypes.c_double), ("status", ctypes.c_int32), ("slot", ctypes.c_int32)]


class mis2_stats(ctypes.Structure):
    _fields_ = [("rounds", ctypes.c_int32), ("rounds2", ctypes.c_int32), ("n_roots", ctypes.c_int64),
                ("n_phase1", ctypes.c_int64), ("n_aggs", ctypes.c_int64), ("c_nnz", ctypes.c_int64),
                ("trace", (ctypes.c_int64 * 4) * MIS2_TRACE_CAP),
                ("trace2", (ctypes.c_int64 * 4) * MIS2_TRACE_CAP),
                ("kernel_ms", ctypes.c_double * MIS2_NUM_KERNEL_CLASSES),
                ("kernel_launches", ctypes.c_int64 * MIS2_NUM_KERNEL_CLASSES),
                ("launches", ctypes.c_int64),
                ("loop_ns", (ctypes.c_int64 * (4 + 4 * MIS2_TRACE_CAP)) * 2)]


_LIB = None


def library_path() -> str:
    return _build.LIB_PATH


def _lib(build_if_missing: bool = False):
    """Load libmis2_gb300.so (raises if it is missing: no fallback)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = _build.LIB_PATH
    if not os.path.exists(path):
        if build_if_missing:
            _build.build()
        else:
            raise ImportError(f"{path} is missing: build it with paper_2204_02934_gb300._build.build()")
    lib = ctypes.CDLL(path)
    P, i32, i64, u64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
    CSR, CFG = ctypes.POINTER(mis2_csr), ctypes.POINTER(mis2_config)
    pi64, pi32 = ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int32)
    sig = {
        "mis2_config_default": (None, [CFG]),
        "mis2_ctx_create": (i32, [ctypes.POINTER(P), i64, i64, CFG]),
        "mis2_ctx_destroy": (i32, [P]),
        "mis2_ctx_set_config": (i32, [P, CFG]),
        "mis2_get_stats": (i32, [P, ctypes.POINTER(mis2_stats)]),
        "mis2_run": (i32, [P, CSR, u64, P, P, pi64, pi32, P]),
        "mis2_run_with_priorities": (i32, [P, CSR, P, i32, P, P, pi64, pi32, P]),
        "mis2_run_snapshots": (i32, [P, CSR, P, i32, P, i32, P, P, pi64, pi32, P]),
        "mis2_aggregate": (i32, [P, CSR, P, i64, u64, i32, P, pi64, P]),
        "mis2_coarsen": (i32, [P, CSR, P, i64, P, P, i64, pi64, P]),
        "mis2_coarsen_level": (i32, [P, CSR, u64, P, P, P, P, P, i64, pi64, pi64, pi64, P]),
        "mis2_coarsen_level_host": (i32, [P, CSR, u64, P, P, P, P, P, i64, pi64, pi64, pi64, P]),
        "mis2_run_noalloc": (i32, [CSR, u64, P, P, pi64, pi32, P]),
        "mis2_batch_create": (i32, [ctypes.POINTER(P), i32, i64, i64, CFG]),
        "mis2_batch_destroy": (i32, [P]),
        "mis2_batch_coarsen": (i32, [P, i32, CSR, u64, i64, i32, pi32, P]),
        "mis2_batch_level_sizes": (i32, [P, i32, P, P, P]),
        "mis2_batch_labels": (i32, [P, i32, i32, P, P]),
        "mis2_batch_coarse": (i32, [P, i32, i32, P, P, i64, P]),
        "mis2_batch_stats": (i32, [P, ctypes.POINTER(mis2_stats)]),
        "mis2_server_config_default": (None, [ctypes.POINTER(mis2_server_config)]),
        "mis2_server_create": (i32, [ctypes.POINTER(P), ctypes.POINTER(mis2_server_config)]),
        "mis2_server_destroy": (i32, [P]),
        "mis2_server_submit": (i32, [P, CSR, u64, pi64]),
        "mis2_server_submit_out": (i32, [P, CSR, u64, ctypes.POINTER(mis2_request_out), pi64]),
        "mis2_server_wait": (i32, [P, i64, ctypes.POINTER(mis2_result)]),
        "mis2_server_cancel": (i32, [P, i64, pi32]),
        "mis2_server_replay": (i32, [P, i32, CSR, i64, P, P, u64, ctypes.POINTER(mis2_result), pi64]),
        "mis2_coarse_weights": (i32, [P, CSR, P, i64, P, P, i64, P, P]),
        "mis2_run_k": (i32, [P, CSR, i32, u64, P, P, pi64, pi32, P]),
        "mis2_color": (i32, [P, CSR, u64, P, P, P, pi32, pi32, P]),
        "mis2_cluster_lists": (i32, [P, P, i64, i64, P, P, P]),
        "mis2_tentative_prolongator": (i32, [P, P, i64, i64, i32, P, P, P, P]),
        "mis2_status_string": (ctypes.c_char_p, [i32]),
        "mis2_last_error": (ctypes.c_char_p, []),
        "mis2_version": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _LIB = lib
    return lib


def _check(rc: int, where: str):
    if rc != MIS2_OK:
        raise Mis2Error(rc, where)


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return ctypes.c_void_p(t.ctypes.data)
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        import torch

        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


# --------------------------------------------------------------- C-ABI names
def mis2_config_default() -> mis2_config:
    cfg = mis2_config()
    _lib().mis2_config_default(ctypes.byref(cfg))
    return cfg


def mis2_ctx_create(max_n: int, max_nnz: int, cfg: mis2_config | None = None) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(_lib().mis2_ctx_create(ctypes.byref(h), max_n, max_nnz, ctypes.byref(cfg) if cfg else None),
           "mis2_ctx_create")
    return h


def mis2_ctx_destroy(ctx) -> None:
    _check(_lib().mis2_ctx_destroy(ctx), "mis2_ctx_destroy")


def mis2_ctx_set_config(ctx, cfg: mis2_config) -> None:
    _check(_lib().mis2_ctx_set_config(ctx, ctypes.byref(cfg)), "mis2_ctx_set_config")


def mis2_get_stats(ctx) -> mis2_stats:
    st = mis2_stats()
    _check(_lib().mis2_get_stats(ctx, ctypes.byref(st)), "mis2_get_stats")
    return st


def mis2_run(ctx, g: mis2_csr, seed: int, in_set, roots, stream=None):
    """Returns (n_roots, n_rounds); in_set / roots are device tensors or None."""
    nr, rounds = ctypes.c_int64(0), ctypes.c_int32(0)
    _check(_lib().mis2_run(ctx, ctypes.byref(g), seed, _ptr(in_set), _ptr(roots), ctypes.byref(nr),
                           ctypes.byref(rounds), _stream(stream)), "mis2_run")
    return nr.value, rounds.value


def mis2_run_with_priorities(ctx, g: mis2_csr, prio_table: np.ndarray, in_set, roots, stream=None):
    tab = np.ascontiguousarray(prio_table, dtype=np.uint32)
    nr, rounds = ctypes.c_int64(0), ctypes.c_int32(0)
    _check(_lib().mis2_run_with_priorities(ctx, ctypes.byref(g), _ptr(tab), tab.shape[0], _ptr(in_set),
                                           _ptr(roots), ctypes.byref(nr), ctypes.byref(rounds), _stream(stream)),
           "mis2_run_with_priorities")
    return nr.value, rounds.value


def mis2_run_snapshots(ctx, g: mis2_csr, prio_table: np.ndarray, snaps, snap_rounds: int, in_set, roots,
                       stream=None):
    tab = np.ascontiguousarray(prio_table, dtype=np.uint32)
    nr, rounds = ctypes.c_int64(0), ctypes.c_int32(0)
    _check(_lib().mis2_run_snapshots(ctx, ctypes.byref(g), _ptr(tab), tab.shape[0], _ptr(snaps), snap_rounds,
                                     _ptr(in_set), _ptr(roots), ctypes.byref(nr), ctypes.byref(rounds),
                                     _stream(stream)), "mis2_run_snapshots")
    return nr.value, rounds.value


def mis2_aggregate(ctx, g: mis2_csr, roots, n_roots: int, seed: int, mode: int, labels, stream=None) -> int:
    na = ctypes.c_int64(0)
    _check(_lib().mis2_aggregate(ctx, ctypes.byref(g), _ptr(roots), n_roots, seed, mode, _ptr(labels),
                                 ctypes.byref(na), _stream(stream)), "mis2_aggregate")
    return na.value


def mis2_coarsen(ctx, g: mis2_csr, labels, n_aggs: int, c_rowptr, c_colind, c_colind_cap: int, stream=None) -> int:
    cn = ctypes.c_int64(0)
    _check(_lib().mis2_coarsen(ctx, ctypes.byref(g), _ptr(labels), n_aggs, _ptr(c_rowptr), _ptr(c_colind),
                               c_colind_cap, ctypes.byref(cn), _stream(stream)), "mis2_coarsen")
    return cn.value


def mis2_coarsen_level(ctx, g: mis2_csr, seed: int, in_set, roots, labels, c_rowptr, c_colind, c_colind_cap: int,
                       stream=None):
    """Returns (n_roots, n_aggs, c_nnz)."""
    nr, na, cn = ctypes.c_int64(0), ctypes.c_int64(0), ctypes.c_int64(0)
    _check(_lib().mis2_coarsen_level(ctx, ctypes.byref(g), seed, _ptr(in_set), _ptr(roots), _ptr(labels),
                                     _ptr(c_rowptr), _ptr(c_colind), c_colind_cap, ctypes.byref(nr),
                                     ctypes.byref(na), ctypes.byref(cn), _stream(stream)), "mis2_coarsen_level")
    return nr.value, na.value, cn.value


def mis2_coarsen_level_host(ctx, g_host: mis2_csr, seed: int, in_set, roots, labels, c_rowptr, c_colind,
                            c_colind_cap: int, stream=None):
    """Host-buffer variant (numpy arrays or pinned CPU tensors).  Returns
    (n_roots, n_aggs, c_nnz)."""
    nr, na, cn = ctypes.c_int64(0), ctypes.c_int64(0), ctypes.c_int64(0)
    _check(_lib().mis2_coarsen_level_host(ctx, ctypes.byref(g_host), seed, _ptr(in_set), _ptr(roots),
                                          _ptr(labels), _ptr(c_rowptr), _ptr(c_colind), c_colind_cap,
                                          ctypes.byref(nr), ctypes.byref(na), ctypes.byref(cn), _stream(stream)),
           "mis2_coarsen_level_host")
    return nr.value, na.value, cn.value


def mis2_run_noalloc(g: mis2_csr, seed: int, in_set, roots, stream=None):
    """MIS-2 through the entry point that allocates nothing (for callers that
    cannot call cudaMalloc); graphs up to MIS2_NOALLOC_MAX_N vertices.
    Returns (n_roots, n_rounds)."""
    nr, rounds = ctypes.c_int64(0), ctypes.c_int32(0)
    _check(_lib().mis2_run_noalloc(ctypes.byref(g), seed, _ptr(in_set), _ptr(roots), ctypes.byref(nr),
                                   ctypes.byref(rounds), _stream(stream)), "mis2_run_noalloc")
    return nr.value, rounds.value


def mis2_status_string(status: int) -> str:
    return _lib().mis2_status_string(status).decode()


def mis2_version() -> str:
    return _lib().mis2_version().decode()


# --------------------------------------------------------------- conveniences
@dataclass
class DeviceGraph:
    """A CSR graph resident in device memory (torch tensors) and its C view."""

    n: int
    nnz: int
    rowptr: object
    colind: object

    @property
    def csr(self) -> mis2_csr:
        import torch

        return mis2_csr(self.n, self.nnz, 1 if self.rowptr.dtype == torch.int64 else 0, 0,
                        self.rowptr.data_ptr(), self.colind.data_ptr() if self.nnz > 0 else None)

    @staticmethod
    def from_host(g, device="cuda") -> "DeviceGraph":
        import torch

        rp = torch.from_numpy(np.ascontiguousarray(g.rowptr)).to(device)
        ci = torch.from_numpy(np.ascontiguousarray(g.colind, dtype=np.int32)).to(device)
        if ci.numel() == 0:
            ci = torch.zeros(4, dtype=torch.int32, device=device)
        return DeviceGraph(int(g.n), int(g.colind.shape[0]), rp, ci)


def host_csr(rowptr: np.ndarray, colind: np.ndarray, n: int) -> mis2_csr:
    return mis2_csr(n, int(colind.shape[0]), 1 if rowptr.dtype == np.int64 else 0, 0,
                    rowptr.ctypes.data, colind.ctypes.data if colind.shape[0] else None)


class Context:
    """Owns a mis2_ctx; methods allocate outputs as torch tensors."""

    def __init__(self, max_n: int, max_nnz: int, cfg: mis2_config | None = None, **overrides):
        cfg = cfg or mis2_config_default()
        for k, v in overrides.items():
            setattr(cfg, k, v)
        self.cfg = cfg
        self.max_n, self.max_nnz = max_n, max_nnz
        self.handle = mis2_ctx_create(max_n, max_nnz, cfg)

    def close(self):
        if self.handle:
            mis2_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def configure(self, **overrides):
        for k, v in overrides.items():
            setattr(self.cfg, k, v)
        mis2_ctx_set_config(self.handle, self.cfg)

    def stats(self) -> mis2_stats:
        return mis2_get_stats(self.handle)

    def run(self, dg: DeviceGraph, seed: int = 0, stream=None):
        import torch

        in_set = torch.empty(max(dg.n, 1), dtype=torch.uint8, device=dg.rowptr.device)
        roots = torch.empty(max(dg.n, 1), dtype=torch.int32, device=dg.rowptr.device)
        nr, rounds = mis2_run(self.handle, dg.csr, seed, in_set, roots, stream)
        return in_set[:dg.n], roots[:nr], rounds

    def run_with_priorities(self, dg: DeviceGraph, prio_table, stream=None):
        import torch

        in_set = torch.empty(max(dg.n, 1), dtype=torch.uint8, device=dg.rowptr.device)
        roots = torch.empty(max(dg.n, 1), dtype=torch.int32, device=dg.rowptr.device)
        nr, rounds = mis2_run_with_priorities(self.handle, dg.csr, prio_table, in_set, roots, stream)
        return in_set[:dg.n], roots[:nr], rounds

    def run_snapshots(self, dg: DeviceGraph, prio_table, snap_rounds: int, stream=None):
        """mis2_run_snapshots: (in_set, roots, rounds, snaps[snap_rounds, 3, n]) with snaps on the device."""
        import torch

        dev = dg.rowptr.device
        in_set = torch.empty(max(dg.n, 1), dtype=torch.uint8, device=dev)
        roots = torch.empty(max(dg.n, 1), dtype=torch.int32, device=dev)
        snaps = torch.empty(max(snap_rounds * 3 * dg.n, 1), dtype=torch.int32, device=dev)
        nr, rounds = mis2_run_snapshots(self.handle, dg.csr, prio_table, snaps, snap_rounds, in_set, roots, stream)
        return in_set[:dg.n], roots[:nr], rounds, snaps[:snap_rounds * 3 * dg.n].view(snap_rounds, 3, dg.n)

    def aggregate(self, dg: DeviceGraph, roots, seed: int = 0, mode: int = MIS2_AGG_ALG3, stream=None):
        import torch

        labels = torch.empty(max(dg.n, 1), dtype=torch.int32, device=dg.rowptr.device)
        na = mis2_aggregate(self.handle, dg.csr, roots, int(roots.numel()), seed, mode, labels, stream)
        return labels[:dg.n], na

    def run_k(self, dg: DeviceGraph, k: int, seed: int = 0, stream=None):
        import torch

        in_set = torch.empty(max(dg.n, 1), dtype=torch.uint8, device=dg.rowptr.device)
        roots = torch.empty(max(dg.n, 1), dtype=torch.int32, device=dg.rowptr.device)
        nr, rounds = mis2_run_k(self.handle, dg.csr, k, seed, in_set, roots, stream)
        return in_set[:dg.n], roots[:nr], rounds

    def color(self, dg: DeviceGraph, seed: int = 0, stream=None):
        """Returns (colors, color_ptr, color_list, n_rounds)."""
        import torch

        dev = dg.rowptr.device
        colors = torch.empty(max(dg.n, 1), dtype=torch.int32, device=dev)
        cptr = torch.empty(dg.n + 1, dtype=torch.int32, device=dev)
        clist = torch.empty(max(dg.n, 1), dtype=torch.int32, device=dev)
        nc, rounds = mis2_color(self.handle, dg.csr, seed, colors, cptr, clist, stream)
        return colors[:dg.n], cptr[:nc + 1], clist[:dg.n], rounds

    def cluster_lists(self, labels, n_aggs: int, stream=None):
        """Returns (c_ptr int32[n_aggs + 1], members int32[n])."""
        import torch

        n = int(labels.numel())
        c_ptr = torch.empty(n_aggs + 1, dtype=torch.int32, device=labels.device)
        members = torch.empty(max(n, 1), dtype=torch.int32, device=labels.device)
        mis2_cluster_lists(self.handle, labels, n, n_aggs, c_ptr, members, stream)
        return c_ptr, members[:n]

    def coarse_weights(self, dg: DeviceGraph, labels, n_aggs: int, c_rowptr, c_colind, stream=None):
        import torch

        w = torch.empty(max(int(c_colind.numel()), 1), dtype=torch.int32, device=dg.rowptr.device)
        mis2_coarse_weights(self.handle, dg.csr, labels, n_aggs, c_rowptr, c_colind, w, stream)
        return w[:int(c_colind.numel())]

    def prolongator(self, labels, n_aggs: int, normalize: bool = True, stream=None):
        import torch

        n = int(labels.numel())
        rp = torch.empty(n + 1, dtype=torch.int32, device=labels.device)
        pc = torch.empty(max(n, 1), dtype=torch.int32, device=labels.device)
        pv = torch.empty(max(n, 1), dtype=torch.float64, device=labels.device)
        mis2_tentative_prolongator(self.handle, labels, n, n_aggs, normalize, rp, pc, pv, stream)
        return rp, pc[:n], pv[:n]

    def coarsen(self, dg: DeviceGraph, labels, n_aggs: int, stream=None):
        import torch

        c_rowptr = torch.empty(n_aggs + 1, dtype=torch.int32, device=dg.rowptr.device)
        cap = max(dg.nnz, 1)
        c_colind = torch.empty(cap, dtype=torch.int32, device=dg.rowptr.device)
        cn = mis2_coarsen(self.handle, dg.csr, labels, n_aggs, c_rowptr, c_colind, cap, stream)
        return c_rowptr, c_colind[:cn]

    def coarsen_level(self, dg: DeviceGraph, seed: int = 0, stream=None):
        import torch

        dev = dg.rowptr.device
        in_set = torch.empty(max(dg.n, 1), dtype=torch.uint8, device=dev)
        roots = torch.empty(max(dg.n, 1), dtype=torch.int32, device=dev)
        labels = torch.empty(max(dg.n, 1), dtype=torch.int32, device=dev)
        c_rowptr = torch.empty(dg.n + 1, dtype=torch.int32, device=dev)
        cap = max(dg.nnz, 1)
        c_colind = torch.empty(cap, dtype=torch.int32, device=dev)
        nr, na, cn = mis2_coarsen_level(self.handle, dg.csr, seed, in_set, roots, labels, c_rowptr, c_colind, cap,
                                        stream)
        return dict(in_set=in_set[:dg.n], roots=roots[:nr], labels=labels[:dg.n], n_aggs=na,
                    c_rowptr=c_rowptr[:na + 1], c_colind=c_colind[:cn])


def mis2_run_k(ctx, g: mis2_csr, k: int, seed: int, in_set, roots, stream=None):
    """Returns (n_roots, n_rounds)."""
    nr, rounds = ctypes.c_int64(0), ctypes.c_int32(0)
    _check(_lib().mis2_run_k(ctx, ctypes.byref(g), k, seed, _ptr(in_set), _ptr(roots), ctypes.byref(nr),
                             ctypes.byref(rounds), _stream(stream)), "mis2_run_k")
    return nr.value, rounds.value


def mis2_color(ctx, g: mis2_csr, seed: int, colors, color_ptr, color_list, stream=None):
    """Returns (n_colors, n_rounds)."""
    nc, rounds = ctypes.c_int32(0), ctypes.c_int32(0)
    _check(_lib().mis2_color(ctx, ctypes.byref(g), seed, _ptr(colors), _ptr(color_ptr), _ptr(color_list),
                             ctypes.byref(nc), ctypes.byref(rounds), _stream(stream)), "mis2_color")
    return nc.value, rounds.value


def mis2_cluster_lists(ctx, labels, n: int, n_aggs: int, c_ptr, members, stream=None):
    _check(_lib().mis2_cluster_lists(ctx, _ptr(labels), n, n_aggs, _ptr(c_ptr), _ptr(members), _stream(stream)),
           "mis2_cluster_lists")


def mis2_coarse_weights(ctx, g: mis2_csr, labels, n_aggs: int, c_rowptr, c_colind, c_weights, stream=None):
    _check(_lib().mis2_coarse_weights(ctx, ctypes.byref(g), _ptr(labels), n_aggs, _ptr(c_rowptr), _ptr(c_colind),
                                      int(c_colind.numel()), _ptr(c_weights), _stream(stream)), "mis2_coarse_weights")


def mis2_tentative_prolongator(ctx, labels, n: int, n_aggs: int, normalize: bool, p_rowptr, p_colind, p_values,
                               stream=None):
    _check(_lib().mis2_tentative_prolongator(ctx, _ptr(labels), n, n_aggs, 1 if normalize else 0, _ptr(p_rowptr),
                                             _ptr(p_colind), _ptr(p_values), _stream(stream)),
           "mis2_tentative_prolongator")


# --------------------------------------------------------------- batches
def mis2_batch_create(max_graphs: int, max_total_n: int, max_total_nnz: int, cfg: mis2_config | None = None):
    h = ctypes.c_void_p()
    _check(_lib().mis2_batch_create(ctypes.byref(h), max_graphs, max_total_n, max_total_nnz,
                                    ctypes.byref(cfg) if cfg else None), "mis2_batch_create")
    return h


def mis2_batch_destroy(b) -> None:
    _check(_lib().mis2_batch_destroy(b), "mis2_batch_destroy")


def mis2_batch_coarsen(b, graphs, seed: int, min_n: int, max_levels: int, stream=None) -> int:
    arr = (mis2_csr * len(graphs))(*graphs)
    nl = ctypes.c_int32(0)
    _check(_lib().mis2_batch_coarsen(b, len(graphs), arr, seed, min_n, max_levels, ctypes.byref(nl),
                                     _stream(stream)), "mis2_batch_coarsen")
    return nl.value


def mis2_batch_level_sizes(b, level: int, n_graphs: int):
    """Returns (n, n_aggs, c_nnz) per graph at `level`."""
    n = np.zeros(n_graphs, np.int64)
    na = np.zeros(n_graphs, np.int64)
    cn = np.zeros(n_graphs, np.int64)
    _check(_lib().mis2_batch_level_sizes(b, level, _ptr(n), _ptr(na), _ptr(cn)), "mis2_batch_level_sizes")
    return n, na, cn


def mis2_batch_labels(b, level: int, graph: int, labels, stream=None) -> None:
    _check(_lib().mis2_batch_labels(b, level, graph, _ptr(labels), _stream(stream)), "mis2_batch_labels")


def mis2_batch_coarse(b, level: int, graph: int, c_rowptr, c_colind, c_colind_cap: int, stream=None) -> None:
    _check(_lib().mis2_batch_coarse(b, level, graph, _ptr(c_rowptr), _ptr(c_colind), c_colind_cap,
                                    _stream(stream)), "mis2_batch_coarse")


def mis2_batch_stats(b) -> mis2_stats:
    st = mis2_stats()
    _check(_lib().mis2_batch_stats(b, ctypes.byref(st)), "mis2_batch_stats")
    return st


class Batch:
    """Owns a mis2_batch: coarsen many graphs' hierarchies together."""

    def __init__(self, max_graphs: int, max_total_n: int, max_total_nnz: int, cfg: mis2_config | None = None,
                 **overrides):
        cfg = cfg or mis2_config_default()
        for k, v in overrides.items():
            setattr(cfg, k, v)
        self.cfg = cfg
        self.handle = mis2_batch_create(max_graphs, max_total_n, max_total_nnz, cfg)
        self.n_graphs = 0
        self.n_levels = 0

    def close(self):
        if self.handle:
            mis2_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def coarsen(self, dgraphs, seed: int = 0, min_n: int = 1000, max_levels: int = 32, stream=None) -> int:
        self._keep = dgraphs
        self.n_graphs = len(dgraphs)
        self.n_levels = mis2_batch_coarsen(self.handle, [d.csr for d in dgraphs], seed, min_n, max_levels, stream)
        return self.n_levels

    def level_sizes(self, level: int):
        return mis2_batch_level_sizes(self.handle, level, self.n_graphs)

    def labels(self, level: int, graph: int, device="cuda"):
        import torch

        n, _, _ = self.level_sizes(level)
        out = torch.empty(max(int(n[graph]), 1), dtype=torch.int32, device=device)
        mis2_batch_labels(self.handle, level, graph, out)
        return out[:int(n[graph])]

    def coarse(self, level: int, graph: int, device="cuda"):
        import torch

        n, na, cn = self.level_sizes(level)
        c_rowptr = torch.empty(int(na[graph]) + 1, dtype=torch.int32, device=device)
        cap = max(int(cn[graph]), 1)
        c_colind = torch.empty(cap, dtype=torch.int32, device=device)
        mis2_batch_coarse(self.handle, level, graph, c_rowptr, c_colind, cap)
        return c_rowptr, c_colind[:int(cn[graph])]

    def stats(self) -> mis2_stats:
        return mis2_batch_stats(self.handle)


# --------------------------------------------------------------- serving
def mis2_server_config_default() -> mis2_server_config:
    c = mis2_server_config()
    _lib().mis2_server_config_default(ctypes.byref(c))
    return c


def mis2_server_create(cfg: mis2_server_config):
    h = ctypes.c_void_p()
    _check(_lib().mis2_server_create(ctypes.byref(h), ctypes.byref(cfg)), "mis2_server_create")
    return h


def mis2_server_destroy(s) -> None:
    _check(_lib().mis2_server_destroy(s), "mis2_server_destroy")


def mis2_server_submit(s, g_host: mis2_csr, seed: int = 0) -> int:
    t = ctypes.c_int64(0)
    _check(_lib().mis2_server_submit(s, ctypes.byref(g_host), seed, ctypes.byref(t)), "mis2_server_submit")
    return t.value


def mis2_server_submit_out(s, g_host: mis2_csr, seed: int, out: mis2_request_out) -> int:
    t = ctypes.c_int64(0)
    _check(_lib().mis2_server_submit_out(s, ctypes.byref(g_host), seed, ctypes.byref(out), ctypes.byref(t)),
           "mis2_server_submit_out")
    return t.value


def mis2_server_wait(s, ticket: int) -> mis2_result:
    r = mis2_result()
    _check(_lib().mis2_server_wait(s, ticket, ctypes.byref(r)), "mis2_server_wait")
    return r


def mis2_server_cancel(s, ticket: int) -> bool:
    """True if the request was still queued and is now withdrawn."""
    c = ctypes.c_int32(0)
    _check(_lib().mis2_server_cancel(s, ticket, ctypes.byref(c)), "mis2_server_cancel")
    return bool(c.value)


def mis2_server_replay(s, pool, arrival_s, pool_index, seed: int = 0):
    """pool: list of host mis2_csr.  Returns (list of mis2_result, max in flight)."""
    arr = (mis2_csr * len(pool))(*pool)
    arrival = np.ascontiguousarray(arrival_s, dtype=np.float64)
    idx = np.ascontiguousarray(pool_index, dtype=np.int32)
    res = (mis2_result * len(arrival))()
    mif = ctypes.c_int64(0)
    _check(_lib().mis2_server_replay(s, len(pool), arr, len(arrival), _ptr(arrival), _ptr(idx), seed, res,
                                     ctypes.byref(mif)), "mis2_server_replay")
    return list(res), mif.value


class Server:
    """Owns a mis2_server (continuous-batching request loop)."""

    def __init__(self, slots=4, mem_budget=8 << 30, slot_max_n=1 << 22, slot_max_nnz=1 << 25, batch_max=0,
                 **cfg_overrides):
        c = mis2_server_config_default()
        c.slots, c.mem_budget, c.slot_max_n, c.slot_max_nnz = slots, mem_budget, slot_max_n, slot_max_nnz
        c.batch_max = batch_max
        for k, v in cfg_overrides.items():
            setattr(c.cfg, k, v)
        self.cfg = c
        self.handle = mis2_server_create(c)

    def close(self):
        if self.handle:
            mis2_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def replay(self, pool_host, arrival_s, pool_index, seed: int = 0):
        return mis2_server_replay(self.handle, pool_host, arrival_s, pool_index, seed)

    def submit(self, g_host: mis2_csr, seed: int = 0) -> int:
        """Queue one request (g_host must stay valid until it completes)."""
        return mis2_server_submit(self.handle, g_host, seed)

    def submit_out(self, g_host: mis2_csr, n: int, nnz: int, seed: int = 0):
        """Queue one request whose results are written to fresh numpy arrays:
        returns (ticket, arrays dict: in_set, roots, labels, c_rowptr, c_colind;
        valid once wait(ticket) returns, trimmed with the result's counts)."""
        bufs = {"in_set": np.zeros(max(n, 1), np.uint8), "roots": np.zeros(max(n, 1), np.int32),
                "labels": np.zeros(max(n, 1), np.int32), "c_rowptr": np.zeros(n + 1, np.int32),
                "c_colind": np.zeros(max(nnz, 1), np.int32)}
        out = mis2_request_out(*(b.ctypes.data for b in bufs.values()), max(nnz, 1))
        t = mis2_server_submit_out(self.handle, g_host, seed, out)
        return t, bufs

    def wait(self, ticket: int) -> mis2_result:
        return mis2_server_wait(self.handle, ticket)

    def cancel(self, ticket: int) -> bool:
        return mis2_server_cancel(self.handle, ticket)
