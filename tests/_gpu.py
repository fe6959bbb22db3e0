"""Helpers for the GPU parity tests: run the CUDA library through the C ABI
and the oracle on the same seeded graph, return numpy arrays."""
import numpy as np

import oracle
from paper_2204_02934_gb300 import mis2


def gpu_available():
    try:
        import torch

        return torch.cuda.is_available()
    except Exception:
        return False


def make_ctx(g, **cfg):
    return mis2.Context(max(g.n, 1), max(g.nnz, 1), **cfg)


def gpu_level(ctx, g, seed=0):
    dg = mis2.DeviceGraph.from_host(g)
    out = ctx.coarsen_level(dg, seed)
    st = ctx.stats()
    res = {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in out.items()}
    res["rounds"] = st.rounds
    res["rounds2"] = st.rounds2
    res["n_phase1"] = st.n_phase1
    res["trace"] = np.array(st.trace, dtype=np.int64)[:min(st.rounds, mis2.MIS2_TRACE_CAP)]
    res["trace2"] = np.array(st.trace2, dtype=np.int64)[:min(st.rounds2, mis2.MIS2_TRACE_CAP)]
    return res


def assert_level_equal(g, gpu, seed=0, mode=0, hash_variant=0):
    lv = oracle.coarsen_level(g, seed=seed, mode=mode, hash_variant=hash_variant, trace_cap=mis2.MIS2_TRACE_CAP)
    assert np.array_equal(gpu["in_set"], lv.in_set), "in_set differs"
    assert np.array_equal(gpu["roots"], lv.roots), "roots differ"
    assert gpu["rounds"] == lv.rounds, (gpu["rounds"], lv.rounds)
    assert np.array_equal(gpu["trace"], lv.trace), "phase-1 worklist trace differs"
    assert gpu["n_phase1"] == lv.n_phase1
    assert gpu["rounds2"] == lv.rounds2, (gpu["rounds2"], lv.rounds2)
    if mode == 0:
        assert np.array_equal(gpu["trace2"], lv.trace2), "phase-2 worklist trace differs"
    assert gpu["n_aggs"] == lv.n_aggs
    assert np.array_equal(gpu["labels"], lv.labels), "labels differ"
    assert np.array_equal(gpu["c_rowptr"].astype(np.int64), lv.c_rowptr), "coarse rowptr differs"
    assert np.array_equal(gpu["c_colind"], lv.c_colind), "coarse colind differs"
    return lv


def hub_graph(side=100, hubs=4, stride=3):
    """A side x side 5-point grid plus `hubs` hub vertices, hub h tied to
    every stride-th grid vertex from h on and to the other hubs: rows of a
    few thousand entries, next to each other, among short grid rows."""
    from paper_2204_02934_gb300 import graphgen as gg

    base = gg.grid2d_5pt(side, side)
    rows = np.repeat(np.arange(base.n, dtype=np.int64), np.diff(base.rowptr.astype(np.int64)))
    keep = rows < base.colind
    pairs = [np.stack([rows[keep], base.colind[keep].astype(np.int64)], axis=1)]
    for h in range(hubs):
        grid_v = np.arange(h, base.n, stride, dtype=np.int64)
        pairs.append(np.stack([np.full_like(grid_v, base.n + h), grid_v], axis=1))
        pairs.append(np.array([[base.n + h, base.n + o] for o in range(h + 1, hubs)], dtype=np.int64).reshape(-1, 2))
    return gg.graph_from_edges(base.n + hubs, np.concatenate(pairs))
