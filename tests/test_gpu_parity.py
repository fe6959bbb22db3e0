"""Bit-exact parity of the CUDA library (through the C ABI) with the CPU
oracle: MIS-2 flags, roots, round counts and per-round worklist traces,
aggregate labels and the coarse CSR, on seeded graphs shaped like the
workloads, edge cases, and every row mapping / loop driver."""
import itertools
import json
import os

import numpy as np
import pytest

import oracle
from paper_2204_02934_gb300 import graphgen as gg
from paper_2204_02934_gb300 import mis2
from _gpu import assert_level_equal, gpu_level, make_ctx

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
LOOPS = [mis2.MIS2_LOOP_HOST, mis2.MIS2_LOOP_DEVICE]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2204_02934_gb300 import _build

    _build.build()


@pytest.mark.parametrize("loop", LOOPS)
def test_fig1_worked_example_on_gpu(loop):
    """Section III-A, Fig. 1 through the priority-injection hook."""
    fx = json.load(open(os.path.join(GOLDEN, "fig1.json")))
    n = fx["n"]
    g = gg.graph_from_edges(n, [(a - 1, b - 1) for a, b in fx["edges"]])
    tab = np.zeros((len(fx["rounds"]), n), dtype=np.uint32)
    for r, rd in enumerate(fx["rounds"]):
        for vid, p in rd["priorities"].items():
            tab[r, int(vid) - 1] = p
    ctx = make_ctx(g, loop=loop)
    in_set, roots, rounds = ctx.run_with_priorities(mis2.DeviceGraph.from_host(g), tab)
    assert (roots.cpu().numpy() + 1).tolist() == fx["result"]
    assert rounds == fx["n_rounds"]


def _unpack(t, b):
    if t == 0:
        return "IN"
    if t == 0xFFFFFFFF:
        return "OUT"
    return [t >> b, t & ((1 << b) - 1)]


@pytest.mark.parametrize("loop", LOOPS)
def test_fig1_round_by_round_on_gpu(loop):
    """Fig. 1 step by step: the injected priorities after each row refresh,
    the column tuples M after each column step and the decisions after each
    decide step, as the figure prints them (tests/golden/fig1.json)."""
    fx = json.load(open(os.path.join(GOLDEN, "fig1.json")))
    n = fx["n"]
    g = gg.graph_from_edges(n, [(a - 1, b - 1) for a, b in fx["edges"]])
    tab = np.zeros((len(fx["rounds"]), n), dtype=np.uint32)
    for r, rd in enumerate(fx["rounds"]):
        for vid, p in rd["priorities"].items():
            tab[r, int(vid) - 1] = p
    ctx = make_ctx(g, loop=loop)
    in_set, roots, rounds, snaps = ctx.run_snapshots(mis2.DeviceGraph.from_host(g), tab, 4)
    snaps = snaps.cpu().numpy().view(np.uint32)
    b = oracle.id_bits(n)
    assert b == 3 and rounds == fx["n_rounds"]
    assert (roots.cpu().numpy() + 1).tolist() == fx["result"]
    for r, rd in enumerate(fx["rounds"]):
        T0, M, T1 = snaps[r]
        for vid, p in rd["priorities"].items():
            assert _unpack(int(T0[int(vid) - 1]), b) == [p, int(vid)], (r, vid)
        for vid, m in rd["column"].items():
            assert _unpack(int(M[int(vid) - 1]), b) == m, (r, vid)
        for vid, d in rd["decide"].items():
            got = _unpack(int(T1[int(vid) - 1]), b)
            assert (got if isinstance(got, str) else "U") == d, (r, vid)
    assert (snaps[len(fx["rounds"]):] == 0xFFFFFFFF).all()  # rounds that did not run


@pytest.mark.parametrize("loop", LOOPS)
def test_snapshots_equal_the_oracle_round_by_round(loop):
    """On hashed priorities (no table) the GPU's per-round T after the
    refresh and M after the column step equal the oracle's exactly, and the
    decisions agree as IN / OUT / undecided."""
    g = gg.random_graph(60, 0.08, 4)
    ctx = make_ctx(g, loop=loop)
    _, roots, rounds, snaps = ctx.run_snapshots(mis2.DeviceGraph.from_host(g), np.zeros((0, g.n), np.uint32), 8)
    snaps = snaps.cpu().numpy().view(np.uint32)
    ref = oracle.mis2(g, 0, snap_cap=8)
    assert rounds == ref[2] and np.array_equal(roots.cpu().numpy(), ref[1])
    status = lambda t: np.where(t == 0, 0, np.where(t == 0xFFFFFFFF, 2, 1))
    for r in range(min(rounds, 8)):
        T0, M, T1 = snaps[r]
        oT0, oM, oT1 = ref[4][r]
        assert np.array_equal(T0, oT0), r
        assert np.array_equal(M, oM), r
        assert np.array_equal(status(T1), status(oT1)), r


def _edges_of(n, mask):
    pairs = list(itertools.combinations(range(n), 2))
    return [p for k, p in enumerate(pairs) if (mask >> k) & 1]


@pytest.mark.parametrize("loop", LOOPS)
def test_exhaustive_small_graphs(loop):
    """Every labelled graph on 5 vertices, both aggregation modes."""
    n = 5
    ctxs = {m: mis2.Context(8, 32, loop=loop, agg_mode=m) for m in (0, 1)}
    for mask in range(1 << 10):
        g = gg.graph_from_edges(n, _edges_of(n, mask))
        for mode in (0, 1):
            assert_level_equal(g, gpu_level(ctxs[mode], g, seed=mask), seed=mask, mode=mode)


def _graphs():
    yield "gnp200", gg.random_graph(200, 0.03, 1)
    yield "gnp500", gg.random_graph(500, 0.01, 2)
    yield "grid2d_37x29", gg.grid2d_5pt(37, 29)
    yield "grid3d7_13", gg.grid3d_7pt(13, 11, 9)
    yield "grid3d27_17", gg.grid3d_27pt(17, 15, 13)
    yield "rgg3000", gg.rgg2d(3000, 10.0, 4)
    yield "rmat12", gg.rmat(12, 8, seed=5)
    yield "rmat12_i32", gg.rmat(12, 8, seed=6, rowptr_dtype=np.int32)
    yield "elasticity5", gg.elasticity3d(5, 4, 3)
    yield "grid_hubs", _grid_with_hubs()


def _grid_with_hubs():
    """A 120x120 grid plus three hubs tied to spread-out grid vertices: the
    hubs' aggregates border hundreds of aggregates, so the coarse rows take
    the large-aggregate (global bitmap) path."""
    side = 120
    base = gg.grid2d_5pt(side, side)
    pairs = gg_pairs(base)
    n = base.n + 3
    extra = [(base.n + h, v) for h in range(3) for v in range(h * 7, base.n, 11)]
    return gg.graph_from_edges(n, np.concatenate([pairs, np.array(extra, dtype=np.int64)]))


def gg_pairs(g):
    rows = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(g.rowptr.astype(np.int64)))
    keep = rows < g.colind
    return np.stack([rows[keep], g.colind[keep].astype(np.int64)], axis=1)


@pytest.mark.parametrize("loop", LOOPS)
@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("name,g", list(_graphs()))
def test_parity_graphs(name, g, mode, loop):
    ctx = make_ctx(g, loop=loop, agg_mode=mode)
    for seed in (0, 7):
        assert_level_equal(g, gpu_level(ctx, g, seed), seed=seed, mode=mode)


@pytest.mark.parametrize("lanes", [1, 2, 4, 8, 16, 32])
@pytest.mark.parametrize("loop", LOOPS)
def test_every_row_mapping(lanes, loop):
    """Group sizes, warp rows and block rows all give the same bits: low
    thresholds push rows of the R-MAT graph into every class."""
    g = gg.rmat(11, 8, seed=9)
    ctx = make_ctx(g, loop=loop, group_lanes=lanes, warp_degree=8, block_degree=64)
    assert_level_equal(g, gpu_level(ctx, g, 3), seed=3)


@pytest.mark.parametrize("variant", [0, 1, 2])
def test_hash_variants(variant):
    g = gg.grid3d_7pt(12, 12, 12)
    ctx = make_ctx(g, hash_variant=variant)
    lv = oracle.coarsen_level(g, seed=0, hash_variant=variant, trace_cap=mis2.MIS2_TRACE_CAP)
    out = gpu_level(ctx, g, 0)
    assert np.array_equal(out["roots"], lv.roots) and out["rounds"] == lv.rounds
    assert np.array_equal(out["labels"], lv.labels)


@pytest.mark.parametrize("loop", LOOPS)
def test_edge_cases(loop):
    cases = [
        gg.graph_from_edges(1, []),
        gg.graph_from_edges(7, []),                                   # isolated vertices
        gg.graph_from_edges(2, [(0, 1)]),
        gg.graph_from_edges(9, list(itertools.combinations(range(9), 2))),  # clique
        gg.graph_from_edges(300, [(i, i + 1) for i in range(299)]),   # path
        gg.graph_from_edges(5000, [(0, i) for i in range(1, 5000)]),  # star: one block row
        gg.graph_from_edges(40, [(0, i) for i in range(1, 20)] + [(20, i) for i in range(21, 40)] + [(5, 25)]),
    ]
    for g in cases:
        ctx = make_ctx(g, loop=loop, block_degree=1024, warp_degree=16)
        assert_level_equal(g, gpu_level(ctx, g, 1), seed=1)


def test_empty_graph():
    g = gg.graph_from_edges(0, [])
    ctx = mis2.Context(1, 1)
    dg = mis2.DeviceGraph.from_host(g)
    in_set, roots, rounds = ctx.run(dg)
    assert roots.numel() == 0 and rounds == 0


def _with_extra_entries(g, duplicates):
    rp = g.rowptr.astype(np.int64)
    rows, cols = [], []
    for v in range(g.n):
        row = list(g.colind[rp[v]:rp[v + 1]])
        cs = row + [v] + (row[:1] if duplicates else [])
        rows.append(len(cs))
        cols.extend(cs)
    rp2 = np.concatenate([[0], np.cumsum(rows)]).astype(np.int64)
    return gg.CSRGraph(g.n, rp2, np.asarray(cols, dtype=np.int32))


def test_self_loops_duplicates_and_unaligned_colind():
    """Stored diagonals (and, for MIS-2, duplicate entries) change nothing; a
    colind that is only 4-byte aligned takes the scalar-load path with the
    same result."""
    import torch

    base = gg.random_graph(300, 0.02, 8)
    for dup in (False, True):
        g2 = _with_extra_entries(base, dup)
        ctx = make_ctx(g2)
        buf = torch.zeros(g2.nnz + 1, dtype=torch.int32, device="cuda")
        buf[1:] = torch.from_numpy(g2.colind).cuda()
        dg = mis2.DeviceGraph(g2.n, g2.nnz, torch.from_numpy(g2.rowptr).cuda(), buf[1:])
        in_set, roots, rounds = ctx.run(dg, 2)
        ref = oracle.mis2(g2, seed=2)
        assert np.array_equal(roots.cpu().numpy(), ref[1]) and rounds == ref[2]
        if not dup:
            out = ctx.coarsen_level(dg, 2)
            lv = oracle.coarsen_level(g2, seed=2)
            assert np.array_equal(out["labels"].cpu().numpy(), lv.labels)
            assert np.array_equal(out["c_colind"].cpu().numpy(), lv.c_colind)


def test_separate_calls_match_level_call():
    """mis2_run -> mis2_aggregate -> mis2_coarsen equals mis2_coarsen_level."""
    g = gg.grid3d_27pt(20, 18, 16)
    ctx = make_ctx(g)
    dg = mis2.DeviceGraph.from_host(g)
    in_set, roots, rounds = ctx.run(dg, 5)
    labels, na = ctx.aggregate(dg, roots, 5)
    c_rowptr, c_colind = ctx.coarsen(dg, labels, na)
    ref = oracle.coarsen_level(g, seed=5)
    assert np.array_equal(roots.cpu().numpy(), ref.roots)
    assert np.array_equal(labels.cpu().numpy(), ref.labels)
    assert np.array_equal(c_colind.cpu().numpy(), ref.c_colind)


def test_host_buffer_entry_point():
    g = gg.grid3d_7pt(30, 30, 30)
    ctx = make_ctx(g)
    n = g.n
    in_set = np.zeros(n, np.uint8)
    roots = np.zeros(n, np.int32)
    labels = np.zeros(n, np.int32)
    c_rowptr = np.zeros(n + 1, np.int32)
    c_colind = np.zeros(g.nnz, np.int32)
    rp = np.ascontiguousarray(g.rowptr)
    ci = np.ascontiguousarray(g.colind)
    nr, na, cn = mis2.mis2_coarsen_level_host(ctx.handle, mis2.host_csr(rp, ci, n), 3, in_set, roots, labels,
                                              c_rowptr, c_colind, g.nnz)
    ref = oracle.coarsen_level(g, seed=3)
    assert np.array_equal(roots[:nr], ref.roots) and np.array_equal(labels, ref.labels)
    assert np.array_equal(c_rowptr[:na + 1].astype(np.int64), ref.c_rowptr)
    assert np.array_equal(c_colind[:cn], ref.c_colind)


def test_determinism_and_loop_drivers_agree():
    g = gg.rmat(13, 8, seed=2)
    outs = []
    for loop in LOOPS * 2:
        ctx = make_ctx(g, loop=loop)
        outs.append(gpu_level(ctx, g, 11))
    for o in outs[1:]:
        for k in ("labels", "c_colind", "roots"):
            assert np.array_equal(o[k], outs[0][k])


@pytest.mark.parametrize("loop", LOOPS)
def test_coarse_capacity_is_checked(loop):
    """Too small a coarse colind buffer is refused (nothing written past it),
    and the next call on the same context is unaffected."""
    import torch

    g = gg.grid3d_27pt(12, 11, 10)
    ctx = make_ctx(g, loop=loop)
    dg = mis2.DeviceGraph.from_host(g)
    n = g.n
    bufs = [torch.empty(n, dtype=t, device="cuda") for t in (torch.uint8, torch.int32, torch.int32)]
    c_rowptr = torch.empty(n + 1, dtype=torch.int32, device="cuda")
    cap = 64
    c_colind = torch.full((cap + 1024,), -7, dtype=torch.int32, device="cuda")
    with pytest.raises(mis2.Mis2Error) as e:
        mis2.mis2_coarsen_level(ctx.handle, dg.csr, 0, *bufs, c_rowptr, c_colind, cap, None)
    assert e.value.status == -1
    assert bool((c_colind[cap:] == -7).all())
    assert_level_equal(g, gpu_level(ctx, g, 0), seed=0)


@pytest.mark.parametrize("loop", LOOPS)
def test_no_worklist_ablation_gives_the_same_result(loop):
    """Visiting every vertex every round (Fig. 2's variant without worklists)
    leaves the MIS-2, the round count, the aggregates and the coarse graph
    unchanged; only the per-round statistics (vertices visited) differ."""
    for g in (gg.grid3d_7pt(21, 19, 17), gg.elasticity3d(6, 5, 4), gg.rmat(11, 8, seed=4), gg.grid2d_5pt(1, 1)):
        ctx = make_ctx(g, loop=loop, ablation=mis2.MIS2_ABLATE_NO_WORKLISTS)
        out = gpu_level(ctx, g, 2)
        lv = oracle.coarsen_level(g, seed=2)
        assert np.array_equal(out["in_set"], lv.in_set) and np.array_equal(out["roots"], lv.roots)
        assert out["rounds"] == lv.rounds and out["rounds2"] == lv.rounds2
        assert np.array_equal(out["labels"], lv.labels)
        assert np.array_equal(out["c_colind"], lv.c_colind)
        if out["rounds"] > 1:
            assert int(out["trace"][1][1]) == g.n  # every vertex visited again


def test_invalid_arguments():
    g = gg.grid2d_5pt(10, 10)
    ctx = make_ctx(g)
    big = gg.grid2d_5pt(20, 20)
    dg = mis2.DeviceGraph.from_host(big)
    with pytest.raises(mis2.Mis2Error) as e:
        ctx.run(dg)
    assert e.value.status == -2  # larger than the context
    with pytest.raises(mis2.Mis2Error):
        mis2.Context(10, 10, group_lanes=3)


# ---------------------------------------------------------------- workloads
@pytest.mark.parametrize("loop", LOOPS)
def test_workload_small_5pt_100x100(loop):
    g = gg.workload_small()
    assert g.n == 10_000 and g.nnz == 39_600
    ctx = make_ctx(g, loop=loop)
    assert_level_equal(g, gpu_level(ctx, g, 0), seed=0)


@pytest.mark.parametrize("loop", LOOPS)
def test_workload_27pt_100(loop):
    g = gg.workload_27pt(100)
    assert g.nnz == 25_463_592
    ctx = make_ctx(g, loop=loop)
    assert_level_equal(g, gpu_level(ctx, g, 0), seed=0)


def test_workload_rmat_scale22():
    g = gg.workload_rmat(22)
    assert g.rowptr.dtype == np.int64
    ctx = make_ctx(g, loop=mis2.MIS2_LOOP_DEVICE)
    assert_level_equal(g, gpu_level(ctx, g, 0), seed=0)


def test_overlapped_and_serial_launches_agree():
    """Programmatic dependent launch (default), serial launches and both
    timing modes give the same level, equal to the oracle's, and the same
    full statistics traces, on back-to-back calls of one context."""
    graphs = [gg.grid3d_27pt(30, 30, 30), gg.rmat(13, 8, seed=3)]
    ref = {}
    for serial in (0, 1):
        for timing in (mis2.MIS2_TIMING_OFF, mis2.MIS2_TIMING_ALL, mis2.MIS2_TIMING_LOOP):
            ctx = mis2.Context(max(g.n for g in graphs), max(g.nnz for g in graphs), loop=mis2.MIS2_LOOP_DEVICE,
                               serial_launches=serial, timing=timing)
            for gi, g in enumerate(graphs):
                for rep in range(2):
                    out = gpu_level(ctx, g, 5)
                    st = ctx.stats()
                    full = (np.array(st.trace, dtype=np.int64), np.array(st.trace2, dtype=np.int64))
                    if gi not in ref:
                        assert_level_equal(g, out, seed=5)
                        ref[gi] = (out, full)
                    o0, f0 = ref[gi]
                    for k in ("in_set", "roots", "labels", "c_rowptr", "c_colind"):
                        assert np.array_equal(out[k], o0[k]), (serial, timing, gi, k)
                    assert np.array_equal(full[0], f0[0]) and np.array_equal(full[1], f0[1])
                    assert not full[0][out["rounds"]:].any() and not full[1][out["rounds2"]:].any()
            ctx.close()


def test_timing_loop_mode_brackets_the_loop_alone():
    g = gg.grid3d_27pt(24, 24, 24)
    ctx = mis2.Context(g.n, g.nnz, loop=mis2.MIS2_LOOP_DEVICE, timing=mis2.MIS2_TIMING_LOOP)
    gpu_level(ctx, g, 0)
    st = ctx.stats()
    names = mis2.KERNEL_CLASSES
    loop = names.index("device_loop")
    assert st.kernel_ms[loop] > 0 and st.kernel_launches[loop] == 2
    assert all(st.kernel_ms[k] == 0 for k in range(len(names)) if k != loop)
    ctx.configure(timing=mis2.MIS2_TIMING_ALL)
    gpu_level(ctx, g, 0)
    st = ctx.stats()
    assert st.kernel_ms[names.index("aggregate")] > 0 and st.kernel_ms[names.index("coarse")] > 0
    with pytest.raises(mis2.Mis2Error):
        ctx.configure(timing=3)
    ctx.close()


def _hub_leftover_graph():
    """A 160x160 grid plus hubs of 40, 600 and 9,000 neighbours, and roots
    chosen (greedily, more than two hops apart in the whole graph) among the
    grid vertices no hub touches: the hubs are phase-3 leftovers of every row
    class (a warp with a hash table, a block sort, the block windows above
    8,192 entries)."""
    side = 160
    base = gg.grid2d_5pt(side, side)
    pairs = [gg_pairs(base)]
    degs = (40, 600, 9000)
    for h, d in enumerate(degs):
        nb = (np.arange(d, dtype=np.int64) * (base.n // d) + 17 * h) % base.n
        pairs.append(np.stack([np.full(d, base.n + h, dtype=np.int64), nb], axis=1))
    g = gg.graph_from_edges(base.n + len(degs), np.concatenate(pairs))
    rp, ci = g.rowptr.astype(np.int64), g.colind
    touched = np.zeros(g.n, dtype=bool)
    touched[base.n:] = True
    touched[ci[rp[base.n]:]] = True
    blocked = np.zeros(g.n, dtype=bool)
    roots = []
    for v in range(base.n):
        if touched[v] or blocked[v]:
            continue
        roots.append(v)
        ring = ci[rp[v]:rp[v + 1]]
        two = np.concatenate([ci[rp[w]:rp[w + 1]] for w in ring] + [ring, [v]])
        blocked[two] = True  # anything within two hops of a root is not a root
        for w in ring:  # ... and within two hops of those: keeps roots > 2 apart
            blocked[ci[rp[w]:rp[w + 1]]] = True
    return g, np.array(roots, dtype=np.int32)


@pytest.mark.parametrize("mode", [0, 1])
def test_phase3_rows_of_every_class_match_the_oracle(mode):
    import torch

    g, roots = _hub_leftover_graph()
    in_set = np.zeros(g.n, dtype=np.uint8)
    in_set[roots] = 1
    ref_labels, ref_na = oracle.aggregate(g, in_set, seed=3, mode=mode)[:2]
    assert (ref_labels[-3:] >= 0).all()
    ctx = make_ctx(g, loop=mis2.MIS2_LOOP_DEVICE, debug_checks=mis2.MIS2_DEBUG_VALIDATE)
    dg = mis2.DeviceGraph.from_host(g)
    labels, na = ctx.aggregate(dg, torch.from_numpy(roots).to(dg.rowptr.device), seed=3, mode=mode)
    assert na == ref_na
    assert np.array_equal(labels.cpu().numpy(), ref_labels)
    ctx.close()
