"""Coarse edge weights and the tentative prolongator (the Galerkin pieces
after the coarse graph) against the oracle, bit for bit, on the workload
shapes, including a skewed graph whose hub aggregates take the bitmap path
and the full-size 27-point level."""
import numpy as np
import pytest

import oracle
from paper_2204_02934_gb300 import graphgen as gg
from paper_2204_02934_gb300 import mis2
from _gpu import hub_graph, make_ctx

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2204_02934_gb300 import _build

    _build.build()


def _graphs():
    yield "grid2d", gg.grid2d_5pt(37, 29)
    yield "grid3d27", gg.grid3d_27pt(17, 15, 13)
    yield "elasticity", gg.elasticity3d(6, 5, 4)
    yield "rmat12", gg.rmat(12, 8, seed=5)
    yield "rgg", gg.rgg2d(3000, 10.0, 4)
    yield "single", gg.grid2d_5pt(1, 1)
    yield "hubs", hub_graph()  # long rows split over many entry chunks
    # runs of empty rows between short ones: entry chunks span many rows
    yield "isolated", gg.graph_from_edges(3000, [(0, 1), (1, 2), (10, 2900), (2900, 2901)] +
                                          [(v, v + 1) for v in range(500, 2400) if v % 50])


@pytest.mark.parametrize("name,g", list(_graphs()))
def test_weights_and_prolongator_match_the_oracle(name, g):
    ctx = make_ctx(g, loop=mis2.MIS2_LOOP_DEVICE)
    dg = mis2.DeviceGraph.from_host(g)
    out = ctx.coarsen_level(dg, 3)
    lv = oracle.coarsen_level(g, seed=3)
    assert np.array_equal(out["labels"].cpu().numpy(), lv.labels)
    w = ctx.coarse_weights(dg, out["labels"], out["n_aggs"], out["c_rowptr"], out["c_colind"])
    w_ref = oracle.coarse_weights(g, lv.labels, lv.n_aggs, lv.c_rowptr, lv.c_colind)
    assert np.array_equal(w.cpu().numpy().astype(np.int64), w_ref)
    for normalize in (False, True):
        rp, pc, pv = ctx.prolongator(out["labels"], out["n_aggs"], normalize)
        pc_ref, pv_ref = oracle.prolongator(lv.labels, lv.n_aggs, normalize)
        assert np.array_equal(rp.cpu().numpy(), np.arange(g.n + 1))
        assert np.array_equal(pc.cpu().numpy(), pc_ref)
        assert np.array_equal(pv.cpu().numpy().view(np.uint64), pv_ref.view(np.uint64))  # bit-exact doubles


def test_weights_on_the_27_point_workload():
    g = gg.workload_27pt(100)
    ctx = make_ctx(g, loop=mis2.MIS2_LOOP_DEVICE)
    dg = mis2.DeviceGraph.from_host(g)
    out = ctx.coarsen_level(dg, 0)
    w = ctx.coarse_weights(dg, out["labels"], out["n_aggs"], out["c_rowptr"], out["c_colind"]).cpu().numpy()
    labels = out["labels"].cpu().numpy()
    rows = np.repeat(np.arange(g.n), np.diff(g.rowptr))
    crossing = int(np.sum(labels[rows] != labels[g.colind]))
    assert int(w.astype(np.int64).sum()) == crossing and (w >= 1).all()
    # symmetric: the weight of (A, B) equals that of (B, A)
    crp = out["c_rowptr"].cpu().numpy().astype(np.int64)
    cci = out["c_colind"].cpu().numpy()
    crow = np.repeat(np.arange(out["n_aggs"]), np.diff(crp))
    key = crow.astype(np.int64) * out["n_aggs"] + cci
    mirror = cci.astype(np.int64) * out["n_aggs"] + crow
    order = np.argsort(key)
    pos = np.searchsorted(key[order], mirror)
    assert np.array_equal(w[order][pos], w)


def test_weights_refuse_a_foreign_coarse_graph():
    import torch

    g = gg.grid2d_5pt(12, 12)
    ctx = make_ctx(g)
    dg = mis2.DeviceGraph.from_host(g)
    out = ctx.coarsen_level(dg, 0)
    empty_rowptr = torch.zeros(out["n_aggs"] + 1, dtype=torch.int32, device="cuda")
    with pytest.raises(mis2.Mis2Error) as e:
        ctx.coarse_weights(dg, out["labels"], out["n_aggs"], empty_rowptr, out["c_colind"][:0])
    assert e.value.status == -4
