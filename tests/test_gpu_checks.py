"""Debug-mode input checks and the bounded-wait failure path.

Every malformed input here stays inside the buffers the library allocated
(contexts are made larger than the graph, bad column ids point one past the
last vertex), so a check that failed to fire could not make a kernel touch
memory outside its allocations.  The forced timeout is the designed bounded
wait: the device loop's barriers wait for an arrival that never comes, every
block gives up after a few thousand polls, the call reports
MIS2_ERR_TIMEOUT and the context keeps working."""
import numpy as np
import pytest

from paper_2204_02934_gb300 import graphgen as gg
from paper_2204_02934_gb300 import mis2
from _gpu import assert_level_equal, gpu_level

pytestmark = pytest.mark.gpu
BAD_GRAPH, TIMEOUT = -4, -5


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2204_02934_gb300 import _build

    _build.build()


def _ctx(g, **cfg):
    return mis2.Context(g.n + 64, g.nnz + 64, **cfg)


def _device(rowptr, colind, n):
    import torch

    rp = torch.from_numpy(np.ascontiguousarray(rowptr)).cuda()
    ci = torch.from_numpy(np.ascontiguousarray(colind, dtype=np.int32)).cuda()
    return mis2.DeviceGraph(n, int(colind.shape[0]), rp, ci)


@pytest.mark.parametrize("loop", [mis2.MIS2_LOOP_HOST, mis2.MIS2_LOOP_DEVICE])
def test_valid_graphs_pass_the_checks(loop):
    for g in (gg.grid3d_27pt(12, 11, 10), gg.rmat(11, 8, seed=3), gg.grid2d_5pt(30, 29)):
        ctx = _ctx(g, loop=loop, debug_checks=mis2.MIS2_DEBUG_VALIDATE)
        assert_level_equal(g, gpu_level(ctx, g, 0), seed=0)


def test_malformed_csr_is_refused():
    g = gg.grid2d_5pt(20, 20)
    ctx = _ctx(g, debug_checks=mis2.MIS2_DEBUG_VALIDATE)
    rp = g.rowptr.copy()
    rp[5], rp[6] = rp[6], rp[5]  # non-decreasing order broken, values still in [0, nnz]
    cases = [(rp, g.colind)]
    ci = g.colind.copy()
    ci[17] = g.n  # one past the last vertex
    cases.append((g.rowptr, ci))
    rp_end = g.rowptr.copy()
    rp_end[-1] -= 1  # last offset is not nnz
    cases.append((rp_end, g.colind))
    for rowptr, colind in cases:
        dg = _device(rowptr, colind, g.n)
        with pytest.raises(mis2.Mis2Error) as e:
            ctx.run(dg)
        assert e.value.status == BAD_GRAPH
        with pytest.raises(mis2.Mis2Error) as e:
            ctx.coarsen_level(dg)
        assert e.value.status == BAD_GRAPH


def test_asymmetric_graph_is_refused():
    g = gg.grid2d_5pt(16, 16)
    # drop the mirror of one edge: v -> w stays, w -> v goes (w's row keeps
    # its length through a self-loop, which the checks and the method allow)
    v = 40
    w = int(g.colind[g.rowptr[v]])
    ci = g.colind.copy()
    s, e = int(g.rowptr[w]), int(g.rowptr[w + 1])
    k = s + int(np.flatnonzero(ci[s:e] == v)[0])
    ci[k] = w
    dg = _device(g.rowptr, ci, g.n)
    ctx = _ctx(g, debug_checks=mis2.MIS2_DEBUG_VALIDATE)
    with pytest.raises(mis2.Mis2Error) as e:
        ctx.run(dg)
    assert e.value.status == BAD_GRAPH
    # and the symmetric original passes
    ctx.run(mis2.DeviceGraph.from_host(g))


def test_roots_and_labels_are_checked():
    import torch

    g = gg.grid2d_5pt(12, 12)
    dg = mis2.DeviceGraph.from_host(g)
    ctx = _ctx(g, debug_checks=mis2.MIS2_DEBUG_VALIDATE)
    _, roots, _ = ctx.run(dg, 0)
    labels, na = ctx.aggregate(dg, roots, 0)  # a real MIS-2 passes
    for bad in ([0, 1], [0, 2], [3, 1], [0, g.n]):  # adjacent, two hops, descending, out of range
        with pytest.raises(mis2.Mis2Error) as e:
            ctx.aggregate(dg, torch.tensor(bad, dtype=torch.int32, device="cuda"), 0)
        assert e.value.status == BAD_GRAPH
    ctx.coarsen(dg, labels, na)
    bad_labels = labels.clone()
    bad_labels[7] = na  # one past the last aggregate
    with pytest.raises(mis2.Mis2Error) as e:
        ctx.coarsen(dg, bad_labels, na)
    assert e.value.status == BAD_GRAPH


def test_forced_barrier_timeout_reports_and_recovers():
    g = gg.grid3d_27pt(20, 18, 16)
    dg = mis2.DeviceGraph.from_host(g)
    ctx = _ctx(g, loop=mis2.MIS2_LOOP_DEVICE, debug_checks=mis2.MIS2_DEBUG_FORCE_TIMEOUT, spin_limit=2000)
    with pytest.raises(mis2.Mis2Error) as e:
        ctx.run(dg, 0)
    assert e.value.status == TIMEOUT
    with pytest.raises(mis2.Mis2Error) as e:
        ctx.coarsen_level(dg, 0)
    assert e.value.status == TIMEOUT
    # the context is still usable once the hook is off
    cfg = mis2.mis2_config_default()
    cfg.loop = mis2.MIS2_LOOP_DEVICE
    mis2.mis2_ctx_set_config(ctx.handle, cfg)
    assert_level_equal(g, gpu_level(ctx, g, 0), seed=0)
    # the host-driven loop has no grid barrier: the hook does not affect it
    hctx = _ctx(g, loop=mis2.MIS2_LOOP_HOST, debug_checks=mis2.MIS2_DEBUG_FORCE_TIMEOUT, spin_limit=2000)
    assert_level_equal(g, gpu_level(hctx, g, 0), seed=0)
