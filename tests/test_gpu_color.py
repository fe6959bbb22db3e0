"""Colour sets of cluster multicolor Gauss-Seidel (Algorithm 4's setup,
colorsets = color(A_c)): the CUDA Jones-Plassmann rounds against the
oracle's first-fit greedy colouring in ascending round-0 tuple order, bit
for bit in the colours and in the ordered colour sets, on fine graphs and on
the coarse graphs of an aggregation."""
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


def _fine():
    yield "grid2d", gg.grid2d_5pt(41, 37)
    yield "grid3d27", gg.grid3d_27pt(15, 13, 11)
    yield "elasticity", gg.elasticity3d(6, 5, 4)
    yield "rmat12", gg.rmat(12, 8, seed=7)
    yield "rmat10_i64", gg.rmat(10, 8, seed=8, rowptr_dtype=np.int64)
    yield "gnp_dense", gg.random_graph(200, 0.9, 3)  # > 64 colours: several windows
    yield "single", gg.grid2d_5pt(1, 1)
    yield "hubs", hub_graph()  # rows above the block-per-row threshold, adjacent to each other
    yield "dense_heavy", gg.random_graph(2600, 0.85, 4)  # every row heavy, hundreds of colours


def _coarse(g, seed=0):
    lv = oracle.coarsen_level(g, seed=seed)
    return gg.CSRGraph(lv.n_aggs, lv.c_rowptr.astype(np.int32), lv.c_colind, g.name + "_coarse")


def _check(g, seed, loop=mis2.MIS2_LOOP_HOST):
    ctx = make_ctx(g, loop=loop)
    dg = mis2.DeviceGraph.from_host(g)
    colors, cptr, clist, rounds = ctx.color(dg, seed)
    ref, nc = oracle.color_greedy(g, seed)
    ref_ptr, ref_list = oracle.color_sets(ref, nc)
    assert np.array_equal(colors.cpu().numpy(), ref)
    assert cptr.numel() == nc + 1
    assert np.array_equal(cptr.cpu().numpy().astype(np.int64), ref_ptr)
    assert np.array_equal(clist.cpu().numpy(), ref_list)
    assert 1 <= rounds <= g.n
    return nc


LOOPS = [mis2.MIS2_LOOP_HOST, mis2.MIS2_LOOP_DEVICE]


@pytest.mark.parametrize("loop", LOOPS)
@pytest.mark.parametrize("seed", [0, 5])
@pytest.mark.parametrize("name,g", list(_fine()))
def test_coloring_matches_the_oracle(name, g, seed, loop):
    nc = _check(g, seed, loop)
    if name in ("gnp_dense", "dense_heavy"):
        assert nc > 64


@pytest.mark.parametrize("name,g", [("grid3d27", gg.grid3d_27pt(30, 28, 26)), ("elasticity", gg.elasticity3d(8, 7, 6)),
                                    ("rmat14", gg.rmat(14, 8, seed=2))])
def test_coarse_graph_coloring_matches_the_oracle(name, g):
    for loop in LOOPS:
        _check(_coarse(g, 3), 3, loop)


def test_device_loop_timeout_reports_and_recovers():
    g = gg.grid3d_27pt(20, 18, 16)
    dg = mis2.DeviceGraph.from_host(g)
    ctx = make_ctx(g, loop=mis2.MIS2_LOOP_DEVICE, debug_checks=mis2.MIS2_DEBUG_FORCE_TIMEOUT, spin_limit=2000)
    with pytest.raises(mis2.Mis2Error) as e:
        ctx.color(dg, 0)
    assert e.value.status == -5  # MIS2_ERR_TIMEOUT
    cfg = mis2.mis2_config_default()
    cfg.loop = mis2.MIS2_LOOP_DEVICE
    mis2.mis2_ctx_set_config(ctx.handle, cfg)
    colors, _, _, _ = ctx.color(dg, 0)
    assert np.array_equal(colors.cpu().numpy(), oracle.color_greedy(g, 0)[0])


def test_empty_graph():
    g = gg.CSRGraph(0, np.zeros(1, dtype=np.int32), np.zeros(0, dtype=np.int32))
    ctx = mis2.Context(1, 1)
    colors, cptr, clist, rounds = ctx.color(mis2.DeviceGraph.from_host(g), 0)
    assert colors.numel() == 0 and cptr.cpu().tolist() == [0] and rounds == 0


@pytest.mark.parametrize("name,g", [("grid3d27", gg.grid3d_27pt(30, 28, 26)), ("rmat14", gg.rmat(14, 8, seed=2)),
                                    ("elasticity", gg.elasticity3d(8, 7, 6))])
def test_cluster_lists_of_an_aggregation(name, g):
    import torch

    lv = oracle.coarsen_level(g, seed=1)
    ctx = make_ctx(g)
    labels = torch.from_numpy(lv.labels.astype(np.int32)).cuda()
    c_ptr, members = ctx.cluster_lists(labels, lv.n_aggs)
    ref_ptr, ref_members = oracle.cluster_lists(lv.labels, lv.n_aggs)
    assert np.array_equal(c_ptr.cpu().numpy().astype(np.int64), ref_ptr)
    assert np.array_equal(members.cpu().numpy(), ref_members)


# key ranges of one, two and three 8-bit radix passes, with empty keys
@pytest.mark.parametrize("n,n_keys", [(1, 1), (5000, 1), (10007, 256), (10007, 257), (300001, 70000),
                                      (2 * 2048 + 1, 4097), (200000, 200000)])
def test_cluster_lists_of_arbitrary_labels(n, n_keys):
    import torch

    keys = (gg.splitmix64(np.arange(n, dtype=np.uint64), 23) % np.uint64(n_keys)).astype(np.int32)
    ctx = mis2.Context(n, 1)
    c_ptr, members = ctx.cluster_lists(torch.from_numpy(keys).cuda(), n_keys)
    ref_ptr, ref_members = oracle.cluster_lists(keys, n_keys)
    assert np.array_equal(c_ptr.cpu().numpy().astype(np.int64), ref_ptr)
    assert np.array_equal(members.cpu().numpy(), ref_members)


def test_cluster_lists_refuse_bad_labels():
    import torch

    ctx = mis2.Context(100, 1)
    labels = torch.zeros(100, dtype=torch.int32, device="cuda")
    labels[37] = 5  # one past the last of 5 aggregates
    with pytest.raises(mis2.Mis2Error) as e:
        ctx.cluster_lists(labels, 5)
    assert e.value.status == -4
    labels[37] = -1
    with pytest.raises(mis2.Mis2Error):
        ctx.cluster_lists(labels, 5)
    with pytest.raises(mis2.Mis2Error):
        ctx.cluster_lists(labels, 101)  # more aggregates than vertices
