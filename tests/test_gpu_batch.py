"""Batched hierarchies: every graph of a batch, at every level, must equal
the oracle's recursive coarsening of that graph alone (bit-exact labels and
coarse CSR, same number of levels)."""
import numpy as np
import pytest

import oracle
from paper_2204_02934_gb300 import graphgen as gg
from paper_2204_02934_gb300 import mis2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2204_02934_gb300 import _build

    _build.build()


def _check_batch(graphs, min_n, seed=0, loop=mis2.MIS2_LOOP_DEVICE, mode=0, max_levels=32):
    tot_n = sum(g.n for g in graphs)
    tot_nnz = sum(g.nnz for g in graphs)
    b = mis2.Batch(len(graphs), max(tot_n, 1), max(tot_nnz, 1), loop=loop, agg_mode=mode)
    dgs = [mis2.DeviceGraph.from_host(g) for g in graphs]
    nlev = b.coarsen(dgs, seed=seed, min_n=min_n, max_levels=max_levels)
    deepest = 0
    for gi, g in enumerate(graphs):
        levels = oracle.hierarchy(g, min_n=min_n, max_levels=max_levels, seed=seed, mode=mode)
        deepest = max(deepest, len(levels))
        for L, lv in enumerate(levels):
            n, na, cn = b.level_sizes(L)
            assert na[gi] == lv.n_aggs, (gi, L)
            assert np.array_equal(b.labels(L, gi).cpu().numpy(), lv.labels), (gi, L)
            crp, cci = b.coarse(L, gi)
            assert np.array_equal(crp.cpu().numpy().astype(np.int64), lv.c_rowptr), (gi, L)
            assert np.array_equal(cci.cpu().numpy(), lv.c_colind), (gi, L)
        if len(levels) < nlev:
            n, na, cn = b.level_sizes(len(levels))
            assert n[gi] == 0, "graph coarsened past its stopping level"
    assert nlev == deepest
    b.close()
    return nlev


@pytest.mark.parametrize("loop", [mis2.MIS2_LOOP_DEVICE, mis2.MIS2_LOOP_HOST])
def test_small_mixed_batch(loop):
    graphs = gg.mixed_batch(24, lo=200, hi=6000, seed=3)
    nlev = _check_batch(graphs, min_n=100, loop=loop)
    assert nlev >= 2


def test_batch_with_skewed_and_tiny_graphs():
    graphs = [gg.rmat(11, 8, seed=1), gg.graph_from_edges(50, [(i, i + 1) for i in range(49)]),
              gg.grid3d_27pt(9, 8, 7), gg.rgg2d(4000, 10.0, 2), gg.graph_from_edges(30, []),
              gg.rmat(10, 8, seed=2, rowptr_dtype=np.int32)]
    _check_batch(graphs, min_n=40, seed=9)


def test_batch_basic_mode_and_level_cap():
    graphs = gg.mixed_batch(8, lo=500, hi=3000, seed=5)
    _check_batch(graphs, min_n=10, mode=1, max_levels=2)


def test_repeated_runs_are_identical():
    graphs = gg.mixed_batch(12, lo=300, hi=4000, seed=8)
    tot_n, tot_nnz = sum(g.n for g in graphs), sum(g.nnz for g in graphs)
    b = mis2.Batch(len(graphs), tot_n, tot_nnz)
    dgs = [mis2.DeviceGraph.from_host(g) for g in graphs]
    b.coarsen(dgs, min_n=100)
    first = [b.labels(0, i).cpu().numpy() for i in range(len(graphs))]
    b.coarsen(dgs, min_n=100)
    for i in range(len(graphs)):
        assert np.array_equal(b.labels(0, i).cpu().numpy(), first[i])


def test_full_mixed_batch_512():
    """The 512-graph mixed batch (1k-200k vertices), coarsened until < 1000."""
    graphs = gg.mixed_batch(512)
    _check_batch(graphs, min_n=1000)
