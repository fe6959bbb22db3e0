"""Distance-k MIS (the generalisation of Algorithm 1) against the oracle's
restatement, bit for bit in the set and the round count; k = 2 equals the
MIS-2 of mis2_run."""
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
    yield "grid2d", gg.grid2d_5pt(41, 37)
    yield "grid3d27", gg.grid3d_27pt(15, 13, 11)
    yield "elasticity", gg.elasticity3d(6, 5, 4)
    yield "rmat12", gg.rmat(12, 8, seed=7)
    yield "rmat10_i64", gg.rmat(10, 8, seed=8, rowptr_dtype=np.int64)
    yield "gnp", gg.random_graph(400, 0.02, 3)
    yield "single", gg.grid2d_5pt(1, 1)
    yield "hubs", hub_graph()  # rows above the block-per-row threshold


@pytest.mark.parametrize("k", [1, 2, 3, 4])
@pytest.mark.parametrize("name,g", list(_graphs()))
def test_misk_matches_the_oracle(name, g, k):
    ctx = make_ctx(g)
    dg = mis2.DeviceGraph.from_host(g)
    in_set, roots, rounds = ctx.run_k(dg, k, 5)
    ref_in, ref_roots, ref_rounds = oracle.misk(g, k, 5)
    assert np.array_equal(in_set.cpu().numpy(), ref_in)
    assert np.array_equal(roots.cpu().numpy(), ref_roots)
    assert rounds == ref_rounds


def test_k2_is_mis2_run():
    g = gg.grid3d_27pt(20, 18, 16)
    dg = mis2.DeviceGraph.from_host(g)
    for loop in (mis2.MIS2_LOOP_HOST, mis2.MIS2_LOOP_DEVICE):
        ctx = make_ctx(g, loop=loop)
        a = ctx.run_k(dg, 2, 9)
        b = ctx.run(dg, 9)
        assert np.array_equal(a[0].cpu().numpy(), b[0].cpu().numpy()) and a[2] == b[2]


def test_k_out_of_range_is_refused():
    g = gg.grid2d_5pt(4, 4)
    ctx = make_ctx(g)
    dg = mis2.DeviceGraph.from_host(g)
    for k in (0, 17):
        with pytest.raises(mis2.Mis2Error):
            ctx.run_k(dg, k)
