"""The packed-tuple ablation (Section V-C, Fig. 2): Algorithm 1 through the
plain tuple engine with Eq. 1's packed tuple must give mis2_run's MIS-2 (the
oracle's, bit for bit, rounds included); with unpacked (status, priority,
id) tuples it must give the oracle's unpacked restatement, which holds the
same priority bits and so the same MIS-2."""
import numpy as np
import pytest

import oracle
from paper_2204_02934_gb300 import graphgen as gg
from paper_2204_02934_gb300 import mis2
from _gpu import hub_graph, make_ctx

pytestmark = pytest.mark.gpu
PACKED = mis2.MIS2_ABLATE_TUPLE_ENGINE
UNPACKED = mis2.MIS2_ABLATE_UNPACKED_TUPLES


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2204_02934_gb300 import _build

    _build.build()


def _graphs():
    yield "grid2d", gg.grid2d_5pt(41, 37)
    yield "grid3d7", gg.grid3d_7pt(20, 19, 18)
    yield "elasticity", gg.elasticity3d(7, 6, 5)  # average degree above 40: 32 lanes per row
    yield "rmat12", gg.rmat(12, 8, seed=7)
    yield "rmat11_i64", gg.rmat(11, 8, seed=8, rowptr_dtype=np.int64)
    yield "hubs", hub_graph()
    yield "single", gg.grid2d_5pt(1, 1)


@pytest.mark.parametrize("seed", [0, 7])
@pytest.mark.parametrize("name,g", list(_graphs()))
def test_packed_tuple_engine_is_mis2(name, g, seed):
    ctx = make_ctx(g, ablation=PACKED)
    in_set, roots, rounds = ctx.run(mis2.DeviceGraph.from_host(g), seed)
    ref = oracle.mis2(g, seed)
    assert np.array_equal(in_set.cpu().numpy(), ref[0])
    assert np.array_equal(roots.cpu().numpy(), ref[1])
    assert rounds == ref[2]


@pytest.mark.parametrize("variant", [mis2.MIS2_HASH_XORSHIFT_STAR, mis2.MIS2_HASH_XORSHIFT, mis2.MIS2_HASH_FIXED])
@pytest.mark.parametrize("name,g", list(_graphs()))
def test_unpacked_tuple_engine_matches_the_oracle(name, g, variant):
    ctx = make_ctx(g, ablation=UNPACKED, hash_variant=variant)
    in_set, roots, rounds = ctx.run(mis2.DeviceGraph.from_host(g), 3)
    ref = oracle.mis2_unpacked(g, 3, hash_variant=variant)
    assert np.array_equal(in_set.cpu().numpy(), ref[0])
    assert np.array_equal(roots.cpu().numpy(), ref[1])
    assert rounds == ref[2]


def test_packed_and_unpacked_break_priority_ties_by_id():
    """Vertices 0 and w adjacent among 2^20 - 2 isolated ones, w drawing the
    same 12 priority bits as vertex 0 in round 0: both tuple forms give the
    tie to the smaller id, and the unpacked engine equals the packed one."""
    n = (1 << 20) - 2
    p0 = oracle.priority_tuple(0, 0, n, 0) >> 20
    w = next(v for v in range(1, n) if oracle.priority_tuple(0, v, n, 0) >> 20 == p0)
    g = gg.graph_from_edges(n, [(0, w)])
    dg = mis2.DeviceGraph.from_host(g)
    pk = make_ctx(g, ablation=PACKED).run(dg, 0)[0].cpu().numpy()
    up = make_ctx(g, ablation=UNPACKED).run(dg, 0)[0].cpu().numpy()
    assert pk[0] == 1 and pk[w] == 0
    assert np.array_equal(up, pk)
    assert np.array_equal(up, oracle.mis2_unpacked(g, 0)[0])


def test_other_calls_refuse_the_tuple_engine():
    g = gg.grid2d_5pt(10, 10)
    dg = mis2.DeviceGraph.from_host(g)
    ctx = make_ctx(g, ablation=UNPACKED)
    _, roots, _ = ctx.run(dg, 0)
    with pytest.raises(mis2.Mis2Error):
        ctx.coarsen_level(dg, 0)
    with pytest.raises(mis2.Mis2Error):
        ctx.aggregate(dg, roots, 0)
