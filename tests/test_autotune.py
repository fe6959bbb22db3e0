"""Autotuner: candidate generation and graph classes on CPU; on the GPU, the
chosen configuration reproduces the default configuration's output."""
import json

import numpy as np
import pytest

from paper_2204_02934_gb300 import graphgen as gg


def test_candidates_and_classes(tmp_path):
    from paper_2204_02934_gb300 import autotune, mis2

    c = autotune.candidates()
    assert all(x["warp_degree"] < x["block_degree"] for x in c)
    loops = {x["loop"] for x in c}
    assert loops == {mis2.MIS2_LOOP_HOST, mis2.MIS2_LOOP_DEVICE}
    assert autotune.graph_class(10**6, 25463592, 26) != autotune.graph_class(4194304, 65245102, 97941)
    p = str(tmp_path / "tuned.json")
    autotune.save(p, "k", {"group_lanes": 1}, 1.5)
    assert autotune.load(p, "k") == {"group_lanes": 1}
    assert autotune.load(p, "missing") is None
    assert json.load(open(p))["k"]["ms"] == 1.5


@pytest.mark.gpu
def test_tuned_config_is_identical_and_fastest(tmp_path):
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle
    from paper_2204_02934_gb300 import _build, autotune, mis2

    _build.build()
    g = gg.rmat(13, 8, seed=4)
    grid = {"group_lanes": [1, 2], "warp_degree": [32, 64], "block_degree": [1024], "loop_blocks_per_sm": [2]}
    best, ms, table = autotune.tune_graph(g, reps=2, grid=grid)
    assert all(r["identical"] for r in table)
    assert ms == min(r["ms"] for r in table)
    ctx = mis2.Context(g.n, g.nnz, cfg=autotune._config(best))
    out = ctx.coarsen_level(mis2.DeviceGraph.from_host(g), 0)
    ref = oracle.coarsen_level(g, seed=0)
    assert np.array_equal(out["labels"].cpu().numpy(), ref.labels)
    path = str(tmp_path / "t.json")
    assert autotune.tuned_config(g, path, reps=1, grid=grid) is not None
    assert autotune.load(path, autotune.graph_class(g.n, g.nnz, int(g.degrees().max()))) is not None


def test_batch_classes(tmp_path):
    from paper_2204_02934_gb300 import autotune

    a = gg.mixed_batch(8, lo=1e3, hi=4e3, seed=3)
    b = gg.mixed_batch(64, lo=1e3, hi=2e5, seed=3)
    assert autotune.batch_class(a) != autotune.batch_class(b)
    assert autotune.batch_class(a) == autotune.batch_class(list(a))


@pytest.mark.gpu
def test_batch_tuning_keeps_the_output(tmp_path):
    """Every batch candidate the tuner times reproduces the default
    configuration's labels and coarse graphs, graph by graph and level by
    level; the chosen one is the fastest of them, and equals the oracle's
    hierarchy."""
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle
    from paper_2204_02934_gb300 import _build, autotune, mis2

    _build.build()
    graphs = gg.mixed_batch(12, lo=1e3, hi=2e4, seed=5)
    best, ms, table = autotune.tune_batch(graphs, min_n=1000, reps=1)
    assert len(table) == 6 and all(r["identical"] for r in table)
    assert ms == min(r["ms"] for r in table)
    b = mis2.Batch(len(graphs), sum(g.n for g in graphs), sum(g.nnz for g in graphs), cfg=autotune._config(best))
    b.coarsen([mis2.DeviceGraph.from_host(g) for g in graphs], min_n=1000)
    for gi, g in enumerate(graphs):
        for L, lv in enumerate(oracle.hierarchy(g, min_n=1000)):
            assert np.array_equal(b.labels(L, gi).cpu().numpy(), lv.labels)
    path = str(tmp_path / "batch.json")
    assert autotune.tuned_batch_config(graphs, path, reps=1) is not None
    assert autotune.load(path, autotune.batch_class(graphs)) is not None
