"""The GPU activity trace used for measurement: record parsing and the
summary on CPU; on the GPU, a traced level lists the library's kernels in
launch order with consistent times."""
import pytest

from paper_2204_02934_gb300 import trace


def test_parse_and_summary(tmp_path):
    p = tmp_path / "t.trace"
    p.write_text("K 2000 5000 7 _ZN4mis210k_mis_loopILi1EiLb0EEEvNS_9GraphViewIT0_EE\n"
                 "S 1000 1500 7 memset_256\n"
                 "K 4500 6000 7 _ZN4mis212k_tile_countINS_6PredInEEEvlT_Pi\n"
                 "C 9000 9400 7 memcpy_2_160\n")
    recs = trace.parse(str(p))
    assert [r["kind"] for r in recs] == ["memset", "kernel", "kernel", "memcpy"]
    s = trace.summary(recs)
    assert s["ops"] == 4 and s["kernels"] == 2
    assert s["span_us"] == pytest.approx(8.4)
    # covered: [1.0, 1.5] + [2.0, 6.0] (the two kernels overlap) + [9.0, 9.4]
    assert s["covered_us"] == pytest.approx(0.5 + 4.0 + 0.4)
    assert s["idle_us"] == pytest.approx(8.4 - 4.9)
    assert s["per_name"]["k_mis_loop"] == {"count": 1, "us": 3.0}
    assert s["per_name"]["memset"]["count"] == 1
    assert trace.summary([]) == {"ops": 0}


def test_short_names():
    assert trace.short_name("_ZN4mis213k_coarse_candIiEEvNS_9GraphViewIT_EEPKiP4int4") == "k_coarse_cand"
    assert trace.short_name("void at::native::fill(int)") == "void at::native::fill"


@pytest.mark.gpu
def test_traced_level_lists_the_library_kernels():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2204_02934_gb300 import _build, graphgen as gg, mis2

    _build.build()
    g = gg.grid3d_27pt(30, 30, 30)
    ctx = mis2.Context(g.n, g.nnz, loop=mis2.MIS2_LOOP_DEVICE)
    dg = mis2.DeviceGraph.from_host(g)
    ctx.coarsen_level(dg, 0)
    with trace.GpuTrace() as t:
        ctx.coarsen_level(dg, 0)
    names = [trace.short_name(r["name"]) for r in t.records if r["kind"] == "kernel"]
    assert names.count("k_mis_loop") == 2
    assert names.index("k_mis_loop") < names.index("k_agg_claim") < names.index("k_coarse_pack")
    assert all(r["end_ns"] >= r["start_ns"] for r in t.records)
    s = trace.summary(t.records)
    assert 0 < s["covered_us"] <= s["span_us"] and s["kernels"] == len(names)
    ctx.close()
