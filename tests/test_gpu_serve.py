"""Serving with continuous batching: every request's result is the same alone
and in the mix (and equal to the oracle's), requests really overlap, and the
memory budget gates admission."""
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


def _mix(z):
    """SplitMix64 finaliser on a uint64 array (wrapping arithmetic)."""
    z = z ^ (z >> np.uint64(30))
    z = z * np.uint64(0xBF58476D1CE4E5B9)
    z = z ^ (z >> np.uint64(27))
    z = z * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def fingerprint(arrays, counts):
    """The server's result fingerprint (mis2_result.checksum), restated."""
    tot = np.zeros(1, dtype=np.uint64)
    for k, a in enumerate(arrays):
        i = np.arange(len(a), dtype=np.uint64)
        x = np.ascontiguousarray(a, dtype=np.int32).view(np.uint32).astype(np.uint64)
        tot += _mix(_mix((np.uint64(k) << np.uint64(40)) + i) ^ x).sum(dtype=np.uint64)
    for j, c in enumerate(counts):
        tot += _mix(np.array([((5 + j) << 40) ^ int(c)], dtype=np.uint64))
    return int(tot[0])


def _oracle_checksum(g, seed):
    lv = oracle.coarsen_level(g, seed=seed)
    arrays = (lv.roots, lv.labels, lv.c_rowptr.astype(np.int32), lv.c_colind)
    return fingerprint(arrays, (len(lv.roots), lv.n_aggs, len(lv.c_colind))), lv


def _pool():
    graphs = [gg.grid3d_7pt(s, s, s) for s in (10, 14, 19, 25)]
    graphs += [gg.rmat(sc, 8, seed=sc, rowptr_dtype=np.int32) for sc in (9, 10, 11, 12)]
    graphs += [gg.grid2d_5pt(40, 37), gg.rgg2d(3000, 10.0, 3)]
    keep = [(np.ascontiguousarray(g.rowptr), np.ascontiguousarray(g.colind)) for g in graphs]
    host = [mis2.host_csr(rp, ci, g.n) for g, (rp, ci) in zip(graphs, keep)]
    return graphs, keep, host


@pytest.mark.parametrize("loop", [mis2.MIS2_LOOP_DEVICE, mis2.MIS2_LOOP_HOST])
def test_results_same_alone_and_in_the_mix(loop):
    """One slot (alone), four slots, and two slots merging up to eight queued
    requests into one union launch: the same fingerprint per request, the
    oracle's."""
    graphs, keep, host = _pool()
    n_req = 80
    idx = (np.arange(n_req) * 7) % len(graphs)
    arrivals = gg.poisson_arrivals(n_req, 2000.0, seed=4)
    expect = [_oracle_checksum(g, 3)[0] for g in graphs]
    results = {}
    for name, slots, bmax in (("alone", 1, 0), ("slots", 4, 0), ("merged", 2, 8)):
        srv = mis2.Server(slots=slots, slot_max_n=20000 * max(bmax, 1), slot_max_nnz=200000 * max(bmax, 1),
                          batch_max=bmax, loop=loop)
        res, mif = srv.replay(host, arrivals, idx, seed=3)
        srv.close()
        assert all(r.status == 0 for r in res)
        results[name] = res
        for r, gi in zip(res, idx):
            assert r.checksum == expect[gi], "result differs from the oracle"
        if name == "alone":
            assert mif == 1
    assert [r.checksum for r in results["alone"]] == [r.checksum for r in results["slots"]]
    assert [r.checksum for r in results["alone"]] == [r.checksum for r in results["merged"]]


def _cfg5_requests():
    """Requests of the serving workload's sizes: a 160^3 7-point grid and
    R-MAT scale 20 (average degree 16), plus two small ones."""
    graphs = [gg.grid3d_7pt(160, 160, 160), gg.rmat(20, 8, seed=21, rowptr_dtype=np.int32),
              gg.grid3d_7pt(20, 20, 20), gg.rmat(14, 8, seed=22, rowptr_dtype=np.int32)]
    keep = [(np.ascontiguousarray(g.rowptr), np.ascontiguousarray(g.colind)) for g in graphs]
    host = [mis2.host_csr(rp, ci, g.n) for g, (rp, ci) in zip(graphs, keep)]
    return graphs, keep, host


@pytest.mark.parametrize("bmax", [0, 4])
def test_cfg5_sized_results_equal_the_oracle_element_by_element(bmax):
    """Every output array of every request, returned through the server
    (one request per slot, and merged launches), equals the oracle's element
    by element, with the requests in flight together."""
    graphs, keep, host = _cfg5_requests()
    refs = [oracle.coarsen_level(g, seed=2) for g in graphs]
    tot_n, tot_nnz = sum(g.n for g in graphs), sum(g.nnz for g in graphs)
    srv = mis2.Server(slots=2, slot_max_n=tot_n if bmax else max(g.n for g in graphs),
                      slot_max_nnz=tot_nnz if bmax else max(g.nnz for g in graphs), batch_max=bmax,
                      mem_budget=32 << 30)
    order = [0, 1, 2, 3, 2, 3, 1, 0]
    subs = [(gi,) + srv.submit_out(host[gi], graphs[gi].n, graphs[gi].nnz, 2) for gi in order]
    for gi, t, bufs in subs:
        r = srv.wait(t)
        ref = refs[gi]
        assert r.status == 0
        assert r.n_roots == len(ref.roots) and r.n_aggs == ref.n_aggs and r.c_nnz == len(ref.c_colind)
        n = graphs[gi].n
        assert np.array_equal(bufs["in_set"][:n], ref.in_set)
        assert np.array_equal(bufs["roots"][:r.n_roots], ref.roots)
        assert np.array_equal(bufs["labels"][:n], ref.labels)
        assert np.array_equal(bufs["c_rowptr"][:r.n_aggs + 1].astype(np.int64), ref.c_rowptr)
        assert np.array_equal(bufs["c_colind"][:r.c_nnz], ref.c_colind)
    srv.close()


def test_merged_launches_take_queued_requests_together():
    """Requests queued at once are served in unions of up to batch_max: some
    share their start time, and each union stays within the slot's capacity."""
    graphs, keep, host = _pool()
    n_req = 40
    idx = np.arange(n_req) % len(graphs)
    srv = mis2.Server(slots=1, slot_max_n=60000, slot_max_nnz=600000, batch_max=8)
    res, mif = srv.replay(host, np.zeros(n_req), idx, seed=1)
    srv.close()
    assert all(r.status == 0 for r in res)
    groups = {}
    for r, gi in zip(res, idx):
        groups.setdefault(r.t_start, []).append(graphs[gi])
    assert max(len(v) for v in groups.values()) >= 2, "no launch merged two requests"
    assert all(len(v) <= 8 and sum(g.n for g in v) <= 60000 for v in groups.values())


def test_requests_overlap_when_they_arrive_together():
    graphs, keep, host = _pool()
    n_req = 32
    idx = np.arange(n_req) % len(graphs)
    srv = mis2.Server(slots=4, slot_max_n=20000, slot_max_nnz=200000)
    res, mif = srv.replay(host, np.zeros(n_req), idx, seed=1)
    srv.close()
    assert mif >= 2
    starts = sorted((r.t_start, r.t_done) for r in res)
    overlapped = any(b[0] < a[1] for a, b in zip(starts, starts[1:]))
    assert overlapped


def test_memory_budget_limits_admission():
    graphs, keep, host = _pool()
    big = int(np.argmax([g.nnz for g in graphs]))
    one = graphs[big]
    need = (one.n + 1) * 4 + 4 * one.nnz + one.n * 9 + 4 * (one.n + 1) + 4 * one.nnz
    srv = mis2.Server(slots=4, mem_budget=need + need // 2, slot_max_n=20000, slot_max_nnz=200000)
    res, mif = srv.replay(host, np.zeros(8), np.full(8, big), seed=0)
    srv.close()
    assert mif == 1, "budget admits one copy of the largest request at a time"
    assert len({r.checksum for r in res}) == 1


def test_oversize_request_is_refused():
    graphs, keep, host = _pool()
    srv = mis2.Server(slots=1, slot_max_n=100, slot_max_nnz=1000)
    with pytest.raises(mis2.Mis2Error) as e:
        mis2.mis2_server_submit(srv.handle, host[3], 0)
    assert e.value.status == -2
    srv.close()


def test_cancel_withdraws_queued_requests_only():
    # one slot: the first request runs, the others queue behind it; every
    # cancelled one reports MIS2_ERR_CANCELLED, every other one the oracle's
    # result, and a finished request cannot be cancelled
    graphs, keep, host = _pool()
    big = int(np.argmax([g.nnz for g in graphs]))
    expect = _oracle_checksum(graphs[big], 5)[0]
    srv = mis2.Server(slots=1, slot_max_n=20000, slot_max_nnz=200000)
    tickets = [srv.submit(host[big], 5) for _ in range(24)]
    cancelled = {t: srv.cancel(t) for t in tickets[8:]}
    assert any(cancelled.values()), "the tail of a 24-deep queue behind one slot was still queued"
    for t in tickets:
        r = srv.wait(t)
        if cancelled.get(t):
            assert r.status == -7 and r.slot == -1
        else:
            assert r.status == 0 and r.checksum == expect
    assert not srv.cancel(tickets[0])  # finished: nothing to withdraw
    with pytest.raises(mis2.Mis2Error):
        srv.cancel(10_000)  # unknown ticket
    srv.close()
