"""mis2_run_noalloc: the MIS-2 entry point for callers that cannot call
cudaMalloc (device memory budgeted up front, an allocator that owns the
device, or code that must not block on allocation).  Its scratch is a fixed
array inside the library, so its results must equal mis2_run's and the
oracle's bit for bit, call after call and at the size limit (where the
worklist, tile and trace regions of the array are used to their ends), a
call must leave the device's free memory unchanged, and oversize graphs must
be refused.

This file is collected last so that a failure here comes after every other
test has run."""
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


def _noalloc(g, seed):
    import torch

    dg = mis2.DeviceGraph.from_host(g)
    in_set = torch.empty(max(g.n, 1), dtype=torch.uint8, device="cuda")
    roots = torch.empty(max(g.n, 1), dtype=torch.int32, device="cuda")
    nr, rounds = mis2.mis2_run_noalloc(dg.csr, seed, in_set, roots)
    torch.cuda.synchronize()
    return in_set[:g.n].cpu().numpy(), roots[:nr].cpu().numpy(), rounds


def _regular(g, seed):
    ctx = mis2.Context(max(g.n, 1), max(g.nnz, 1))
    in_set, roots, rounds = ctx.run(mis2.DeviceGraph.from_host(g), seed)
    out = in_set.cpu().numpy(), roots.cpu().numpy(), rounds
    ctx.close()
    return out


def test_noalloc_matches_mis2_run_on_two_calls_in_a_row():
    """Two different graphs back to back: the second call must not see the
    first call's leftovers in the shared scratch (bit-exact, like every
    parity test here)."""
    cases = [(gg.grid3d_27pt(40, 40, 40), 0), (gg.rmat(15, 8, seed=3, rowptr_dtype=np.int32), 5)]
    for g, seed in cases:
        a = _noalloc(g, seed)
        b = _regular(g, seed)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) and a[2] == b[2]


def test_noalloc_at_the_size_limit_matches_the_oracle():
    """A graph of exactly MIS2_NOALLOC_MAX_N vertices (512 x 512 5-point
    grid), twice in a row, against the oracle and mis2_run."""
    g = gg.grid2d_5pt(512, 512)
    assert g.n == mis2.MIS2_NOALLOC_MAX_N
    ref = oracle.mis2(g, 4)
    for _ in range(2):
        a = _noalloc(g, 4)
        assert np.array_equal(a[0], ref[0]) and np.array_equal(a[1], ref[1]) and a[2] == ref[2]
    b = _regular(g, 4)
    assert np.array_equal(a[0], b[0]) and a[2] == b[2]


def test_noalloc_call_leaves_free_device_memory_unchanged():
    """After a warm-up call (which may load the library's device code and so
    commit the array), a further call allocates nothing: cudaMemGetInfo's
    free bytes are the same before and after it."""
    import torch

    g = gg.grid3d_27pt(30, 30, 30)
    dg = mis2.DeviceGraph.from_host(g)
    in_set = torch.empty(g.n, dtype=torch.uint8, device="cuda")
    roots = torch.empty(g.n, dtype=torch.int32, device="cuda")
    first = mis2.mis2_run_noalloc(dg.csr, 1, in_set, roots)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    again = mis2.mis2_run_noalloc(dg.csr, 1, in_set, roots)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert free1 == free0
    assert again == first


def test_noalloc_refuses_graphs_above_the_maximum():
    g = gg.grid2d_5pt(mis2.MIS2_NOALLOC_MAX_N // 500 + 1, 500)
    assert g.n > mis2.MIS2_NOALLOC_MAX_N
    with pytest.raises(mis2.Mis2Error) as e:
        _noalloc(g, 0)
    assert e.value.status == -1
    assert b"MIS2_NOALLOC_MAX_N" in mis2._lib().mis2_last_error()
