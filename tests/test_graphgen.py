"""Generators: symmetric, sorted, unique, no self-loops; closed-form sizes."""
import numpy as np
import pytest

from paper_2204_02934_gb300 import graphgen as gg


def _check_csr(g):
    rp = g.rowptr.astype(np.int64)
    assert rp[0] == 0 and rp[-1] == g.nnz and (np.diff(rp) >= 0).all()
    rows = np.repeat(np.arange(g.n), np.diff(rp))
    ci = g.colind.astype(np.int64)
    assert ((ci >= 0) & (ci < g.n)).all()
    assert (rows != ci).all(), "self-loop"
    key = rows * g.n + ci
    assert (np.diff(key) > 0).all(), "rows not sorted/unique"
    rev = np.sort(ci * g.n + rows)
    assert (rev == key).all(), "not symmetric"


@pytest.mark.parametrize("nx,ny", [(1, 1), (1, 7), (5, 3), (100, 100)])
def test_grid2d(nx, ny):
    g = gg.grid2d_5pt(nx, ny)
    _check_csr(g)
    assert g.n == nx * ny and g.nnz == 4 * nx * ny - 2 * (nx + ny)


@pytest.mark.parametrize("d", [(1, 1, 1), (2, 3, 4), (10, 10, 10)])
def test_grid3d(d):
    nx, ny, nz = d
    g7 = gg.grid3d_7pt(*d)
    _check_csr(g7)
    assert g7.nnz == 6 * nx * ny * nz - 2 * (nx * ny + ny * nz + nx * nz)
    g27 = gg.grid3d_27pt(*d)
    _check_csr(g27)
    assert g27.nnz == (3 * nx - 2) * (3 * ny - 2) * (3 * nz - 2) - nx * ny * nz


def test_27pt_100_size():
    g = gg.workload_27pt(100)
    assert g.n == 1_000_000 and g.nnz == 25_463_592 == 298 ** 3 - 10 ** 6


def test_elasticity():
    g = gg.elasticity3d(4, 3, 2)
    _check_csr(g)
    assert g.degrees().max() == 80 or g.n < 81


def test_rmat_small():
    g = gg.rmat(10, 8, seed=3)
    _check_csr(g)
    assert g.rowptr.dtype == np.int64
    assert 8 < g.nnz / g.n <= 16
    d = g.degrees()
    assert d.max() > 10 * np.median(d)  # skewed


def test_rgg():
    g = gg.rgg2d(20000, 10.0, 5)
    _check_csr(g)
    assert 8.5 < g.nnz / g.n < 10.5


def test_batch_sizes():
    sizes, types = gg.batch_sizes(512)
    assert sizes.min() >= 1000 and sizes.max() <= 200000
    assert 30000 < sizes.mean() < 45000
    assert set(types.tolist()) == {0, 1, 2}


def test_determinism():
    a = gg.rmat(9, 8, seed=5)
    b = gg.rmat(9, 8, seed=5)
    assert (a.colind == b.colind).all()
