"""The synthetic inputs: simple symmetric CSR, deterministic, and shaped like the
paper's R-MAT test graphs (Sec. 4.1, Tables 2 and 4)."""
import numpy as np
import pytest

import graphgen as gg


def _check_simple_symmetric(g):
    assert g.rowptr[0] == 0 and np.all(np.diff(g.rowptr) >= 0) and g.rowptr[-1] == g.nnz
    src = np.repeat(np.arange(g.n, dtype=np.int64), g.degrees)
    dst = g.colidx.astype(np.int64)
    assert np.all((dst >= 0) & (dst < g.n))
    assert not np.any(src == dst), "self loop"
    fwd = np.sort(src * g.n + dst)
    assert np.all(np.diff(fwd) > 0), "duplicate entry"
    assert np.array_equal(fwd, np.sort(dst * g.n + src)), "not symmetric"
    for v in range(min(g.n, 200)):
        row = g.colidx[g.rowptr[v]:g.rowptr[v + 1]]
        assert np.all(np.diff(row) > 0)


@pytest.mark.parametrize("make", [
    lambda: gg.rmat(12, 8, gg.RMAT_B, 3),
    lambda: gg.rmat(12, 8, gg.RMAT_ER, 2, permute=False),
    lambda: gg.gnm(10000, 50000, 1),
    lambda: gg.grid2d(31, 17, 4),
    lambda: gg.rgg(5000, 4),
])
def test_simple_symmetric_csr(make):
    _check_simple_symmetric(make())


def test_deterministic():
    a = gg.rmat(13, 8, gg.RMAT_G, 9)
    b = gg.rmat(13, 8, gg.RMAT_G, 9)
    c = gg.rmat(13, 8, gg.RMAT_G, 10)
    assert np.array_equal(a.rowptr, b.rowptr) and np.array_equal(a.colidx, b.colidx)
    assert not np.array_equal(a.colidx[:100], c.colidx[:100])


def test_gnm_exact_edge_count():
    g = gg.gnm(10000, 50000, 1)
    assert g.m == 50000 and g.n == 10000


def test_grid_degrees():
    g = gg.grid2d(10, 7, 0, permute=False)
    assert g.m == 10 * 6 + 9 * 7
    assert g.max_degree == 4 and g.degrees.min() == 2


def test_permutation_is_bijection():
    for n in [1, 2, 3, 1000, 4097]:
        p = gg.permutation(n, 5)
        assert sorted(p.tolist()) == list(range(n))


def test_rgg_average_degree():
    g = gg.rgg(20000, 8)
    assert 6.5 < 2 * g.m / g.n < 8.5  # boundary effects lower it slightly below 8


@pytest.mark.slow
@pytest.mark.parametrize("abcd,edges,maxdeg,var,isolated", [
    # Table 4 (scale 24 rows): edges, max degree, variance, % isolated vertices
    (gg.RMAT_ER, 134217654, 42, 16.00, 0.0),
    (gg.RMAT_B, 133658229, 38143, 8085.64, 30.81),
])
def test_rmat_scale24_matches_paper_table(abcd, edges, maxdeg, var, isolated):
    g = gg.rmat(24, 8, abcd, 3)
    d = g.degrees
    assert abs(g.m - edges) / edges < 1e-3
    assert abs(g.max_degree - maxdeg) / maxdeg < 0.1
    assert abs(float(np.var(d)) - var) / var < 0.02
    assert abs(100.0 * float((d == 0).mean()) - isolated) < 1.0
