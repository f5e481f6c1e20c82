"""The larger R-MAT-B graphs of Table 4 (scales 25-27) on one GPU.

Each graph is checked against Table 4's statistics (the generator), colored
in the launch configuration bench.py uses, compared with the oracle's stored
result where tests/golden/make_fullsize.py has written one, and always checked
for properties that hold at any size (a proper coloring, 1 <= color <=
degree + 1, rounds <= n, |U_r| strictly decreasing).  Scale 27 sits just under
the int32 limit of the CSR (nnz = 2,143,667,248 in Table 4).
"""
import hashlib
import json
import os

import numpy as np
import pytest

import graphgen as gg

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# Table 4, R-MAT-B rows: edges, max degree, degree variance, % isolated vertices
TABLE4_B = {
    25: (267592474, 54974, 9539.17, 32.34),
    26: (535599280, 77844, 11213.79, 33.87),
    27: (1071833624, 111702, 13165.52, 35.37),
}


@pytest.fixture(scope="module")
def gcpkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1205_3809_gb300 as m
    m.library()
    return m


def _stored(name):
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "fullsize.json")
    return json.load(open(path)).get(name)


def _check_proper(g, colors, chunk=1 << 24):
    deg = g.degrees
    assert np.all((colors >= 1) & (colors <= deg + 1))
    for v0 in range(0, g.n, chunk):
        v1 = min(g.n, v0 + chunk)
        b, e = int(g.rowptr[v0]), int(g.rowptr[v1])
        src = np.repeat(np.arange(v0, v1, dtype=np.int32), deg[v0:v1])
        assert not np.any(colors[src] == colors[g.colidx[b:e]])


@pytest.mark.parametrize("scale", [25, 26, 27])
def test_large_rmat_b(gcpkg, scale):
    g = gg.rmat(scale, 8, gg.RMAT_B, 3)
    edges, maxdeg, var, isolated = TABLE4_B[scale]
    d = g.degrees
    assert abs(g.m - edges) / edges < 1e-3
    assert abs(g.max_degree - maxdeg) / maxdeg < 0.1
    assert abs(float(np.var(d)) - var) / var < 0.02
    assert abs(100.0 * float((d == 0).mean()) - isolated) < 1.0
    rp, ci = torch.from_numpy(g.rowptr).cuda(), torch.from_numpy(g.colidx).cuda()
    res = gcpkg.color(rp, ci, round_sizes=True)
    colors = res.colors.cpu().numpy()
    del rp, ci
    torch.cuda.empty_cache()
    assert 1 <= res.rounds <= g.n
    sizes = np.asarray(res.round_sizes)
    assert sizes[0] == g.n and np.all(np.diff(sizes) < 0)
    assert res.ncolors == int(colors.max()) <= g.max_degree + 1
    _check_proper(g, colors)
    exp = _stored(f"rmat_b_s{scale}_seed3")
    if exp is not None:
        sha = hashlib.sha256(g.rowptr.astype("<i4").tobytes() + g.colidx.astype("<i4").tobytes()).hexdigest()
        assert sha == exp["graph_sha256"]
        assert (res.ncolors, res.rounds) == (exp["ncolors"], exp["rounds"])
        assert sizes.tolist() == exp["round_sizes"]
        assert hashlib.sha256(colors.astype("<i4").tobytes()).hexdigest() == exp["colors_sha256"]
    gcpkg.release()
