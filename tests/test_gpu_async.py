"""Asynchronous Algorithm 2 (Phase 1 reads live colors): schedule-dependent, so
checked for what must hold whatever the schedule -- a proper coloring, every
color between 1 and degree + 1, ncolors the largest color, rounds <= n -- and
for the cases whose result does not depend on the schedule."""
import numpy as np
import pytest

import graphgen as gg

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def gcpkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1205_3809_gb300 as m
    m.library()
    return m


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _valid(g, res):
    c = res.colors.cpu().numpy()
    src = np.repeat(np.arange(g.n, dtype=np.int64), g.degrees)
    assert not np.any(c[src] == c[g.colidx]), g.name
    assert np.all((c >= 1) & (c <= g.degrees + 1)), g.name
    assert res.ncolors == (int(c.max()) if g.n else 0)
    assert 1 <= res.rounds <= max(g.n, 1)


GRAPHS = [
    lambda: gg.path(97), lambda: gg.cycle(31), lambda: gg.complete(40), lambda: gg.star(5000, 2500),
    lambda: gg.gnm(10000, 50000, 1), lambda: gg.rmat(14, 8, gg.RMAT_B, 3), lambda: gg.rmat(13, 8, gg.RMAT_G, 5),
    lambda: gg.grid2d(100, 77, 4), lambda: gg.complete(600),
]


@pytest.mark.parametrize("make", GRAPHS)
def test_valid_index_priority(gcpkg, make):
    g = make()
    _valid(g, gcpkg.color_async(_dev(g.rowptr), _dev(g.colidx)))


@pytest.mark.parametrize("make", GRAPHS[4:7])
def test_valid_with_keys(gcpkg, make):
    g = make()
    keys = (gg.draws(7, 3, g.n) & np.uint64(0xFFFF)).astype(np.uint32)
    _valid(g, gcpkg.color_async(_dev(g.rowptr), _dev(g.colidx), _dev(keys.view(np.int32))))


def test_schedule_free_cases(gcpkg):
    g = gg.edgeless(50)
    r = gcpkg.color_async(_dev(g.rowptr), _dev(g.colidx))
    assert (r.ncolors, r.rounds) == (1, 1)
    g = gg.complete(64)                   # a clique needs n colors whatever the order
    r = gcpkg.color_async(_dev(g.rowptr), _dev(g.colidx))
    assert r.ncolors == 64
    r = gcpkg.color_async(_dev(np.zeros(1, np.int32)), _dev(np.zeros(0, np.int32)))
    assert (r.ncolors, r.rounds) == (0, 0)


def test_max_rounds_status(gcpkg):
    g = gg.complete(300)
    r = gcpkg.color_async(_dev(g.rowptr), _dev(g.colidx), max_rounds=1, check=False)
    assert r.status == gcpkg.GC_ERR_MAX_ROUNDS or r.rounds == 1


def test_large_rmat_b_against_synchronous(gcpkg):
    """Scale 20: valid, and within the synchronous form's rounds (the asynchronous
    Phase 1 sees part of the round's colors, which only helps)."""
    g = gg.rmat(20, 8, gg.RMAT_B, 3)
    rp, ci = _dev(g.rowptr), _dev(g.colidx)
    a = gcpkg.color_async(rp, ci)
    s = gcpkg.color(rp, ci)
    _valid(g, a)
    assert a.rounds <= s.rounds
