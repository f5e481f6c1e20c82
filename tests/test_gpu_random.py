"""Randomised parity: many small seeded graphs of every generator family, each
colored under a randomly drawn option set (bin limits, block shape, loop mode,
color width, tail switch) and priority (index, keys with many ties, distinct
keys), against the oracle, bit for bit."""
import numpy as np
import pytest

import graphgen as gg
import oracle

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


def _draw(seed, i, k):
    return int(gg.draws(seed, 60 + k, 1, start=i)[0] >> np.uint64(11))


def _graph(i):
    kind = _draw(7, i, 0) % 7
    size = 2 + _draw(7, i, 1) % 20000
    s = _draw(7, i, 2) % 100000
    if kind == 0:
        return gg.gnm(size, min(size * (size - 1) // 2, size * (1 + _draw(7, i, 3) % 12)), s)
    if kind == 1:
        return gg.rmat(max(1, size.bit_length() - 1), 8, gg.RMAT_B, s)
    if kind == 2:
        return gg.rmat(max(1, size.bit_length() - 1), 16, gg.RMAT_G, s)
    if kind == 3:
        return gg.grid2d(1 + size // 50, 1 + size % 50, s)
    if kind == 4:
        return gg.rgg(size, s, avg_degree=4.0 + _draw(7, i, 4) % 20)
    if kind == 5:
        return gg.complete(2 + size % 160)
    return gg.complete_bipartite(1 + size % 40, 1 + (size // 40) % 300)


def _options(i):
    sm = [1, 4, 16, 32][_draw(9, i, 0) % 4]
    mm = max(sm, [1, 40, 128, 256][_draw(9, i, 1) % 4])
    return {"small_max_degree": sm, "medium_max_degree": mm,
            "block_threads": [128, 256][_draw(9, i, 2) % 2],
            "loop_mode": [0, 0, 1, 2][_draw(9, i, 3) % 4],
            "color_bits": [0, 32][_draw(9, i, 4) % 2],
            "tail_volume": [0, 0, 500, 1 << 30][_draw(9, i, 5) % 4]}


def _priority(i, n):
    kind = _draw(11, i, 0) % 3
    if kind == 0:
        return None
    d = gg.draws(11, 70 + i, n)
    if kind == 1:
        return (d & np.uint64(7)).astype(np.uint32)           # many ties: index decides
    return (d >> np.uint64(32)).astype(np.uint32)


@pytest.mark.parametrize("block", range(16))
def test_random_graphs_options_priorities(gcpkg, block):
    for i in range(block * 25, block * 25 + 25):
        g = _graph(i)
        opts = _options(i)
        prio = _priority(i, g.n)
        pt = None if prio is None else _dev(prio.view(np.int32))
        res = gcpkg.color(_dev(g.rowptr), _dev(g.colidx), pt, options=opts, round_sizes=True)
        ref = oracle.iterative(g.rowptr, g.colidx, prio)
        assert (res.ncolors, res.rounds) == (ref.ncolors, ref.rounds), (i, g.name, opts)
        assert np.array_equal(res.colors.cpu().numpy(), ref.colors), (i, g.name, opts)
        assert np.array_equal(res.round_sizes, ref.round_sizes), (i, g.name, opts)
