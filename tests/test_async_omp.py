"""The paper's multicore form of Algorithm 2 (oracle/async_omp.c), a timed CPU
baseline: pinned to Algorithm 1 with one thread, checked for validity with many."""
import numpy as np
import pytest

import graphgen as gg
import oracle
from oracle import async_omp


@pytest.mark.parametrize("g", [gg.gnm(3000, 15000, 1), gg.rmat(12, 8, gg.RMAT_B, 3), gg.grid2d(40, 40, 2),
                               gg.complete(30), gg.star(50, 49)], ids=lambda g: g.name)
def test_one_thread_is_greedy_in_index_order(g):
    """One thread visits U in order and reads every earlier color: Algorithm 1, one round."""
    colors, nc, rd, rc = async_omp.color(g.rowptr, g.colidx, threads=1)
    want, wnc = oracle.greedy(g.rowptr, g.colidx)
    assert rc == 0 and rd == 1 and nc == wnc
    assert np.array_equal(colors, want)


@pytest.mark.parametrize("threads", [2, 4, 8])
def test_many_threads_give_a_valid_coloring(threads):
    for g in (gg.rmat(13, 8, gg.RMAT_B, 5), gg.rgg(4000, 2), gg.complete(40), gg.path(200)):
        colors, nc, rd, rc = async_omp.color(g.rowptr, g.colidx, threads=threads)
        assert rc == 0 and 1 <= rd <= g.n
        assert async_omp.valid(g.rowptr, g.colidx, colors) and nc == int(colors.max())
        keys = (gg.draws(9, 1, g.n) & np.uint64(0xFF)).astype(np.uint32)
        colors, nc, rd, rc = async_omp.color(g.rowptr, g.colidx, keys, threads=threads)
        assert rc == 0 and async_omp.valid(g.rowptr, g.colidx, colors)


def test_degenerate_inputs():
    assert async_omp.color(np.zeros(1, np.int32), np.zeros(0, np.int32), threads=2)[1:] == (0, 0, 0)
    g = gg.edgeless(5)
    colors, nc, rd, rc = async_omp.color(g.rowptr, g.colidx, threads=2)
    assert rc == 0 and (nc, rd) == (1, 1) and np.all(colors == 1)


def test_validity_check_catches_a_bad_coloring():
    g = gg.cycle(6)
    colors, _, _, _ = async_omp.color(g.rowptr, g.colidx, threads=1)
    assert async_omp.valid(g.rowptr, g.colidx, colors)
    bad = colors.copy()
    bad[1] = bad[0]
    assert not async_omp.valid(g.rowptr, g.colidx, bad)
