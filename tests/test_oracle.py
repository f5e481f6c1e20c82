"""Pins for the CPU oracle, each taken from outside the oracle itself.

Algorithm 1 (Greedy) and Algorithm 2 (Iterative) are in Sec. 3 of the paper.
The synchronous-round reading of Algorithm 2 (Phase 1 reads only the previous
round's colors) is the one the oracle implements.
"""
import itertools

import numpy as np
import pytest

import graphgen as gg
import oracle
from tests.conftest import read_golden


def _edges_graph(d):
    n = int(d["n"][0])
    e = [tuple(map(int, x.split("-"))) for x in d["edges"]]
    return gg.from_edges(n, [a for a, _ in e], [b for _, b in e])


def _adj(g):
    return [g.colidx[g.rowptr[v]:g.rowptr[v + 1]].tolist() for v in range(g.n)]


def _assert_proper(g, colors):
    src = np.repeat(np.arange(g.n), g.degrees)
    assert not np.any(colors[src] == colors[g.colidx]), "monochromatic edge"
    assert np.all(colors >= 1)
    # first-fit never exceeds degree + 1 (Sec. 3.1)
    assert np.all(colors <= g.degrees + 1)


# ---------------------------------------------------------------- goldens

@pytest.mark.parametrize("name", ["g7_index.txt", "g7_priority.txt", "c6_index.txt"])
def test_hand_worked_traces(name):
    d = read_golden(name)
    g = _edges_graph(d)
    prio = None if d["priority"] == ["none"] else np.array(list(map(int, d["priority"])), np.uint32)
    r = oracle.iterative(g.rowptr, g.colidx, prio)
    assert r.colors.tolist() == list(map(int, d["colors"]))
    assert r.rounds == int(d["rounds"][0])
    assert r.round_sizes.tolist() == list(map(int, d["round_sizes"]))
    assert r.settle_round.tolist() == list(map(int, d["settle"]))
    if "greedy" in d:
        c, _ = oracle.greedy(g.rowptr, g.colidx)
        assert c.tolist() == list(map(int, d["greedy"]))


# ------------------------------------------------------------ closed forms
# Derived by hand from Algorithm 2 in synchronous rounds.

@pytest.mark.parametrize("n", [0, 1, 2, 7, 100])
def test_edgeless_one_round_one_color(n):
    """No neighbours: round 1 colors every vertex 1 and nothing conflicts."""
    g = gg.edgeless(n)
    r = oracle.iterative(g.rowptr, g.colidx)
    assert r.rounds == (1 if n > 0 else 0)
    assert r.ncolors == (1 if n > 0 else 0)
    assert r.colors.tolist() == [1] * n
    assert r.round_sizes.tolist() == ([n] if n > 0 else [])


@pytest.mark.parametrize("n", [2, 3, 5, 9])
def test_complete_graph_n_rounds(n):
    """K_n: in round r the vertices r-1.. all take color r; vertex r-1 keeps it."""
    g = gg.complete(n)
    r = oracle.iterative(g.rowptr, g.colidx)
    assert r.rounds == n
    assert r.colors.tolist() == list(range(1, n + 1))
    assert r.round_sizes.tolist() == list(range(n, 0, -1))


@pytest.mark.parametrize("n", [2, 3, 6, 11])
def test_index_path_settles_one_vertex_per_round(n):
    """Path 0-1-..-(n-1): vertex k settles in round k+1; colors alternate 1, 2."""
    g = gg.path(n)
    r = oracle.iterative(g.rowptr, g.colidx)
    assert r.rounds == n
    assert r.colors.tolist() == [1 + (k % 2) for k in range(n)]
    assert r.settle_round.tolist() == list(range(1, n + 1))


@pytest.mark.parametrize("n", [3, 6, 40])
def test_stars(n):
    """Hub 0: leaves conflict with the hub in round 1 and all take 2.
    Hub n-1: only the hub conflicts and takes 2."""
    g = gg.star(n, 0)
    r = oracle.iterative(g.rowptr, g.colidx)
    assert r.rounds == 2 and r.colors.tolist() == [1] + [2] * (n - 1)
    g = gg.star(n, n - 1)
    r = oracle.iterative(g.rowptr, g.colidx)
    assert r.rounds == 2 and r.colors.tolist() == [1] * (n - 1) + [2]
    assert r.round_sizes.tolist() == [n, 1]


@pytest.mark.parametrize("a,b", [(1, 1), (2, 5), (4, 3)])
def test_complete_bipartite_low_side_first(a, b):
    """K_{a,b} with the low indices on one side: that side keeps 1, the other takes 2."""
    g = gg.complete_bipartite(a, b)
    r = oracle.iterative(g.rowptr, g.colidx)
    assert r.rounds == 2
    assert r.colors.tolist() == [1] * a + [2] * b
    assert r.round_sizes.tolist() == [a + b, b]


def test_round_two_closed_form_on_random_graph():
    """Round 1 colors all 1, so U_2 = {v : some neighbour precedes v}; those take 2."""
    g = gg.gnm(300, 900, 11)
    r = oracle.iterative(g.rowptr, g.colidx, max_rounds=1, allow_max_rounds=True)
    has_lower = np.array([np.any(g.colidx[g.rowptr[v]:g.rowptr[v + 1]] < v) for v in range(g.n)])
    assert r.round_sizes.tolist() == [g.n]
    r2 = oracle.iterative(g.rowptr, g.colidx, max_rounds=2, allow_max_rounds=True)
    assert r2.round_sizes[1] == has_lower.sum()
    assert np.all(r2.colors[has_lower] == 2) and np.all(r2.colors[~has_lower] == 1)


# -------------------------------------------- one-thread reduction (Sec. 3.2)

@pytest.mark.parametrize("seed", range(5))
def test_sequential_visibility_is_greedy(seed):
    """Run by one thread, Phase 1 is Algorithm 1, so round 1 leaves no conflict."""
    g = gg.gnm(200, 700 + 40 * seed, seed)
    r = oracle.iterative(g.rowptr, g.colidx, mode="sequential")
    c, nc = oracle.greedy(g.rowptr, g.colidx)
    assert r.rounds == 1 and np.array_equal(r.colors, c) and r.ncolors == nc


def test_sequential_visibility_with_priority_is_greedy_in_that_order():
    g = gg.gnm(150, 600, 3)
    p = (gg.draws(9, 7, g.n) >> np.uint64(40)).astype(np.uint32)
    order = np.array(sorted(range(g.n), key=lambda v: (int(p[v]), v)), np.int32)
    r = oracle.iterative(g.rowptr, g.colidx, p, mode="sequential")
    c, _ = oracle.greedy(g.rowptr, g.colidx, order)
    assert r.rounds == 1 and np.array_equal(r.colors, c)


# ------------------------------------------------------------------ greedy

@pytest.mark.parametrize("seed", range(4))
def test_greedy_is_first_fit_fixed_point(seed):
    """Algorithm 1 in natural order: color[v] = min{i>0 : no lower neighbour has i}."""
    g = gg.gnm(250, 1000, 100 + seed)
    c, nc = oracle.greedy(g.rowptr, g.colidx)
    for v, nb in enumerate(_adj(g)):
        taken = {int(c[w]) for w in nb if w < v}
        assert c[v] == next(i for i in itertools.count(1) if i not in taken)
    _assert_proper(g, c)
    assert nc == c.max()


def test_greedy_back_degree_bound_and_smallest_last():
    """Greedy uses <= B+1 colors, B = max back degree of the ordering (Sec. 3.1); in
    smallest-last order B is the degeneracy (max removal degree)."""
    g = gg.rmat(12, 8, gg.RMAT_G, 5)
    for order in [None, oracle.largest_first_order(g.rowptr)]:
        c, nc = oracle.greedy(g.rowptr, g.colidx, order)
        pos = np.empty(g.n, np.int64)
        pos[np.arange(g.n) if order is None else order] = np.arange(g.n)
        src = np.repeat(np.arange(g.n), g.degrees)
        back = np.bincount(src[pos[g.colidx] < pos[src]], minlength=g.n)
        assert nc <= back.max() + 1
        _assert_proper(g, c)
    order, rdeg = oracle.smallest_last_order(g.rowptr, g.colidx)
    assert sorted(order.tolist()) == list(range(g.n))
    c, nc = oracle.greedy(g.rowptr, g.colidx, order)
    assert nc <= rdeg.max() + 1


def test_orderings_hand_cases():
    # star with hub 2 plus pendant path 4-5: degrees [1,1,3,1,1,1]... build it
    g = gg.from_edges(6, [2, 2, 2, 4], [0, 1, 3, 5])
    assert oracle.largest_first_order(g.rowptr).tolist() == [2, 0, 1, 3, 4, 5]
    # smallest-last: removal picks min current degree, ties by index:
    # 0 (deg1), 1 (deg1), 2 (deg1 now), 3 (deg0), 4 (deg1), 5 (deg0) -> reverse
    order, rdeg = oracle.smallest_last_order(g.rowptr, g.colidx)
    assert order.tolist() == [5, 4, 3, 2, 1, 0]
    assert rdeg.tolist() == [1, 1, 1, 0, 1, 0]


# ------------------------------------------------------- chromatic number

def test_chromatic_number_known_graphs():
    assert oracle.chromatic_number(*_csr(gg.complete(6))) == 6
    assert oracle.chromatic_number(*_csr(gg.cycle(7))) == 3
    assert oracle.chromatic_number(*_csr(gg.cycle(8))) == 2
    assert oracle.chromatic_number(*_csr(gg.complete_bipartite(3, 4))) == 2
    assert oracle.chromatic_number(*_csr(gg.edgeless(5))) == 1
    assert oracle.chromatic_number(*_csr(gg.edgeless(0))) == 0
    # Petersen graph: outer 5-cycle, inner pentagram, spokes; chi = 3
    u = [0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 0, 1, 2, 3, 4]
    v = [1, 2, 3, 4, 0, 7, 8, 9, 5, 6, 5, 6, 7, 8, 9]
    assert oracle.chromatic_number(*_csr(gg.from_edges(10, u, v))) == 3


def _csr(g):
    return g.rowptr, g.colidx


@pytest.mark.parametrize("seed", range(30))
def test_iterative_and_greedy_vs_brute_force(seed):
    """chi(G) <= colors used, on random graphs of <= 12 vertices."""
    n = 4 + seed % 9
    m = min(n * (n - 1) // 2, (seed * 7) % (n * (n - 1) // 2 + 1))
    g = gg.gnm(n, m, 1000 + seed)
    chi = oracle.chromatic_number(g.rowptr, g.colidx)
    r = oracle.iterative(g.rowptr, g.colidx)
    c, nc = oracle.greedy(g.rowptr, g.colidx)
    assert chi <= r.ncolors and chi <= nc
    _assert_proper(g, r.colors)
    assert r.rounds <= n


# ------------------------------------- exhaustive small graphs (set form)

def _iterative_by_sets(n, adj, key):
    """Algorithm 2, synchronous rounds, written with Python sets straight from the
    pseudo-code: U <- V; while U: Phase 1 on a snapshot; R <- conflicts; U <- R."""
    color = [0] * n
    U = set(range(n))
    sizes = []
    while U:
        sizes.append(len(U))
        prev = list(color)
        for v in U:
            taken = {prev[w] for w in adj[v]}
            color[v] = next(i for i in itertools.count(1) if i not in taken)
        U = {v for v in U if any(color[w] == color[v] and key(w) < key(v) for w in adj[v])}
    return color, sizes


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6])
def test_exhaustive_all_graphs_up_to_6_vertices(n):
    pairs = list(itertools.combinations(range(n), 2))
    for mask in range(1 << len(pairs)):
        es = [pairs[i] for i in range(len(pairs)) if mask >> i & 1]
        g = gg.from_edges(n, [a for a, _ in es], [b for _, b in es])
        adj = _adj(g)
        r = oracle.iterative(g.rowptr, g.colidx)
        col, sizes = _iterative_by_sets(n, adj, lambda v: v)
        assert r.colors.tolist() == col and r.round_sizes.tolist() == sizes, es


def test_exhaustive_with_priorities_5_vertices():
    n = 5
    pairs = list(itertools.combinations(range(n), 2))
    keys = [np.array(p, np.uint32) for p in ([4, 3, 2, 1, 0], [1, 1, 0, 0, 2], [7, 0, 7, 0, 7])]
    for mask in range(1 << len(pairs)):
        es = [pairs[i] for i in range(len(pairs)) if mask >> i & 1]
        g = gg.from_edges(n, [a for a, _ in es], [b for _, b in es])
        adj = _adj(g)
        for p in keys:
            r = oracle.iterative(g.rowptr, g.colidx, p)
            col, sizes = _iterative_by_sets(n, adj, lambda v: (int(p[v]), v))
            assert r.colors.tolist() == col and r.round_sizes.tolist() == sizes, (es, p)


# ------------------------------------------------------------- invariants

@pytest.mark.parametrize("kind", ["er", "g", "b", "gnm", "grid", "rgg"])
def test_invariants_random_graphs(kind):
    g = {"er": lambda: gg.rmat(11, 8, gg.RMAT_ER, 1),
         "g": lambda: gg.rmat(11, 8, gg.RMAT_G, 2),
         "b": lambda: gg.rmat(11, 8, gg.RMAT_B, 3),
         "gnm": lambda: gg.gnm(3000, 12000, 4),
         "grid": lambda: gg.grid2d(40, 50, 5),
         "rgg": lambda: gg.rgg(3000, 6)}[kind]()
    r = oracle.iterative(g.rowptr, g.colidx)
    _assert_proper(g, r.colors)
    assert r.ncolors <= g.max_degree + 1
    assert 1 <= r.rounds <= g.n
    sizes = r.round_sizes
    assert sizes[0] == g.n and np.all(np.diff(sizes) < 0), "the least vertex of U settles each round"
    # settle_round agrees with the sizes: |U_r| = #{v : settle(v) >= r}
    for k in range(1, r.rounds + 1):
        assert sizes[k - 1] == int((r.settle_round >= k).sum())


@pytest.mark.parametrize("seed", range(3))
def test_priority_equals_relabeling(seed):
    """Metamorphic pin for the priority: coloring G with key p equals coloring the
    graph relabelled by rank of (p[v], v) with index priority, read back through
    the relabelling (Phase 1 is order-free; Phase 2 uses the same strict order)."""
    g = gg.rmat(10, 8, gg.RMAT_B, 20 + seed)
    p = (gg.draws(seed, 3, g.n) >> np.uint64(58)).astype(np.uint32)  # many ties
    rank = np.empty(g.n, np.int64)
    rank[np.lexsort((np.arange(g.n), p))] = np.arange(g.n)
    h = gg.relabel(g, rank)
    a = oracle.iterative(g.rowptr, g.colidx, p)
    b = oracle.iterative(h.rowptr, h.colidx)
    assert np.array_equal(a.colors, b.colors[rank])
    assert a.rounds == b.rounds and np.array_equal(a.round_sizes, b.round_sizes)


def test_max_rounds_reports_status():
    g = gg.path(10)
    r = oracle.iterative(g.rowptr, g.colidx, max_rounds=4, allow_max_rounds=True)
    assert r.status == oracle.ORC_ERR_MAX_ROUNDS and r.rounds == 4
