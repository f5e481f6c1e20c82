"""CUDA path vs the CPU oracle, element by element, through the C ABI.

Coloring is integer work, so the bar is bit-exact: the colors array, ncolors,
the number of rounds and |U_r| of every round.
"""
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
    m.library()  # fails loudly if the library was not built
    return m


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _check(gcpkg, g, prio=None, options=None):
    rp, ci = _dev(g.rowptr), _dev(g.colidx)
    pt = None if prio is None else _dev(prio.view(np.int32))
    res = gcpkg.color(rp, ci, pt, options=options, round_sizes=True)
    ref = oracle.iterative(g.rowptr, g.colidx, prio)
    got = res.colors.cpu().numpy()
    assert res.rounds == ref.rounds, (g.name, res.rounds, ref.rounds)
    assert res.ncolors == ref.ncolors, (g.name, res.ncolors, ref.ncolors)
    diff = np.nonzero(got != ref.colors)[0]
    assert diff.size == 0, (g.name, diff[:10], got[diff[:10]], ref.colors[diff[:10]])
    assert np.array_equal(res.round_sizes, ref.round_sizes), g.name
    return res


SMALL = [
    lambda: gg.edgeless(1),
    lambda: gg.edgeless(5),
    lambda: gg.path(2),
    lambda: gg.path(97),
    lambda: gg.cycle(31),
    lambda: gg.complete(40),
    lambda: gg.star(300, 0),
    lambda: gg.star(300, 299),
    lambda: gg.star(5000, 2500),
    lambda: gg.complete_bipartite(7, 70),
    lambda: gg.gnm(10000, 50000, 1),            # G(n=10,000, m=50,000), seed 1
    lambda: gg.rmat(12, 8, gg.RMAT_ER, 2),
    lambda: gg.rmat(13, 8, gg.RMAT_G, 5),
    lambda: gg.rmat(14, 8, gg.RMAT_B, 3),
    lambda: gg.grid2d(100, 77, 4),
    lambda: gg.rgg(20000, 4),
]


@pytest.mark.parametrize("make", SMALL)
def test_parity_index_priority(gcpkg, make):
    _check(gcpkg, make())


@pytest.mark.parametrize("make", SMALL[9:])
def test_parity_with_priority(gcpkg, make):
    g = make()
    # few distinct keys, so ties (broken by index) are common
    prio = (gg.draws(77, 5, g.n) >> np.uint64(56)).astype(np.uint32)
    _check(gcpkg, g, prio)


@pytest.mark.parametrize("opts", [
    {"loop_mode": 1},
    {"color_bits": 32},
    {"color_bits": 32, "loop_mode": 1},
    {"small_max_degree": 1, "medium_max_degree": 1},     # nearly everything in 256-entry chunks
    {"small_max_degree": 32, "medium_max_degree": 32},   # no medium bin
    {"small_max_degree": 1, "medium_max_degree": 256},   # nearly everything warp-per-vertex
    {"small_max_degree": 5, "medium_max_degree": 40},
    {"block_threads": 128},
    {"narrow_color_limit": 3},                           # restart with 32-bit state
    {"narrow_color_limit": 200, "loop_mode": 1},
    {"loop_mode": 2},                                    # CUDA graph with a device-side while loop
    {"loop_mode": 2, "color_bits": 32, "block_threads": 128},
    {"loop_mode": 2, "narrow_color_limit": 3},           # overflow stops the graph, 32-bit restart
    {"tail_volume": -1},                                 # grid barriers to the end
    {"tail_volume": 1 << 30},                            # one block runs every round from 2 on
    {"tail_volume": 3000},                               # the switch happens mid-run
    {"tail_volume": 1 << 30, "block_threads": 128, "narrow_color_limit": 3},
])
def test_parity_launch_variants(gcpkg, opts):
    for g in [gg.rmat(13, 8, gg.RMAT_B, 7), gg.complete(300), gg.gnm(3000, 30000, 9)]:
        _check(gcpkg, g, options=opts)


def test_degrees_at_bin_edges(gcpkg):
    """Vertices with degree exactly at and just above each bin limit and chunk
    size (32, 33, 256, 257, 512, 513), plus long rows (hubs joined to a path)."""
    n = 6000
    u, v = list(range(n - 1)), list(range(1, n))
    spec = [(10, 32), (20, 33), (30, 256), (40, 257), (50, 512), (60, 513), (70, 2049)]
    hubs = {h for h, _ in spec}
    for hub, d in spec:
        nb = [(hub + 100 + 37 * j) % n for j in range(4 * d)]
        nb = [w for w in dict.fromkeys(nb) if w not in hubs and abs(w - hub) > 1][:d - 2]
        u += [hub] * len(nb)
        v += nb
    g = gg.from_edges(n, u, v)
    assert [int(g.degrees[h]) for h, _ in spec] == [d for _, d in spec]
    _check(gcpkg, g)
    _check(gcpkg, g, options={"color_bits": 32})
    _check(gcpkg, g, options={"small_max_degree": 31, "medium_max_degree": 255})


def test_many_long_rows(gcpkg):
    """About 20,000 rows longer than 256 entries (G(20,000, 3M), average degree
    300): round 1's long-row pass gives each warp several of them and appends
    the conflicting ones with one atomic per warp; every later round runs on
    hub chunks.  Index priority, random keys with many ties, and the per-round
    launch form."""
    g = gg.gnm(20000, 3000000, 11)
    assert int((g.degrees > 256).sum()) > 19000
    _check(gcpkg, g)
    keys = (gg.draws(5, 9, g.n) >> np.uint64(56)).astype(np.uint32)
    _check(gcpkg, g, prio=keys)
    _check(gcpkg, g, options={"loop_mode": 1})


def test_many_colors_window_rescan(gcpkg):
    """K_600: first-fit colors beyond the 64- and 256-wide mask windows."""
    res = _check(gcpkg, gg.complete(600))
    assert res.ncolors == 600
    res = _check(gcpkg, gg.complete(600), options={"small_max_degree": 1, "medium_max_degree": 256})
    res = _check(gcpkg, gg.complete(200), options={"small_max_degree": 1, "medium_max_degree": 256})


def test_n_zero(gcpkg):
    res = gcpkg.color(_dev(np.zeros(1, np.int32)), _dev(np.zeros(0, np.int32)))
    assert res.ncolors == 0 and res.rounds == 0


def test_max_rounds_status(gcpkg):
    g = gg.path(50)
    for opts in ({"loop_mode": 0}, {"loop_mode": 1}, {"loop_mode": 2}, {"tail_volume": 1 << 30},
                 {"tail_volume": -1}):
        res = gcpkg.color(_dev(g.rowptr), _dev(g.colidx), options={"max_rounds": 7, **opts}, check=False)
        assert res.status == gcpkg.GC_ERR_MAX_ROUNDS and res.rounds == 7


def test_tail_switch_round_sizes(gcpkg):
    """The single-block tail gives the same rounds as grid barriers throughout, on a
    graph whose last rounds are long (an index-ordered path settles one vertex a round)."""
    g = gg.from_edges(3000, np.arange(2999), np.arange(1, 3000))
    for t in (-1, 100, 1 << 30):
        res = _check(gcpkg, g, options={"tail_volume": t})
        assert res.rounds == 3000


def test_repeat_calls_reuse_workspace(gcpkg):
    g = gg.rmat(14, 8, gg.RMAT_G, 1)
    rp, ci = _dev(g.rowptr), _dev(g.colidx)
    a = gcpkg.color(rp, ci)
    b = gcpkg.color(rp, ci)
    assert torch.equal(a.colors, b.colors)
    small = gg.gnm(100, 300, 2)
    _check(gcpkg, small)
    c = gcpkg.color(rp, ci)
    assert torch.equal(a.colors, c.colors)


def test_host_entry_point(gcpkg):
    g = gg.rmat(13, 8, gg.RMAT_B, 4)
    res = gcpkg.color_host(g.rowptr, g.colidx)
    ref = oracle.iterative(g.rowptr, g.colidx)
    assert np.array_equal(res.colors, ref.colors) and res.rounds == ref.rounds
    prio = (gg.draws(3, 5, g.n) >> np.uint64(40)).astype(np.uint32)
    res = gcpkg.color_host(g.rowptr, g.colidx, prio)
    ref = oracle.iterative(g.rowptr, g.colidx, prio)
    assert np.array_equal(res.colors, ref.colors) and res.ncolors == ref.ncolors


@pytest.mark.parametrize("scale,opts", [(18, None), (19, {"validate": 1}), (19, {"loop_mode": 2})])
def test_host_entry_point_in_chunks(gcpkg, scale, opts):
    """Host inputs large enough that colidx goes over in several chunks, round 1
    running on each as it arrives (8 chunks at scale 19)."""
    g = gg.rmat(scale, 8, gg.RMAT_B, 6)
    assert g.nnz >= 2 << 20
    res = gcpkg.color_host(g.rowptr, g.colidx, options=opts)
    ref = oracle.iterative(g.rowptr, g.colidx)
    assert (res.ncolors, res.rounds) == (ref.ncolors, ref.rounds)
    assert np.array_equal(res.colors, ref.colors)
    prio = (gg.draws(4, 5, g.n) >> np.uint64(44)).astype(np.uint32)
    res = gcpkg.color_host(g.rowptr, g.colidx, prio, options=opts)
    ref = oracle.iterative(g.rowptr, g.colidx, prio)
    assert np.array_equal(res.colors, ref.colors) and res.ncolors == ref.ncolors


def test_host_entry_point_edgeless(gcpkg):
    g = gg.edgeless(100)
    res = gcpkg.color_host(g.rowptr, g.colidx)
    assert res.ncolors == 1 and res.rounds == 1 and np.all(res.colors == 1)


def test_validation_rejects_bad_graphs(gcpkg):
    g = gg.gnm(500, 2000, 3)
    assert gcpkg.validate_csr(_dev(g.rowptr), _dev(g.colidx)) == gcpkg.GC_OK
    bad = g.colidx.copy()
    bad[7] = g.n + 3                                   # out of range
    assert gcpkg.validate_csr(_dev(g.rowptr), _dev(bad)) == gcpkg.GC_ERR_BAD_GRAPH
    asym = g.colidx.copy()
    asym[11] = (asym[11] + 1) % g.n                    # breaks symmetry (or makes a loop)
    assert gcpkg.validate_csr(_dev(g.rowptr), _dev(asym)) == gcpkg.GC_ERR_BAD_GRAPH
    rp = g.rowptr.copy()
    rp[5], rp[6] = rp[6], rp[5] - 1                    # a negative degree
    assert gcpkg.validate_csr(_dev(rp), _dev(g.colidx)) == gcpkg.GC_ERR_BAD_GRAPH
    res = gcpkg.color(_dev(g.rowptr), _dev(bad), options={"validate": 1}, check=False)
    assert res.status == gcpkg.GC_ERR_BAD_GRAPH


def test_invalid_arguments(gcpkg):
    g = gg.gnm(50, 100, 1)
    for opts in [{"small_max_degree": 33}, {"medium_max_degree": 257}, {"block_threads": 96},
                 {"loop_mode": 3}, {"color_bits": 8}, {"medium_max_degree": 3, "small_max_degree": 10}]:
        res = gcpkg.color(_dev(g.rowptr), _dev(g.colidx), options=opts, check=False)
        assert res.status == gcpkg.GC_ERR_INVALID


def test_full_size_rmat_er_scale22_bit_exact(gcpkg):
    """R-MAT-ER scale 22, seed 2: the full oracle run at the full size."""
    g = gg.rmat(22, 8, gg.RMAT_ER, 2)
    _check(gcpkg, g)


def _fullsize(name):
    import hashlib
    import json
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "fullsize.json")
    return json.load(open(path))[name], hashlib


@pytest.mark.parametrize("name,make", [
    ("rmat_b_s24_seed3", lambda: gg.rmat(24, 8, gg.RMAT_B, 3)),
    ("rmat_g_s23_seed5", lambda: gg.rmat(23, 8, gg.RMAT_G, 5)),
])
def test_full_size_against_stored_oracle_result(gcpkg, name, make):
    """Full-size workloads in the launch configuration bench.py times (defaults):
    colors hash, ncolors, rounds and every |U_r| against values the oracle
    wrote (tests/golden/make_fullsize.py)."""
    exp, hashlib = _fullsize(name)
    g = make()
    graph_sha = hashlib.sha256(g.rowptr.astype("<i4").tobytes() + g.colidx.astype("<i4").tobytes()).hexdigest()
    assert graph_sha == exp["graph_sha256"], "generator output differs from the stored graph"
    res = gcpkg.color(_dev(g.rowptr), _dev(g.colidx), round_sizes=True)
    colors = res.colors.cpu().numpy()
    assert res.ncolors == exp["ncolors"] and res.rounds == exp["rounds"]
    assert res.round_sizes.tolist() == exp["round_sizes"]
    assert hashlib.sha256(colors.astype("<i4").tobytes()).hexdigest() == exp["colors_sha256"]
    # properties that hold at any size
    src = np.repeat(np.arange(g.n), g.degrees)
    assert not np.any(colors[src] == colors[g.colidx])
    assert np.all((colors >= 1) & (colors <= g.degrees + 1))
