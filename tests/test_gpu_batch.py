"""Batched coloring (many graphs, one persistent launch) against the oracle.

Each graph of a batch must get exactly what the oracle gives it alone: colors,
color count and round count, bit for bit, whether the batch runs as plain
launches or as a replayed CUDA graph, with index or key priority.
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
    m.library()
    return m


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _small_mix():
    gs = gg.batch_mix(60, 4, n_min=1, n_max=3000)
    gs.insert(3, gg.edgeless(0))               # an empty graph inside the batch
    gs.insert(10, gg.complete(40))
    gs.insert(20, gg.star(700, 350))           # one row above the per-warp threshold
    gs.insert(30, gg.edgeless(9))
    gs.append(gg.edgeless(0))                  # and one at the end
    return gs


@pytest.fixture(params=[1, 2], ids=["shared-grid", "block-per-graph"])
def mode(request):
    """batch_mode: all graphs in one persistent grid (1) or one thread block per graph (2)."""
    return request.param


def _plan(gcpkg, graphs, keys=None, options=None, mode=0):
    rp, ci, voff, eoff = gcpkg.pack_batch((g.rowptr, g.colidx) for g in graphs)
    pr = None if keys is None else _dev(np.concatenate(keys).view(np.int32))
    opts = dict(options or {})
    if mode:
        opts["batch_mode"] = mode
    b = gcpkg.Batch(_dev(rp), _dev(ci), voff, eoff, pr, options=opts)
    assert not mode or b.mode == mode
    return b, voff


def _check(graphs, b, voff, keys=None, which=None):
    colors = b.colors.cpu().numpy()
    nc = b.ncolors.cpu().numpy()
    rd = b.rounds.cpu().numpy()
    for i, g in enumerate(graphs):
        if which is not None and i not in which:
            continue
        ref = oracle.iterative(g.rowptr, g.colidx, None if keys is None else keys[i])
        got = colors[voff[i]:voff[i + 1]]
        assert (int(nc[i]), int(rd[i])) == (ref.ncolors, ref.rounds), (i, g.name)
        assert np.array_equal(got, ref.colors), (i, g.name)


@pytest.mark.parametrize("graph", [False, True])
def test_small_mix_bit_exact(gcpkg, graph, mode):
    gs = _small_mix()
    b, voff = _plan(gcpkg, gs, mode=mode)
    for _ in range(2):                     # a second run (or graph replay) gives the same
        b.colors.fill_(-1)
        b.run(graph=graph)
        mr, mc = b.status()
        _check(gs, b, voff)
    assert mr == int(b.rounds.max()) and mc == int(b.ncolors.max())
    assert b.launch_count == (2 if mode == 2 else 5)
    b.close()


def test_priority_keys(gcpkg, mode):
    gs = _small_mix()
    keys = [(gg.draws(100 + i, 5, g.n) & np.uint64(0xFF)).astype(np.uint32) for i, g in enumerate(gs)]
    b, voff = _plan(gcpkg, gs, keys, mode=mode)
    b.run(graph=True)
    b.status()
    _check(gs, b, voff, keys)


@pytest.mark.parametrize("options", [
    {"small_max_degree": 8, "medium_max_degree": 64},
    {"small_max_degree": 1, "medium_max_degree": 1, "block_threads": 128},
    {"color_bits": 32},
    {"batch_mode": 2, "max_rounds": 1000},
    {"batch_mode": 2, "local_thread_degree": -1},     # a lane group for every vertex
    {"batch_mode": 2, "local_thread_degree": 1000},   # one thread for every vertex
])
def test_options_do_not_change_results(gcpkg, options):
    gs = _small_mix()[:30]
    b, voff = _plan(gcpkg, gs, options=options)
    b.run()
    b.status()
    _check(gs, b, voff)


def test_empty_batches(gcpkg, mode):
    b = gcpkg.Batch(_dev(np.zeros(0, np.int32)), _dev(np.zeros(0, np.int32)), np.zeros(1, np.int64),
                    np.zeros(1, np.int64), options={"batch_mode": mode})
    b.run()
    assert b.status() == (0, 0)
    gs = [gg.edgeless(0), gg.edgeless(0)]
    b, voff = _plan(gcpkg, gs, options={"batch_mode": mode})
    b.run(graph=True)
    assert b.status() == (0, 0)
    assert b.ncolors.cpu().tolist() == [0, 0] and b.rounds.cpu().tolist() == [0, 0]


def test_colidx_contents_may_change_between_runs(gcpkg, mode):
    c = gg.cycle(50)                      # every row has 2 entries: any relabelling keeps rowptr
    g1 = [c, gg.star(20, 0)]
    rp, ci, voff, eoff = gcpkg.pack_batch((g.rowptr, g.colidx) for g in g1)
    ci_d = _dev(ci)
    b = gcpkg.Batch(_dev(rp), ci_d, voff, eoff, options={"batch_mode": mode})
    b.run(graph=True)
    b.status()
    _check(g1, b, voff)
    q = gg.relabel(c, gg.permutation(50, 7))
    assert np.array_equal(q.rowptr, c.rowptr)
    ci_d[:c.nnz] = _dev(q.colidx)
    b.run(graph=True)
    b.status()
    _check([q, g1[1]], b, voff)
    b.close()


def test_rejects_bad_inputs(gcpkg, mode):
    gs = [gg.path(5), gg.cycle(6)]
    rp, ci, voff, eoff = gcpkg.pack_batch((g.rowptr, g.colidx) for g in gs)
    down = voff.copy()
    down[1] = voff[2] + 1                              # decreasing offsets, same total
    with pytest.raises(gcpkg.GcError) as e:
        gcpkg.Batch(_dev(rp), _dev(ci), down, eoff)
    assert e.value.code == gcpkg.GC_ERR_INVALID
    bad = rp.copy()
    bad[0] = 1                                         # graph 0's rowptr must start at 0
    with pytest.raises(gcpkg.GcError) as e:
        gcpkg.Batch(_dev(bad), _dev(ci), voff, eoff)
    assert e.value.code == gcpkg.GC_ERR_BAD_GRAPH
    badc = ci.copy()
    badc[eoff[1]] = 6                                  # id 6 is outside graph 1 (n = 6)
    with pytest.raises(gcpkg.GcError) as e:
        gcpkg.Batch(_dev(rp), _dev(badc), voff, eoff, options={"validate": 1, "batch_mode": mode})
    assert e.value.code == gcpkg.GC_ERR_BAD_GRAPH
    # without validation the run replaces the id, stays in bounds and reports it
    b = gcpkg.Batch(_dev(rp), _dev(badc), voff, eoff, options={"batch_mode": mode})
    b.run()
    with pytest.raises(gcpkg.GcError) as e:
        b.status()
    assert e.value.code == gcpkg.GC_ERR_BAD_GRAPH
    with pytest.raises(gcpkg.GcError) as e:           # loop mode needs the host each round
        gcpkg.Batch(_dev(rp), _dev(ci), voff, eoff, options={"loop_mode": 1})
    assert e.value.code == gcpkg.GC_ERR_INVALID
    with pytest.raises(gcpkg.GcError) as e:
        gcpkg.Batch(_dev(rp), _dev(ci), voff, eoff, options={"batch_mode": 3})
    assert e.value.code == gcpkg.GC_ERR_INVALID


def test_full_size_mix_4096_graphs(gcpkg, mode):
    """The batched workload: 4,096 graphs, sizes log-uniform in [1,000, 200,000],
    grids / random geometric / R-MAT-G in turn, seed 4, one CUDA-graph launch.
    Sampled graphs against the oracle; every graph against gc_color alone on a
    sample, and every coloring checked for validity."""
    gs = gg.batch_mix(4096, 4)
    rp, ci, voff, eoff = gcpkg.pack_batch((g.rowptr, g.colidx) for g in gs)
    b = gcpkg.Batch(_dev(rp), _dev(ci), voff, eoff)
    assert b.mode == 2                        # what the default picks for this workload
    if mode == 1:
        b.close()
        b = gcpkg.Batch(_dev(rp), _dev(ci), voff, eoff, options={"batch_mode": 1})
    b.run(graph=True)
    b.run(graph=True)
    b.status()
    sample = set(range(0, 4096, 173)) | {int(np.argmax([g.n for g in gs]))}
    _check(gs, b, voff, which=sample)
    colors = b.colors.cpu().numpy()
    nc = b.ncolors.cpu().numpy()
    rd = b.rounds.cpu().numpy()
    for i in range(0, 4096, 41):
        g = gs[i]
        res = gcpkg.color(_dev(g.rowptr), _dev(g.colidx))
        assert (res.ncolors, res.rounds) == (int(nc[i]), int(rd[i]))
        assert np.array_equal(res.colors.cpu().numpy(), colors[voff[i]:voff[i + 1]])
    # validity of every coloring (per graph, to keep host memory small)
    for i, g in enumerate(gs):
        c = colors[voff[i]:voff[i + 1]]
        src = np.repeat(np.arange(g.n, dtype=np.int32), g.degrees)
        assert np.all(c[src] != c[g.colidx]), i
        assert g.n == 0 or (c.min() >= 1 and int(nc[i]) == int(c.max()))


def test_autotune_graph_and_cache(gcpkg, tmp_path, monkeypatch):
    monkeypatch.setenv("GC_TUNE_CACHE", str(tmp_path / "tune.json"))
    g = gg.rmat(14, 8, gg.RMAT_B, 3)
    rp, ci = _dev(g.rowptr), _dev(g.colidx)
    cands = [{"small_max_degree": 8, "medium_max_degree": 64, "block_threads": 128},
             {"small_max_degree": 32, "medium_max_degree": 256, "block_threads": 256}]
    best, table = gcpkg.autotune(rp, ci, candidates=cands, reps=2)
    assert best in cands and len(table) == 2 and all(ms > 0 for _, ms in table)
    again, table2 = gcpkg.autotune(rp, ci, candidates=cands, reps=2)
    assert again == best and table2 == table          # served from the cache
    res = gcpkg.color(rp, ci, options=best)
    ref = oracle.iterative(g.rowptr, g.colidx)
    assert np.array_equal(res.colors.cpu().numpy(), ref.colors)


def test_autotune_batch(gcpkg, tmp_path, monkeypatch):
    monkeypatch.setenv("GC_TUNE_CACHE", str(tmp_path / "tune.json"))
    gs = _small_mix()
    rp, ci, voff, eoff = gcpkg.pack_batch((g.rowptr, g.colidx) for g in gs)
    cands = [{"small_max_degree": 16, "medium_max_degree": 128, "block_threads": 256, "batch_mode": 1},
             {"small_max_degree": 32, "medium_max_degree": 256, "block_threads": 256, "batch_mode": 1},
             {"batch_mode": 2}]
    best, table = gcpkg.autotune_batch(_dev(rp), _dev(ci), voff, eoff, candidates=cands, reps=2)
    assert best in cands and all(ms > 0 for _, ms in table)
    b = gcpkg.Batch(_dev(rp), _dev(ci), voff, eoff, options=best)
    b.run(graph=True)
    b.status()
    _check(gs, b, voff)


def test_learned_priority_on_a_batch(gcpkg, mode):
    """Features on the union graph equal each graph's own features, so the learned
    keys of a batch are each graph's learned keys and every graph gets the oracle's
    learned coloring."""
    from oracle import learned as L
    gs = _small_mix()[:40]
    rp, ci, voff, eoff = gcpkg.pack_batch((g.rowptr, g.colidx) for g in gs)
    keys = torch.zeros(int(voff[-1]), dtype=torch.int32, device="cuda")
    b = gcpkg.Batch(_dev(rp), _dev(ci), voff, eoff, keys, options={"batch_mode": mode})
    params = gcpkg.load_priority_model()
    b.learned_priority(_dev(params), out=keys)
    f = b.features().cpu().numpy()
    b.run(graph=True)
    b.status()
    got_keys = keys.cpu().numpy().view(np.uint32)
    want = []
    for i, g in enumerate(gs):
        assert np.array_equal(f[voff[i]:voff[i + 1]].view(np.uint32),
                              L.features(g.rowptr, g.colidx).view(np.uint32)), i
        k = L.learned_keys(g.rowptr, g.colidx, params)
        assert np.array_equal(got_keys[voff[i]:voff[i + 1]], k), i
        want.append(k)
    _check(gs, b, voff, keys=want)


def test_round_stats(gcpkg, mode):
    """Per-round telemetry of a batch run: |U_r| over the batch is the sum of
    every graph's own |U_r| (the oracle's), round 1 reads every entry, round 2
    every row of U_2, and later rounds no more than the rows of U_r (exactly
    those rows with one block per graph, which reads whole rows)."""
    gs = _small_mix()
    b, voff = _plan(gcpkg, gs, mode=mode)
    b.run(graph=True)
    mr, _ = b.status()
    sizes, vols, bits = b.round_stats()
    assert bits == (8 if mode == 2 else 16) and len(sizes) == len(vols) == mr
    want = np.zeros(mr, np.int64)
    deg_in_round = np.zeros(mr, np.int64)
    for g in gs:
        ref = oracle.iterative(g.rowptr, g.colidx)
        want[:len(ref.round_sizes)] += ref.round_sizes
        for k in range(1, mr + 1):
            deg_in_round[k - 1] += int(g.degrees[ref.settle_round >= k].sum())
    assert sizes.tolist() == want.tolist()
    assert vols[0] == sum(int(g.rowptr[-1]) for g in gs)
    if mr >= 2:
        assert vols[1] == deg_in_round[1]
    assert np.all(vols[2:] <= deg_in_round[2:])
    if mode == 2:
        assert vols[1:].tolist() == deg_in_round[1:].tolist()
    short, _, _ = b.round_stats(cap=1)
    assert short.tolist() == [int(voff[-1])]
    b.close()


def test_block_per_graph_wide_colors_and_large_graphs(gcpkg):
    """One block per graph: a graph whose colors outgrow a byte (K_300 needs 300)
    is recolored by the 32-bit pass, and a graph too large for shared memory
    (a 500 x 500 grid, 250,000 vertices) keeps its colors in global memory;
    both, and the small graphs around them, match the oracle."""
    gs = [gg.complete(300), gg.path(7), gg.grid2d(500, 500, 3), gg.rgg(3000, 11), gg.complete(30)]
    b, voff = _plan(gcpkg, gs, mode=2)
    for graph in (False, True):
        b.colors.fill_(-1)
        b.run(graph=graph)
        mr, mc = b.status()
        _check(gs, b, voff)
    assert mc == 300 and mr == 300
    keys = [(gg.draws(7 + i, 2, g.n) & np.uint64(0xF)).astype(np.uint32) for i, g in enumerate(gs)]
    b, voff = _plan(gcpkg, gs, keys, mode=2)
    b.run()
    b.status()
    _check(gs, b, voff, keys)
    # 16 KB of shared memory: every graph above 16,384 vertices (4,096 with
    # 32-bit colors) splits its colors between shared and global memory
    b, voff = _plan(gcpkg, gs, options={"local_shared_bytes": 16384}, mode=2)
    b.run(graph=True)
    b.status()
    _check(gs, b, voff)
    with pytest.raises(gcpkg.GcError):
        _plan(gcpkg, gs, options={"local_shared_bytes": 1024}, mode=2)


def test_color_batched_one_call(gcpkg, mode):
    """gc_color_batched (plan, run, status, free in one call) gives what a plan gives."""
    gs = _small_mix()[:25]
    rp, ci, voff, eoff = gcpkg.pack_batch((g.rowptr, g.colidx) for g in gs)
    colors, nc, rd = gcpkg.color_batched(_dev(rp), _dev(ci), voff, eoff, options={"batch_mode": mode})
    b, _ = _plan(gcpkg, gs, mode=mode)
    b.run()
    b.status()
    assert torch.equal(colors, b.colors) and torch.equal(nc, b.ncolors) and torch.equal(rd, b.rounds)
    _check(gs, b, voff)
    badc = ci.copy()
    badc[eoff[1]] = 10 ** 6
    with pytest.raises(gcpkg.GcError) as e:
        gcpkg.color_batched(_dev(rp), _dev(badc), voff, eoff, options={"batch_mode": mode})
    assert e.value.code == gcpkg.GC_ERR_BAD_GRAPH
