"""Learned vertex priority on the GPU against the oracle, through the C ABI.

Features, network scores and keys are exact functions of the graph and the
parameters (integer features, fp32 fused multiply-add chains in a fixed order,
bf16 rounding to nearest even), so they are compared bit for bit; the
gradient sums samples in a different order, so it is compared within a bound;
the coloring under a learned key is integer work and bit-exact again.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle
from oracle import learned as L

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


def _params(seed, scale=0.3):
    d = gg.draws(seed, 7, L.N_PARAMS)
    u = (d >> np.uint64(11)).astype(np.float64) / float(1 << 53)
    return ((u * 2.0 - 1.0) * scale).astype(np.float32)


def _inputs(seed, n, lo=0.0, hi=16.0):
    d = gg.draws(seed, 9, n * L.N_IN)
    u = (d >> np.uint64(11)).astype(np.float64) / float(1 << 53)
    return (lo + (hi - lo) * u).astype(np.float32).reshape(n, L.N_IN)


GRAPHS = [
    lambda: gg.edgeless(7),
    lambda: gg.path(97),
    lambda: gg.star(5000, 2500),                 # one row of 4999 entries: the warp walk
    lambda: gg.complete(70),                     # rows of 69 entries, all on the warp walk
    lambda: gg.gnm(10000, 50000, 1),
    lambda: gg.rmat(14, 8, gg.RMAT_B, 3),        # hubs and many isolated vertices
    lambda: gg.rmat(13, 8, gg.RMAT_G, 5),
    lambda: gg.grid2d(100, 77, 4),
]


@pytest.mark.parametrize("make", GRAPHS)
def test_features_bit_exact(gcpkg, make):
    g = make()
    got = gcpkg.features(_dev(g.rowptr), _dev(g.colidx)).cpu().numpy()
    want = L.features(g.rowptr, g.colidx)
    bad = np.nonzero(np.any(got.view(np.uint32) != want.view(np.uint32), axis=1))[0]
    assert bad.size == 0, (g.name, bad[:5], got[bad[:5]], want[bad[:5]])


def test_features_empty(gcpkg):
    f = gcpkg.features(_dev(np.zeros(1, np.int32)), _dev(np.zeros(0, np.int32)))
    assert f.shape == (0, 6)


@pytest.mark.parametrize("n", [1, 63, 256, 1000, 70001])
def test_forward_bit_exact(gcpkg, n):
    p = _params(n)
    x = _inputs(n + 1, n, lo=-2.0, hi=24.0)
    got = gcpkg.mlp_forward(_dev(p), _dev(x)).cpu().numpy()
    want = L.mlp_forward(p, x)
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))


def test_forward_on_graph_features(gcpkg):
    g = gg.rmat(14, 8, gg.RMAT_B, 3)
    p = _params(77, scale=0.5)
    got = gcpkg.mlp_forward(_dev(p), gcpkg.features(_dev(g.rowptr), _dev(g.colidx))).cpu().numpy()
    want = L.mlp_forward(p, L.features(g.rowptr, g.colidx))
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))


def test_forward_empty(gcpkg):
    out = gcpkg.mlp_forward(_dev(_params(1)), _dev(np.zeros((0, 6), np.float32)))
    assert out.numel() == 0


@pytest.mark.parametrize("n,scale", [(1, 1.0), (64, 1.0 / 64), (1000, 1e-3), (100003, 1e-5)])
def test_grad_matches_oracle(gcpkg, n, scale):
    p = _params(100 + n)
    x = _inputs(200 + n, n)
    t = np.linspace(-1.0, 1.0, n).astype(np.float32)
    grad = torch.zeros(L.N_PARAMS, dtype=torch.float32, device="cuda")
    sse = torch.zeros(1, dtype=torch.float32, device="cuda")
    gcpkg.mlp_grad(_dev(p), _dev(x), _dev(t), scale, grad, sse)
    want, want_sse = L.mlp_grad(p, x, t, scale, rounding=True)
    got = grad.cpu().numpy().astype(np.float64)
    # fp32 sums of n terms in another order: error below n * 2^-23 of the sum of
    # magnitudes; bounded here by 1e-4 of the largest gradient entry plus that
    assert np.all(np.abs(got - want) <= 1e-4 * np.abs(want).max() + 1e-5 * np.abs(want)), \
        np.abs(got - want).max()
    assert abs(float(sse.item()) - want_sse) <= 1e-4 * want_sse + 1e-6


def test_grad_accumulates(gcpkg):
    p, x = _params(5), _inputs(6, 500)
    t = np.zeros(500, np.float32)
    grad = torch.zeros(L.N_PARAMS, dtype=torch.float32, device="cuda")
    sse = torch.zeros(1, dtype=torch.float32, device="cuda")
    for _ in range(2):
        gcpkg.mlp_grad(_dev(p), _dev(x), _dev(t), 1.0, grad, sse)
    want, want_sse = L.mlp_grad(p, x, t, 1.0)
    assert np.allclose(grad.cpu().numpy(), 2 * want, rtol=1e-4, atol=1e-4 * np.abs(want).max())
    assert abs(float(sse.item()) - 2 * want_sse) <= 1e-4 * want_sse


def test_adam_matches_oracle(gcpkg):
    p = _params(8).astype(np.float64)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    pd, md, vd = _dev(p.astype(np.float32)), _dev(m.astype(np.float32)), _dev(v.astype(np.float32))
    for step in range(1, 6):
        g = np.sin(np.arange(L.N_PARAMS) * 0.13 * step).astype(np.float32)
        gcpkg.adam_step(pd, md, vd, _dev(g), step, 1e-2, 0.9, 0.999, 1e-8)
        p, m, v = L.adam(p, m, v, g, step, 1e-2, 0.9, 0.999, 1e-8)
    assert np.allclose(pd.cpu().numpy(), p, rtol=1e-5, atol=1e-6)
    assert np.allclose(md.cpu().numpy(), m, rtol=1e-5, atol=1e-7)


def test_train_step_is_grad_then_adam(gcpkg):
    p, x = _params(9), _inputs(10, 3000)
    t = np.linspace(0, 1, 3000).astype(np.float32)
    tr = gcpkg.MlpTrainer(_dev(p), lr=1e-3)
    sse = tr.step(_dev(x), _dev(t))
    g, want_sse = L.mlp_grad(p, x, t, 1.0 / 3000)
    want_p, _, _ = L.adam(p, np.zeros(L.N_PARAMS), np.zeros(L.N_PARAMS), g, 1, 1e-3, 0.9, 0.999, 1e-8)
    assert abs(float(sse.item()) - want_sse) <= 1e-4 * want_sse
    # first Adam step moves each parameter by about lr * sign(g); compare where |g| is not tiny
    big = np.abs(g) > 1e-3 * np.abs(g).max()
    assert np.allclose(tr.params.cpu().numpy()[big], want_p[big], rtol=1e-5, atol=1e-6)


def test_keys_bit_exact(gcpkg):
    d = gg.draws(12, 3, 100000)
    s = ((d >> np.uint64(11)).astype(np.float64) / float(1 << 53) * 20.0 - 10.0).astype(np.float32)
    s[:8] = [0.0, -0.0, np.inf, -np.inf, np.nan, 1e-45, -1e-45, 3.4e38]
    got = gcpkg.priority_keys(_dev(s)).cpu().numpy().view(np.uint32)
    assert np.array_equal(got, L.priority_keys(s))


@pytest.mark.parametrize("make", GRAPHS[1:])
def test_learned_coloring_bit_exact(gcpkg, make):
    g = make()
    p = _params(31, scale=0.5)
    rp, ci = _dev(g.rowptr), _dev(g.colidx)
    keys = gcpkg.learned_priority(rp, ci, _dev(p))
    res = gcpkg.color(rp, ci, keys, round_sizes=True)
    want_keys = L.learned_keys(g.rowptr, g.colidx, p)
    assert np.array_equal(keys.cpu().numpy().view(np.uint32), want_keys)
    ref = oracle.iterative(g.rowptr, g.colidx, want_keys)
    assert (res.ncolors, res.rounds) == (ref.ncolors, ref.rounds)
    assert np.array_equal(res.colors.cpu().numpy(), ref.colors)
    assert np.array_equal(res.round_sizes, ref.round_sizes)


def _training_set(seeds, scales):
    xs, ts = [], []
    for seed, s in zip(seeds, scales):
        g = gg.rmat(s, 8, gg.RMAT_G, seed)
        xs.append(L.features(g.rowptr, g.colidx))
        ts.append(L.smallest_last_targets(g.rowptr, g.colidx))
    return np.concatenate(xs), np.concatenate(ts)


def test_training_on_gpu_beats_index_priority(gcpkg):
    """A network trained here, by the GPU kernels, on smallest-last positions of small
    R-MAT-G graphs colors an unseen R-MAT-G graph with fewer colors than index order."""
    x, t = _training_set(range(900, 912), [11, 12, 13] * 4)
    perm = gg.permutation(x.shape[0], 3)
    xd, td = _dev(x[perm]), _dev(t[perm])
    tr = gcpkg.MlpTrainer(_dev(_params(1, scale=0.2)), lr=3e-3)
    batch, losses = 4096, []
    n = x.shape[0]
    for step in range(600):
        off = (step * batch) % (n - batch)
        sse = tr.step(xd[off:off + batch], td[off:off + batch])
        if step % 100 == 0 or step == 599:
            losses.append(float(sse.item()) / batch)
    assert losses[-1] < 0.5 * losses[0], losses
    g = gg.rmat(15, 8, gg.RMAT_G, 5)
    rp, ci = _dev(g.rowptr), _dev(g.colidx)
    plain = gcpkg.color(rp, ci)
    learned = gcpkg.color_learned(rp, ci, tr.params)
    assert learned.ncolors < plain.ncolors, (learned.ncolors, plain.ncolors)
    # and the learned coloring is the oracle's under the oracle's own keys
    ref = oracle.iterative(g.rowptr, g.colidx, L.learned_keys(g.rowptr, g.colidx, tr.params.cpu().numpy()))
    assert np.array_equal(learned.colors.cpu().numpy(), ref.colors)


def _valid(g, colors):
    src = np.repeat(np.arange(g.n, dtype=np.int64), g.degrees)
    assert np.all(colors[src] != colors[g.colidx]), "monochromatic edge"
    assert np.all((colors >= 1) & (colors <= g.degrees + 1))


def test_committed_model_on_rmat_g_scale23(gcpkg):
    """The shipped network on R-MAT-G scale 23 (edge factor 8, seed 5): fewer colors
    than index priority, and the coloring is the oracle's under the oracle's keys."""
    g = gg.rmat(23, 8, gg.RMAT_G, 5)
    rp, ci = _dev(g.rowptr), _dev(g.colidx)
    p = gcpkg.load_priority_model()
    plain = gcpkg.color(rp, ci)
    learned = gcpkg.color_learned(rp, ci, _dev(p), round_sizes=True)
    assert learned.ncolors < plain.ncolors, (learned.ncolors, plain.ncolors)
    keys = L.learned_keys(g.rowptr, g.colidx, p)
    ref = oracle.iterative(g.rowptr, g.colidx, keys)
    assert (learned.ncolors, learned.rounds) == (ref.ncolors, ref.rounds)
    assert np.array_equal(learned.colors.cpu().numpy(), ref.colors)
    assert np.array_equal(learned.round_sizes, ref.round_sizes)


def test_committed_model_on_rmat_b_scale24(gcpkg):
    """The shipped network on the skewed R-MAT-B scale 24 graph (seed 3), a family it
    was not trained on: a valid coloring with no more colors than index priority, and
    the oracle's result under the oracle's own keys (stored by make_fullsize.py)."""
    import hashlib
    import json
    import os
    g = gg.rmat(24, 8, gg.RMAT_B, 3)
    rp, ci = _dev(g.rowptr), _dev(g.colidx)
    plain = gcpkg.color(rp, ci)
    learned = gcpkg.color_learned(rp, ci, round_sizes=True)
    assert learned.ncolors <= plain.ncolors, (learned.ncolors, plain.ncolors)
    colors = learned.colors.cpu().numpy()
    _valid(g, colors)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "fullsize.json")
    exp = json.load(open(path)).get("rmat_b_s24_seed3_learned")
    if exp is not None:
        assert (learned.ncolors, learned.rounds) == (exp["ncolors"], exp["rounds"])
        assert learned.round_sizes.tolist() == exp["round_sizes"]
        assert hashlib.sha256(colors.astype("<i4").tobytes()).hexdigest() == exp["colors_sha256"]
