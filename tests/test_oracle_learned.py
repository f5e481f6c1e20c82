"""Pins of the learned-priority oracle (oracle/learned.c, oracle/learned.py), each
against something other than the oracle itself: torch's bf16 conversion, closed
forms on stars and paths, a scipy.sparse route to the neighbour statistics,
Mitchell's published error bound, hand-worked networks, central finite
differences, torch autograd and torch's Adam."""
import math

import numpy as np
import pytest
import torch

import graphgen as gg
import oracle
from oracle import learned as L


def _params(seed, scale=0.3):
    d = gg.draws(seed, 7, L.N_PARAMS)
    u = (d >> np.uint64(11)).astype(np.float64) / float(1 << 53)
    return ((u * 2.0 - 1.0) * scale).astype(np.float32)


def _inputs(seed, n, lo=0.0, hi=16.0):
    d = gg.draws(seed, 9, n * L.N_IN)
    u = (d >> np.uint64(11)).astype(np.float64) / float(1 << 53)
    return (lo + (hi - lo) * u).astype(np.float32).reshape(n, L.N_IN)


# ---------------------------------------------------------------- bf16

def test_bf16_matches_torch_conversion():
    d = gg.draws(3, 1, 20000)
    bits = (d & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    x = bits.view(np.float32)
    x = x[np.isfinite(x)]
    ties = (np.arange(1, 2000, dtype=np.uint32) << np.uint32(16)) | np.uint32(0x8000)
    special = np.array([0.0, -0.0, 1.0, -1.0, np.inf, -np.inf, 3.3895314e38, 1e-45, -1e-45,
                        1.00390625, 1.01171875], np.float32)
    x = np.concatenate([x, ties.view(np.float32), special])
    got = L.bf16(x)
    want = torch.from_numpy(x.copy()).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))


# ---------------------------------------------------------------- features

def _mitchell_exact(m: int) -> float:
    e = m.bit_length() - 1
    return e + (((m - (1 << e)) << 16) >> e) / 65536.0


def test_features_star_closed_form():
    for n, hub in [(6, 0), (9, 8), (40, 17)]:
        g = gg.star(n, hub)
        f = L.features(g.rowptr, g.colidx)
        k = n - 1
        lk = _mitchell_exact(k + 1)
        assert f[hub].tolist() == [lk, float(int(math.log2(k + 1))), 1.0, 1.0, lk, 1.0]
        leaves = [v for v in range(n) if v != hub]
        assert np.all(f[leaves] == np.array([1.0, 1.0, lk, lk, lk, lk], np.float32))


def test_features_path_and_isolated():
    g = gg.path(5)   # degrees 1 2 2 2 1
    f = L.features(g.rowptr, g.colidx)
    # L(x) = Mitchell's log2(1 + x): L(1) = 1, L(2) = 1.5, L(3) = 2, L(4) = 2.25
    assert f[0].tolist() == [1.0, 1.0, 1.5, 1.5, 1.5, 1.5]     # one neighbour, of degree 2
    assert f[1].tolist() == [1.5, 1.0, 1.0, 1.5, 2.0, 1.0]     # neighbours of degree 1 and 2
    assert f[2].tolist() == [1.5, 1.0, 1.5, 1.5, 2.25, 1.5]    # two neighbours of degree 2
    assert f[4].tolist() == f[0].tolist() and f[3].tolist() == f[1].tolist()
    g0 = gg.edgeless(3)
    assert np.all(L.features(g0.rowptr, g0.colidx) == 0.0)
    assert L.features(np.zeros(1, np.int32), np.zeros(0, np.int32)).shape == (0, 6)


def test_mitchell_log_against_log2():
    # exact at powers of two, below log2 elsewhere by less than 0.0861 (Mitchell 1962)
    g = gg.from_edges(4097, np.zeros(4096, np.int32), np.arange(1, 4097, dtype=np.int32))
    f = L.features(g.rowptr, g.colidx)
    deg = g.degrees
    exact = np.log2(1.0 + deg)
    err = exact - f[:, 0]
    assert np.all(err >= 0) and np.all(err < 0.0861)
    pow2 = ((deg + 1) & deg) == 0
    assert np.all(err[pow2] == 0)
    assert np.array_equal(f[:, 1], np.floor(exact).astype(np.float32))


@pytest.mark.parametrize("make", [
    lambda: gg.rmat(12, 8, gg.RMAT_B, 3),
    lambda: gg.gnm(3000, 9000, 5),
    lambda: gg.grid2d(20, 30, 1),
])
def test_features_match_sparse_route(make):
    sp = pytest.importorskip("scipy.sparse")
    g = make()
    A = sp.csr_matrix((np.ones(g.nnz), g.colidx, g.rowptr), shape=(g.n, g.n))
    deg = np.asarray(A.sum(axis=1)).ravel().astype(np.int64)
    s = (A @ deg.astype(np.float64)).astype(np.int64)
    D = sp.csr_matrix((deg[g.colidx].astype(np.float64), g.colidx, g.rowptr), shape=(g.n, g.n))
    mx = np.asarray(D.max(axis=1).todense()).ravel().astype(np.int64)
    # (a sparse row minimum counts the implicit zeros, so take it with reduceat)
    mn = np.zeros(g.n, np.int64)
    nz = deg > 0
    mn[nz] = np.minimum.reduceat(deg[g.colidx], g.rowptr[:-1][nz])
    f = L.features(g.rowptr, g.colidx)
    for v in range(0, g.n, max(1, g.n // 400)):
        d = int(deg[v])
        want = [_mitchell_exact(d + 1), float(d + 1).__floor__().bit_length() - 1]
        if d > 0:
            want += [_mitchell_exact(int(s[v]) // d + 1), _mitchell_exact(int(mx[v]) + 1),
                     _mitchell_exact(int(s[v]) + 1), _mitchell_exact(int(mn[v]) + 1)]
        else:
            want += [0.0] * 4
        assert f[v].tolist() == want, v


# ---------------------------------------------------------------- forward

def _hand_params():
    p = np.zeros(L.N_PARAMS, np.float32)
    W1, b1, W2, b2, W3, _ = L.unpack(p)
    W1[0, 0] = 1.0            # a1[0] = relu(x0)
    W1[3, 2] = -2.0           # a1[3] = relu(-2 x2 + 1)
    b1[3] = 1.0
    W2[0, 0] = 2.0            # a2[0] = relu(2 a1[0])
    W2[1, 3] = 1.0            # a2[1] = relu(a1[3] - 0.5)   (row = output unit)
    b2[1] = -0.5
    W3[0] = 0.5
    W3[1] = 4.0
    p[L.OFF_B3] = 0.25
    return p


def test_forward_hand_worked():
    p = _hand_params()
    x = np.zeros((4, 6), np.float32)
    x[0, 0] = 3.0                     # a2[0] = 6 -> 3 ; a1[3] = 1 -> a2[1] = 0.5 -> 2
    x[1, 0] = -3.0                    # a2[0] = 0 ; a2[1] = 0.5 -> 2
    x[2, 2] = 0.125                   # a1[3] = 0.75 -> a2[1] = 0.25 -> 1
    x[3, 2] = 1.0                     # a1[3] = 0 -> a2[1] = 0
    y = L.mlp_forward(p, x)
    assert y.tolist() == [0.25 + 3.0 + 2.0, 0.25 + 2.0, 0.25 + 1.0, 0.25]
    # inputs and weights round to bf16 first: 1 + 2^-9 rounds to 1
    x2 = np.zeros((1, 6), np.float32)
    x2[0, 0] = 1.0 + 2.0 ** -9
    assert L.mlp_forward(p, x2)[0] == 0.25 + 1.0 + 2.0


def test_forward_zero_weights_gives_bias():
    p = np.zeros(L.N_PARAMS, np.float32)
    p[L.OFF_B3] = -1.75
    assert np.all(L.mlp_forward(p, _inputs(1, 50)) == -1.75)


def _torch_forward(p, x):
    """float64 torch network with bf16 rounding at the same points."""
    W1, b1, W2, b2, W3, b3 = (torch.from_numpy(np.array(a, np.float64)) for a in L.unpack(p))
    r = lambda t: t.to(torch.bfloat16).to(torch.float64)
    a0 = r(torch.from_numpy(x.astype(np.float64)))
    a1 = r(torch.relu(torch.nn.functional.linear(a0, r(W1), b1)))
    a2 = r(torch.relu(torch.nn.functional.linear(a1, r(W2), b2)))
    return (a2 @ r(W3) + b3).numpy()


def test_forward_matches_torch_float64():
    p = _params(11)
    x = _inputs(12, 4000)
    y = L.mlp_forward(p, x).astype(np.float64)
    ref = _torch_forward(p, x)
    scale = np.abs(ref).max() + 1.0
    diff = np.abs(y - ref)
    # fp32 chains against float64: tiny, except where a bf16 activation lands on
    # the other side of a rounding boundary (a few samples, one bf16 step each)
    assert np.mean(diff <= 1e-5 * scale) > 0.98
    assert diff.max() <= 2e-2 * scale


# ---------------------------------------------------------------- gradient

def test_grad_matches_finite_differences():
    p = _params(21)
    x = _inputs(22, 64)
    t = np.linspace(0.0, 1.0, 64)
    g, sse = L.mlp_grad(p, x, t, scale=1.0 / 64, rounding=False)
    p64 = p.astype(np.float64)

    def loss(q):
        y = L.forward64(q, x)[0]
        return float(np.sum((y - t) ** 2)) / 64

    assert abs(sse - loss(p64) * 64) < 1e-9 * max(1.0, sse)
    h = 1e-6
    idx = list(range(0, L.N_PARAMS, 7)) + [L.OFF_B3, L.OFF_W3 + 5, L.OFF_B2 + 3, L.OFF_B1 + 1]
    for i in idx:
        e = np.zeros_like(p64)
        e[i] = h
        fd = (loss(p64 + e) - loss(p64 - e)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-5 * (abs(fd) + 1e-3), (i, fd, g[i])


def test_grad_matches_torch_autograd():
    p = _params(31)
    x = _inputs(32, 200)
    t = np.cos(np.arange(200) * 0.1)
    g, _ = L.mlp_grad(p, x, t, scale=0.5, rounding=False)
    pt = torch.from_numpy(p.astype(np.float64)).requires_grad_(True)
    W1, b1 = pt[L.OFF_W1:L.OFF_B1].view(32, 6), pt[L.OFF_B1:L.OFF_W2]
    W2, b2 = pt[L.OFF_W2:L.OFF_B2].view(32, 32), pt[L.OFF_B2:L.OFF_W3]
    W3, b3 = pt[L.OFF_W3:L.OFF_B3], pt[L.OFF_B3]
    a = torch.from_numpy(x.astype(np.float64))
    y = torch.relu(torch.relu(a @ W1.T + b1) @ W2.T + b2) @ W3 + b3
    (0.5 * ((y - torch.from_numpy(t)) ** 2).sum()).backward()
    assert np.allclose(g, pt.grad.numpy(), rtol=1e-10, atol=1e-12)


def test_grad_rounded_form_uses_bf16_weights():
    # with every weight and input already a bf16 value and activations that stay
    # exact, the rounded and unrounded gradients agree
    p = _hand_params()
    x = np.zeros((3, 6), np.float32)
    x[:, 0] = [3.0, -1.0, 0.5]
    x[:, 2] = [0.125, 0.0, 1.0]
    t = np.array([1.0, 2.0, 3.0])
    g1, s1 = L.mlp_grad(p, x, t, scale=1.0, rounding=True)
    g0, s0 = L.mlp_grad(p, x, t, scale=1.0, rounding=False)
    assert np.allclose(g1, g0) and abs(s1 - s0) < 1e-12
    # and a weight that is not a bf16 value enters the rounded form rounded
    p2 = p.copy()
    p2[L.OFF_W3 + 0] = 0.5 + 2.0 ** -12
    g2, _ = L.mlp_grad(p2, x, t, scale=1.0, rounding=True)
    assert np.allclose(g2, g1)


# ---------------------------------------------------------------- Adam

def test_adam_matches_torch():
    p0 = _params(41).astype(np.float64)
    pt = torch.nn.Parameter(torch.from_numpy(p0.copy()))
    opt = torch.optim.Adam([pt], lr=3e-3, betas=(0.9, 0.99), eps=1e-8)
    p, m, v = p0.copy(), np.zeros_like(p0), np.zeros_like(p0)
    for step in range(1, 5):
        g = np.sin(np.arange(L.N_PARAMS) * 0.37 * step)
        pt.grad = torch.from_numpy(g.copy())
        opt.step()
        p, m, v = L.adam(p, m, v, g, step, 3e-3, 0.9, 0.99, 1e-8)
    assert np.allclose(p, pt.detach().numpy(), rtol=1e-12, atol=1e-14)


# ---------------------------------------------------------------- keys

def test_keys_follow_score_order():
    d = gg.draws(5, 2, 5000)
    s = ((d >> np.uint64(11)).astype(np.float64) / float(1 << 53) * 200.0 - 100.0).astype(np.float32)
    s[:10] = [0.0, -0.0, np.inf, -np.inf, np.nan, 1e-45, -1e-45, 3.4e38, -3.4e38, 1.0]
    k = oracle.learned.priority_keys(s)
    clean = np.where(np.isnan(s), np.inf, s).astype(np.float64)
    i, j = np.triu_indices(200, 1)
    a, b = clean[i], clean[j]
    ka, kb = k[i].astype(np.int64), k[j].astype(np.int64)
    assert np.all((a < b) == (ka < kb)) and np.all((a == b) == (ka == kb))
    order = np.argsort(clean, kind="stable")
    assert np.array_equal(np.argsort(k, kind="stable"), order)
    assert k[0] == k[1] and k[4] == k[2]


def test_smallest_last_targets_are_log_positions():
    g = gg.rmat(10, 8, gg.RMAT_G, 2)
    t = L.smallest_last_targets(g.rowptr, g.colidx)
    order, _ = oracle.smallest_last_order(g.rowptr, g.colidx)
    pos = np.exp2(t.astype(np.float64)) - 1.0
    assert np.array_equal(np.sort(pos.round().astype(np.int64)), np.arange(g.n))
    assert np.allclose(pos[order], np.arange(g.n), rtol=1e-6, atol=1e-6)
    assert t[order[0]] == 0.0 and t[order[1]] == 1.0 and t[order[3]] == 2.0


@pytest.mark.parametrize("seed,winner", [
    (10, "largest_first"),   # G(40, 120) seeds where serial Greedy does better in largest-first order,
    (12, "smallest_last"),   # better in smallest-last order,
    (1, "smallest_last"),    # and equally well (a tie labels by smallest-last)
])
def test_ordering_targets_label_by_fewer_greedy_colors(seed, winner):
    """The label rule: both orderings colored by Algorithm 1, the one with fewer
    colors gives the targets (log2(1 + position)), smallest-last on a tie."""
    g = gg.gnm(40, 120, seed)
    t, lab = L.ordering_targets(g.rowptr, g.colidx)
    sl, _ = oracle.smallest_last_order(g.rowptr, g.colidx)
    lf = oracle.largest_first_order(g.rowptr)
    c_sl = oracle.greedy(g.rowptr, g.colidx, sl)[1]
    c_lf = oracle.greedy(g.rowptr, g.colidx, lf)[1]
    assert lab["colors"] == {"smallest_last": c_sl, "largest_first": c_lf}
    assert (c_lf < c_sl) == (winner == "largest_first") and (c_sl < c_lf) == (seed == 12)
    assert lab["ordering"] == winner
    order = lf if winner == "largest_first" else sl
    assert np.array_equal(t[order], np.log2(1.0 + np.arange(g.n)).astype(np.float32))


def test_learned_keys_compose():
    g = gg.rmat(9, 8, gg.RMAT_G, 4)
    p = _params(51)
    k = L.learned_keys(g.rowptr, g.colidx, p)
    assert np.array_equal(k, L.priority_keys(L.mlp_forward(p, L.features(g.rowptr, g.colidx))))
    c = oracle.iterative(g.rowptr, g.colidx, priority=k)
    assert c.ncolors >= 1 and c.rounds >= 1
