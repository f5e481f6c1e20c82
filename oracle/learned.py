"""Oracle of the learned vertex priority (features, network, gradient, Adam, keys).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle``: the library never imports
it.  The paper colors in index order (Sec. 3.2) and cites vertex orderings for
Greedy (smallest-last, largest-first: Sec. 1, Sec. 3.1); the learned priority
replaces the index by a key that a small network computes from per-vertex
features, trained to place each vertex where an ordering the oracle computes
puts it (on a log scale of the position): smallest-last or largest-first,
whichever lets serial Greedy use fewer colors on that graph.

``features`` and ``mlp_forward`` wrap ``learned.c`` (the score decides the order
of the keys, so it is computed in the network's own precision: bf16 operands,
fp32 fused multiply-add chains in index order).  The gradient, Adam and the
key map are float64 numpy written from their definitions.  What pins each one
is listed in ``learned.c`` and ``tests/test_oracle_learned.py``.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _csr, _load, _ptr, greedy, largest_first_order, smallest_last_order

N_IN, N_HIDDEN = 6, 32
OFF_W1 = 0
OFF_B1 = OFF_W1 + N_HIDDEN * N_IN
OFF_W2 = OFF_B1 + N_HIDDEN
OFF_B2 = OFF_W2 + N_HIDDEN * N_HIDDEN
OFF_W3 = OFF_B2 + N_HIDDEN
OFF_B3 = OFF_W3 + N_HIDDEN
N_PARAMS = OFF_B3 + 1


def unpack(params):
    """(W1 [32,6], b1 [32], W2 [32,32], b2 [32], W3 [32], b3) views of the flat vector."""
    p = np.asarray(params)
    return (p[OFF_W1:OFF_B1].reshape(N_HIDDEN, N_IN), p[OFF_B1:OFF_W2],
            p[OFF_W2:OFF_B2].reshape(N_HIDDEN, N_HIDDEN), p[OFF_B2:OFF_W3],
            p[OFF_W3:OFF_B3], p[OFF_B3])


def bf16(x) -> np.ndarray:
    """Round float32 values to bf16 (nearest, ties to even), returned as float32."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    out = np.empty_like(x)
    _load().orc_bf16_array(_ptr(x), int(x.size), _ptr(out))
    return out


def features(rowptr, colidx) -> np.ndarray:
    """float32 [n, 6] vertex features (definition in learned.c)."""
    rowptr, colidx, n = _csr(rowptr, colidx)
    out = np.zeros((max(n, 0), N_IN), np.float32)
    rc = _load().orc_features(n, _ptr(rowptr), _ptr(colidx), _ptr(out))
    if rc != 0:
        raise RuntimeError(f"orc_features failed: {rc}")
    return out


def mlp_forward(params, x, activations: bool = False):
    """Network output (float32 [n]) in its own precision; with activations=True also
    the bf16 activations a1, a2 (float32 [n, 32] each)."""
    params = np.ascontiguousarray(params, dtype=np.float32)
    assert params.shape == (N_PARAMS,)
    x = np.ascontiguousarray(x, dtype=np.float32).reshape(-1, N_IN)
    n = x.shape[0]
    y = np.zeros(n, np.float32)
    a1 = np.zeros((n, N_HIDDEN), np.float32) if activations else None
    a2 = np.zeros((n, N_HIDDEN), np.float32) if activations else None
    rc = _load().orc_mlp_forward(_ptr(params), _ptr(x), n, _ptr(y), _ptr(a1), _ptr(a2))
    if rc != 0:
        raise RuntimeError(f"orc_mlp_forward failed: {rc}")
    return (y, a1, a2) if activations else y


def forward64(params, x):
    """The same network in float64 with no rounding at all (for derivative checks)."""
    W1, b1, W2, b2, W3, b3 = (np.asarray(a, np.float64) for a in unpack(np.asarray(params, np.float64)))
    a0 = np.asarray(x, np.float64).reshape(-1, N_IN)
    a1 = np.maximum(a0 @ W1.T + b1, 0.0)
    a2 = np.maximum(a1 @ W2.T + b2, 0.0)
    return a2 @ W3 + b3, a0, a1, a2


def mlp_grad(params, x, t, scale: float, rounding: bool = True):
    """Gradient of scale * sum_b (y_b - t_b)^2 with respect to the parameters, float64.

    rounding=True: the network as the kernels run it -- bf16 weights in every
    product, the bf16 activations of ``mlp_forward``, and rounding passing
    gradients straight through.  rounding=False: the unrounded float64 network.
    Returns (grad float64 [1313], sse float).
    """
    params = np.asarray(params, np.float32)
    t = np.asarray(t, np.float64).reshape(-1)
    if rounding:
        y, a1, a2 = mlp_forward(params, x, activations=True)
        a0 = bf16(np.asarray(x, np.float32).reshape(-1, N_IN)).astype(np.float64)
        y, a1, a2 = y.astype(np.float64), a1.astype(np.float64), a2.astype(np.float64)
        W = bf16(params).astype(np.float64)
    else:
        y, a0, a1, a2 = forward64(params, x)
        W = params.astype(np.float64)
    _, _, W2, _, W3, _ = unpack(W)
    err = y - t
    dy = 2.0 * scale * err
    d2 = dy[:, None] * W3[None, :] * (a2 > 0)
    d1 = (d2 @ W2) * (a1 > 0)
    g = np.zeros(N_PARAMS, np.float64)
    g[OFF_W1:OFF_B1] = (d1.T @ a0).ravel()
    g[OFF_B1:OFF_W2] = d1.sum(axis=0)
    g[OFF_W2:OFF_B2] = (d2.T @ a1).ravel()
    g[OFF_B2:OFF_W3] = d2.sum(axis=0)
    g[OFF_W3:OFF_B3] = dy @ a2
    g[OFF_B3] = dy.sum()
    return g, float(err @ err)


def adam(params, m, v, grad, step: int, lr: float, beta1: float, beta2: float, eps: float):
    """One Adam step (Kingma and Ba, 2015, Algorithm 1) in float64; returns (params, m, v)."""
    p = np.asarray(params, np.float64)
    g = np.asarray(grad, np.float64)
    m = beta1 * np.asarray(m, np.float64) + (1.0 - beta1) * g
    v = beta2 * np.asarray(v, np.float64) + (1.0 - beta2) * g * g
    m_hat = m / (1.0 - beta1 ** step)
    v_hat = v / (1.0 - beta2 ** step)
    return p - lr * m_hat / (np.sqrt(v_hat) + eps), m, v


def priority_keys(scores) -> np.ndarray:
    """uint32 keys in the order of the float32 scores: smaller score, smaller key.

    -0 and +0 give one key; NaN gives the key of +inf.  On the binary32 pattern u
    (sign s): the key is u with the sign bit set when s = 0, and ~u when s = 1.
    """
    s = np.array(scores, dtype=np.float32).reshape(-1)
    s[np.isnan(s)] = np.inf
    s[s == 0] = 0.0
    u = s.view(np.uint32)
    return np.where(u >> np.uint32(31), ~u, u | np.uint32(0x80000000)).astype(np.uint32)


def learned_keys(rowptr, colidx, params) -> np.ndarray:
    """Priority keys of every vertex: keys(network(features))."""
    return priority_keys(mlp_forward(params, features(rowptr, colidx)))


def position_targets(order) -> np.ndarray:
    """Training target of each vertex: log2(1 + its position in `order`),
    position 0 = colored first; float32 [n].

    The log spreads the front of the ordering (the dense core, which decides the
    number of colors) over as wide a range as the rest, and keeps the target of
    the first vertices the same in graphs of any size.
    """
    order = np.asarray(order)
    n = order.shape[0]
    pos = np.empty(n, np.float64)
    pos[order] = np.arange(n, dtype=np.float64)
    return np.log2(1.0 + pos).astype(np.float32)


def smallest_last_targets(rowptr, colidx) -> np.ndarray:
    """position_targets of the smallest-last ordering."""
    order, _ = smallest_last_order(rowptr, colidx)
    return position_targets(order)


def ordering_targets(rowptr, colidx):
    """Training targets from the two vertex orderings the paper cites for Greedy
    (Sec. 1, Sec. 3.1): smallest-last and largest-first, both computed here.
    Each is colored by Algorithm 1 (serial Greedy) in its order, and the one that
    uses fewer colors labels the graph; on a tie, smallest-last (its color count
    is bounded by the degeneracy + 1).

    Returns (position_targets of the chosen ordering, {"ordering": its name,
    "colors": {"smallest_last": c, "largest_first": c}}).
    """
    sl, _ = smallest_last_order(rowptr, colidx)
    lf = largest_first_order(rowptr)
    c_sl = greedy(rowptr, colidx, sl)[1]
    c_lf = greedy(rowptr, colidx, lf)[1]
    order, name = (lf, "largest_first") if c_lf < c_sl else (sl, "smallest_last")
    return position_targets(order), {"ordering": name,
                                     "colors": {"smallest_last": int(c_sl), "largest_first": int(c_lf)}}
