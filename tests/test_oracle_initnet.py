"""Pins of the FP64 network reference (learned initialiser) against central
finite differences of the loss and the closed form of the first Adam step."""
import numpy as np

from oracle import initnet as N


def _problem(seed, B=3):
    g = np.random.default_rng(seed)
    p = g.standard_normal(N.N_PARAMS) * 0.05
    X = np.zeros((B, N.IN_PAD))
    X[:, :N.IN] = g.standard_normal((B, N.IN)) * 0.1
    T = g.standard_normal((B, N.OUT))
    mask = (g.random((B, N.OUT)) < 0.6).astype(float)
    return p, X, T, mask


def test_sizes():
    assert N.N_PARAMS == 512 * 4160 + 512 + 512 * 512 + 512 + 384 * 512 + 384
    p = np.arange(N.N_PARAMS, dtype=float)
    assert np.array_equal(N.pack(N.unpack(p)), p)


def test_gradient_matches_central_differences():
    p, X, T, mask = _problem(0)
    L, g = N.loss_grad(p, X, T, mask)
    assert abs(L - N.loss(p, X, T, mask)) <= 1e-12 * abs(L)
    rng = np.random.default_rng(1)
    offs = np.cumsum([0] + [int(np.prod(s)) for _, s in N.SHAPES])
    picks = []
    for k in range(len(N.SHAPES)):           # a few entries of every block
        picks += list(rng.integers(offs[k], offs[k + 1], size=4))
    h = 1e-6
    for i in picks:
        e = np.zeros_like(p); e[i] = h
        fd = (N.loss(p + e, X, T, mask) - N.loss(p - e, X, T, mask)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])), (i, fd, g[i])


def test_relu_gates_and_mask():
    # a zero mask gives a zero loss and gradient; a dead first hidden layer
    # (h1 = 0) passes no gradient to W1, b1, W2, and h2 = relu(b2)
    p, X, T, mask = _problem(2)
    L, g = N.loss_grad(p, X, T, np.zeros_like(mask))
    assert L == 0.0 and not np.any(g)
    P = N.unpack(p.copy())
    P["b1"][:] = -1e3                            # h1 = 0 for every sample
    q = N.pack(P)
    L, g = N.loss_grad(q, X, T, mask)
    G = N.unpack(g)
    assert not np.any(G["W1"]) and not np.any(G["b1"]) and not np.any(G["W2"])
    h2 = np.maximum(P["b2"], 0.0)
    y = np.broadcast_to(P["W3"] @ h2 + P["b3"], T.shape)
    dy = 2 * mask * (y - T) / mask.sum()
    assert np.allclose(G["b3"], dy.sum(0))
    assert np.allclose(G["W3"], np.outer(dy.sum(0), h2))


def test_first_adam_step_is_signed_lr():
    g = np.array([3.0, -2.0, 1e-3, 0.0])
    p, m, v = N.adam(np.zeros(4), np.zeros(4), np.zeros(4), g, step=1, lr=0.01, eps=1e-12)
    assert np.allclose(p, -0.01 * np.sign(g))
