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


def _core_problem(seed, B=3):
    g = np.random.default_rng(seed)
    p = g.standard_normal(N.N_PARAMS) * 0.03
    X = np.zeros((B, N.IN_PAD))
    mask = np.zeros((B, N.OUT))
    for b in range(B):
        R, d = int(g.integers(1, 9)), g.integers(2, 9, size=3)
        core = np.zeros((16, 16, 16))
        core[:d[0], :d[1], :d[2]] = g.standard_normal(tuple(d))
        core /= np.linalg.norm(core)
        X[b, :4096] = core.ravel(order="F")
        X[b, 4096 + R - 1] = 1.0
        for l in range(3):
            m = np.zeros((16, 8)); m[:d[l], :R] = 1.0
            mask[b, l * 128:(l + 1) * 128] = m.T.ravel()
    return p, X, mask


def test_recon_layouts_and_value():
    # the core and factor layouts against a plain loop, and L for known factors
    p, X, mask = _core_problem(4, B=2)
    S = N.core_of(X)
    assert S[1, 3, 2, 1] == X[1, 3 + 16 * 2 + 256 * 1]
    g = np.random.default_rng(5)
    Y = g.standard_normal((2, N.OUT))
    A, B_, C_ = N.factors_of(Y, mask)
    assert A[0, 4, 2] == Y[0, 0 * 128 + 2 * 16 + 4] * mask[0, 2 * 16 + 4]
    L, _ = N.recon_loss_grad_y(X, Y, mask)
    ref = 0.0
    for b in range(2):
        T = np.zeros((16, 16, 16))
        for r in range(8):
            T += np.multiply.outer(np.multiply.outer(A[b][:, r], B_[b][:, r]), C_[b][:, r])
        ref += np.sum((S[b] - T) ** 2)
    assert abs(L - ref / 2) <= 1e-12 * ref


def test_recon_gradient_matches_central_differences():
    p, X, mask = _core_problem(6)
    L, g = N.recon_loss_grad(p, X, mask)
    rng = np.random.default_rng(7)
    offs = np.cumsum([0] + [int(np.prod(s)) for _, s in N.SHAPES])
    picks = []
    for k in range(len(N.SHAPES)):
        picks += list(rng.integers(offs[k], offs[k + 1], size=4))
    h = 1e-6
    for i in picks:
        e = np.zeros_like(p); e[i] = h
        fd = (N.recon_loss_grad(p + e, X, mask)[0] - N.recon_loss_grad(p - e, X, mask)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])), (i, fd, g[i])
    # the gradient with respect to the outputs, also by differences
    Y = rng.standard_normal((3, N.OUT)) * 0.3
    L0, dY = N.recon_loss_grad_y(X, Y, mask)
    for (b, o) in [(0, 5), (1, 130), (2, 300), (0, 383)]:
        e = np.zeros_like(Y); e[b, o] = h
        fd = (N.recon_loss_grad_y(X, Y + e, mask)[0] - N.recon_loss_grad_y(X, Y - e, mask)[0]) / (2 * h)
        assert abs(fd - dY[b, o]) <= 1e-6 * max(1.0, abs(dY[b, o]))
