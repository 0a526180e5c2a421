"""FP64 reference of the learned initialiser's network (test infrastructure).

The thesis has no learned initialiser (dGN starts from random factors or
from the compressed core, Sec. 4.1.2); this is the definition the GPU network
kernels are checked against: a two-hidden-layer perceptron,

    h1 = relu(W1 x + b1),  h2 = relu(W2 h1 + b2),  y = W3 h2 + b3,

with two losses: the masked mean squared error against given factors,
L = sum mask (y - t)^2 / sum mask, and the reconstruction error of the input
core by the proposed factors (the CP objective of Sec. 3.1 on that core);
their gradients by the chain rule (reverse mode), and one Adam step (Kingma & Ba,
"Adam: a method for stochastic optimization", 2015, Algorithm 1).  Rows of
X, Y, T, mask are samples; the parameter vector is
W1 (512 x 4160, row-major) | b1 | W2 (512 x 512) | b2 | W3 (384 x 512) | b3.

``rnd`` is applied to both operands of every matrix product (identity by
default): tests pass a BF16 rounding there to compare with tensor-core
kernels at their own operand precision.  Pinned by central finite
differences of both losses and the closed form of the first Adam step.
"""
import numpy as np

IN, IN_PAD, H, OUT = 4104, 4160, 512, 384
SHAPES = [("W1", (H, IN_PAD)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (OUT, H)), ("b3", (OUT,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def _ident(a):
    return a


def unpack(p):
    """Split the parameter vector into named arrays (views)."""
    out, o = {}, 0
    for name, shp in SHAPES:
        n = int(np.prod(shp))
        out[name] = p[o:o + n].reshape(shp)
        o += n
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], dtype=np.float64).ravel() for name, _ in SHAPES])


def forward(p, X, rnd=_ident):
    """y and the hidden activations for the rows of X."""
    P = unpack(np.asarray(p, dtype=np.float64))
    X = np.asarray(X, dtype=np.float64)
    h1 = np.maximum(rnd(X) @ rnd(P["W1"]).T + P["b1"], 0.0)
    h2 = np.maximum(rnd(h1) @ rnd(P["W2"]).T + P["b2"], 0.0)
    y = rnd(h2) @ rnd(P["W3"]).T + P["b3"]
    return y, (X, h1, h2)


def loss(p, X, T, mask, rnd=_ident):
    y, _ = forward(p, X, rnd)
    m = np.asarray(mask, dtype=np.float64)
    return float(np.sum(m * (y - T) ** 2) / max(np.sum(m), 1.0))


def loss_grad(p, X, T, mask, rnd=_ident):
    """L and dL/dp (same layout as p), by reverse-mode differentiation."""
    P = unpack(np.asarray(p, dtype=np.float64))
    y, (X, h1, h2) = forward(p, X, rnd)
    m = np.asarray(mask, dtype=np.float64)
    denom = max(np.sum(m), 1.0)
    r = m * (y - np.asarray(T, dtype=np.float64))
    L = float(np.sum(r * r) / denom)
    dy = 2.0 * r / denom
    g = {}
    g["W3"] = rnd(dy).T @ rnd(h2)
    g["b3"] = dy.sum(axis=0)
    dh2 = (rnd(dy) @ rnd(P["W3"])) * (h2 > 0)
    g["W2"] = rnd(dh2).T @ rnd(h1)
    g["b2"] = dh2.sum(axis=0)
    dh1 = (rnd(dh2) @ rnd(P["W2"])) * (h1 > 0)
    g["W1"] = rnd(dh1).T @ rnd(X)
    g["b1"] = dh1.sum(axis=0)
    return L, pack(g)


def adam(p, m, v, g, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step; returns the new (p, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def core_of(X):
    """The normalised cores held in the input rows: B x 16 x 16 x 16 (column-major layout)."""
    X = np.asarray(X, dtype=np.float64)
    return X[:, :4096].reshape(-1, 16, 16, 16, order="C").transpose(0, 3, 2, 1)


def factors_of(Y, mask):
    """The three factor blocks (B x 16 x 8 each) held in output rows, masked."""
    Z = np.asarray(Y, dtype=np.float64) * np.asarray(mask, dtype=np.float64)
    return [Z[:, l * 128:(l + 1) * 128].reshape(-1, 8, 16).transpose(0, 2, 1) for l in range(3)]


def recon_loss_grad_y(X, Y, mask):
    """Reconstruction loss of the cores by the proposed factors,
        L = (1/B) sum_b || S_b - sum_r a_r (x) b_r (x) c_r ||^2,
    (S_b the normalised core of row b, factors from row b of Y under the mask)
    and dL/dY, by the CP gradient: dL/dA = -(2/B) E_(1) (C kr B), etc."""
    S = core_of(X)
    A, Bm, Cm = factors_of(Y, mask)
    E = S - np.einsum("bir,bjr,bkr->bijk", A, Bm, Cm)
    n = S.shape[0]
    L = float(np.sum(E * E) / n)
    gA = -2.0 / n * np.einsum("bijk,bjr,bkr->bir", E, Bm, Cm)
    gB = -2.0 / n * np.einsum("bijk,bir,bkr->bjr", E, A, Cm)
    gC = -2.0 / n * np.einsum("bijk,bir,bjr->bkr", E, A, Bm)
    dY = np.concatenate([g.transpose(0, 2, 1).reshape(n, 128) for g in (gA, gB, gC)], axis=1)
    return L, dY * np.asarray(mask, dtype=np.float64)


def recon_loss_grad(p, X, mask, rnd=_ident):
    """The reconstruction loss of the network's proposals and dL/dp."""
    P = unpack(np.asarray(p, dtype=np.float64))
    y, (X, h1, h2) = forward(p, X, rnd)
    L, dy = recon_loss_grad_y(X, y, mask)
    g = {}
    g["W3"] = rnd(dy).T @ rnd(h2)
    g["b3"] = dy.sum(axis=0)
    dh2 = (rnd(dy) @ rnd(P["W3"])) * (h2 > 0)
    g["W2"] = rnd(dh2).T @ rnd(h1)
    g["b2"] = dh2.sum(axis=0)
    dh1 = (rnd(dh2) @ rnd(P["W2"])) * (h1 > 0)
    g["W1"] = rnd(dh1).T @ rnd(X)
    g["b1"] = dh1.sum(axis=0)
    return L, pack(g)
