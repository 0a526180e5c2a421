"""Training and use of the learned initialiser (binding-level loop only).

The network, its loss gradient and the Adam step are the library's kernels
(cpd_initnet_grad, cpd_initnet_adam); this module only draws the initial
parameters and walks the training data in mini-batches.  Training data come
from the batched solver itself (cpd_batch_initnet_data: network inputs made
from compressed cores, targets from the plain method's core CPDs).
"""
from __future__ import annotations

import numpy as np

from . import cpd as _cpd

SHAPES = [("W1", (_cpd.INITNET_HIDDEN, _cpd.INITNET_IN_PAD)), ("b1", (_cpd.INITNET_HIDDEN,)),
          ("W2", (_cpd.INITNET_HIDDEN, _cpd.INITNET_HIDDEN)), ("b2", (_cpd.INITNET_HIDDEN,)),
          ("W3", (_cpd.INITNET_OUT, _cpd.INITNET_HIDDEN)), ("b3", (_cpd.INITNET_OUT,))]


def init_params(seed: int = 0, device="cuda"):
    """He-normal weights (zero on the input padding columns), zero biases."""
    import torch
    g = np.random.default_rng(seed)
    parts = []
    for name, shp in SHAPES:
        if name.startswith("b"):
            parts.append(np.zeros(shp))
            continue
        fan_in = _cpd.INITNET_IN if name == "W1" else shp[1]
        w = g.standard_normal(shp) * np.sqrt(2.0 / fan_in)
        if name == "W1":
            w[:, _cpd.INITNET_IN:] = 0.0
        parts.append(w)
    p = np.concatenate([x.ravel() for x in parts]).astype(np.float32)
    assert p.size == _cpd.cpd_initnet_param_count()
    return torch.from_numpy(p).to(device)


def train(params, X, target, mask, epochs: int = 10, batch: int = 512, lr: float = 1e-3, seed: int = 0,
          stream=None):
    """Adam over the rows of X (device tensors); the loss is the masked mean
    squared error against ``target``, or with ``target=None`` the
    reconstruction error of the input cores by the proposed factors.
    Returns the mean loss of every epoch."""
    import torch
    n = X.shape[0]
    dev = X.device
    m = torch.zeros_like(params)
    v = torch.zeros_like(params)
    grad = torch.empty_like(params)
    loss = torch.zeros(1, dtype=torch.float64, device=dev)
    ws = torch.empty(max(_cpd.cpd_initnet_workspace_size(batch), 256), dtype=torch.uint8, device=dev)
    g = np.random.default_rng(seed)
    step, hist = 0, []
    for _ in range(epochs):
        perm = torch.from_numpy(g.permutation(n)).to(dev)
        total, cnt = torch.zeros(1, dtype=torch.float64, device=dev), 0
        for s in range(0, n - batch + 1, batch):
            idx = perm[s:s + batch]
            xb, mb = X[idx].contiguous(), mask[idx].contiguous()
            tb = target[idx].contiguous() if target is not None else None
            _cpd.cpd_initnet_grad(params, xb, tb, mb, grad=grad, loss=loss, stream=stream, workspace=ws)
            step += 1
            _cpd.cpd_initnet_adam(params, m, v, grad, step, lr=lr, stream=stream)
            total += loss
            cnt += 1
        hist.append(float(total.item()) / max(cnt, 1))
    return hist
