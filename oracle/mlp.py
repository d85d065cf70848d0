"""FP64 reference of the per-amplitude MLP (test infrastructure).

This file is part of the oracle. Only tests may import it; the product path
never does. Forward pass and backpropagation of the mean-squared error for
x -> (Linear + ReLU)^L -> Linear, written out with NumPy; parameters in the
flat layout of the C interface (per layer W[in][out] then b[out]). Used to
check the GPU gradients, which keep weights and activations in BF16.
"""
from __future__ import annotations

import numpy as np


def unflatten(p, sizes):
    """Per-layer (W[in][out], b[out]) from the flat parameter vector of the C interface. The learned
    part is an extension of the method; the paper has none."""
    out, off = [], 0
    for (din, dout) in sizes:
        W = p[off:off + din * dout].reshape(din, dout)
        off += din * dout
        b = p[off:off + dout]
        off += dout
        out.append((W, b))
    return out


def loss_and_grad(p, sizes, X, T):
    """Mean-squared-error loss of the per-amplitude MLP and its gradient by backpropagation, in the
    flat parameter layout. The learned part is an extension of the method; the paper has none."""
    layers = unflatten(np.asarray(p, dtype=np.float64), sizes)
    acts, pres = [np.asarray(X, dtype=np.float64)], []
    for k, (W, b) in enumerate(layers):
        z = acts[-1] @ W + b
        pres.append(z)
        acts.append(np.maximum(z, 0.0) if k < len(layers) - 1 else z)
    Y = acts[-1]
    n = Y.size
    loss = np.sum((Y - T) ** 2) / n
    g = 2.0 * (Y - T) / n
    grads = []
    for k in range(len(layers) - 1, -1, -1):
        W, b = layers[k]
        gW = acts[k].T @ g
        gb = g.sum(axis=0)
        grads.append((gW, gb))
        if k > 0:
            g = (g @ W.T) * (pres[k - 1] > 0)
    grads.reverse()
    flat = np.concatenate([np.concatenate([gW.reshape(-1), gb]) for gW, gb in grads])
    return loss, flat
