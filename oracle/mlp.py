"""ORACLE -- test infrastructure only (see oracle/__init__.py).

Plain FP64 numpy forward and backward of the density-guess network: fully connected layers
nin -> nh (x L, ReLU) -> nout, mean-squared-error loss; parameter layout per layer W_l (out x in,
row-major) followed by b_l, as in the CUDA library.
"""
import numpy as np


def unpack(params, dims):
    layers, off = [], 0
    for a, b in zip(dims[:-1], dims[1:]):
        W = params[off:off + a * b].reshape(b, a)
        off += a * b
        bias = params[off:off + b]
        off += b
        layers.append((W, bias))
    return layers


def forward(params, dims, X):
    acts = [X]
    Z = []
    layers = unpack(params, dims)
    for l, (W, b) in enumerate(layers):
        z = acts[-1] @ W.T + b
        Z.append(z)
        acts.append(np.maximum(z, 0.0) if l < len(layers) - 1 else z)
    return Z, acts


def loss(params, dims, X, Y):
    _, acts = forward(params, dims, X)
    return float(np.mean((acts[-1] - Y) ** 2))


def gradient(params, dims, X, Y):
    """Backpropagation of the mean-squared error (chain rule written out per layer)."""
    Z, acts = forward(params, dims, X)
    layers = unpack(params, dims)
    grads = []
    dA = 2.0 * (acts[-1] - Y) / Y.size
    for l in range(len(layers) - 1, -1, -1):
        W, _ = layers[l]
        dZ = dA if l == len(layers) - 1 else dA * (Z[l] > 0)
        grads.append((dZ.T @ acts[l], dZ.sum(axis=0)))
        dA = dZ @ W
    out = []
    for dW, db in reversed(grads):
        out += [dW.ravel(), db]
    return np.concatenate(out)
