"""FP64 reference of the surrogate network: forward pass, backpropagation of the
mean squared error, and one Adam step, written from their textbook
definitions (GELU: Hendrycks & Gimpel 2016, exact erf form; Adam: Kingma &
Ba 2015, Algorithm 1).  The paper has no network; this is the CPU side the
GPU training kernels are checked against.

TEST INFRASTRUCTURE ONLY: tests/ are the only callers.  Nothing here is
shared with the CUDA path.

Parameter layout (shared by definition with the C ABI, not by code): for each
layer l, W_l of shape [dims[l+1], dims[l]] row-major, then b_l [dims[l+1]],
concatenated into one flat vector.
"""
from __future__ import annotations

import math

import numpy as np

_erf = np.vectorize(math.erf, otypes=[np.float64])


def gelu(z):
    """z Phi(z), Phi the standard normal distribution function."""
    return 0.5 * z * (1.0 + _erf(z / math.sqrt(2.0)))


def dgelu(z):
    """d/dz [z Phi(z)] = Phi(z) + z phi(z), phi the standard normal density."""
    return 0.5 * (1.0 + _erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def unpack(theta, dims):
    """Flat parameter vector -> [(W_l, b_l)]."""
    out, o = [], 0
    for l in range(len(dims) - 1):
        n, k = dims[l + 1], dims[l]
        W = theta[o:o + n * k].reshape(n, k)
        o += n * k
        b = theta[o:o + n]
        o += n
        out.append((W, b))
    assert o == len(theta)
    return out


def param_count(dims):
    return sum(dims[l + 1] * dims[l] + dims[l + 1] for l in range(len(dims) - 1))


def forward(theta, dims, x):
    """Returns (y, zs, acts): zs[l] pre-activations, acts[l] inputs of layer l."""
    layers = unpack(np.asarray(theta, np.float64), dims)
    a = np.asarray(x, np.float64)
    zs, acts = [], []
    for l, (W, b) in enumerate(layers):
        acts.append(a)
        z = a @ W.T + b
        zs.append(z)
        a = gelu(z) if l < len(layers) - 1 else z
    return a, zs, acts


def loss(theta, dims, x, t):
    """Mean over every output element of (y - t)^2."""
    y, _, _ = forward(theta, dims, x)
    return float(np.mean((y - np.asarray(t, np.float64)) ** 2))


def grad(theta, dims, x, t):
    """Gradient of `loss` with respect to theta, by the chain rule layer by layer."""
    layers = unpack(np.asarray(theta, np.float64), dims)
    y, zs, acts = forward(theta, dims, x)
    t = np.asarray(t, np.float64)
    delta = 2.0 * (y - t) / y.size          # dL/dz of the last (linear) layer
    g = []
    for l in range(len(layers) - 1, -1, -1):
        W, _ = layers[l]
        g.append((delta.sum(axis=0), delta.T @ acts[l]))   # (db, dW)
        if l > 0:
            delta = (delta @ W) * dgelu(zs[l - 1])
    flat = []
    for db, dW in reversed(g):
        flat.append(dW.ravel())
        flat.append(db)
    return np.concatenate(flat)


def adam_step(theta, g, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One step of Adam with bias correction; returns (theta, m, v)."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mhat = m / (1.0 - b1 ** step)
    vhat = v / (1.0 - b2 ** step)
    return theta - lr * mhat / (np.sqrt(vhat) + eps), m, v
