"""CPU pins of the FP64 surrogate-network reference (oracle/mlp_ref.py):
GELU and its derivative against independent values, the backpropagated
gradient against central finite differences of the loss, and Adam's first
step against its closed form."""
import math

import numpy as np
import pytest

from oracle import mlp_ref as R


def test_gelu_special_values():
    # z Phi(z): Phi(0) = 1/2, Phi(1) = 0.8413447460685429 (normal table); z (Phi(z) - 1/2) is even
    assert R.gelu(np.array([0.0]))[0] == 0.0
    assert abs(R.gelu(np.array([1.0]))[0] - 0.8413447460685429) < 1e-15
    z = np.linspace(-4, 4, 33)
    assert np.allclose(R.gelu(z) - z / 2, R.gelu(-z) + z / 2, atol=1e-15)
    assert np.allclose(R.gelu(np.array([40.0, -40.0])), [40.0, 0.0])


def test_dgelu_matches_finite_difference():
    z = np.linspace(-5, 5, 41)
    h = 1e-5
    fd = (R.gelu(z + h) - R.gelu(z - h)) / (2 * h)
    assert np.max(np.abs(fd - R.dgelu(z))) < 1e-9


@pytest.mark.parametrize("dims", [[4, 8, 8, 3], [2, 5, 1], [4, 6, 6, 6, 6, 7]])
def test_gradient_matches_central_differences(dims):
    rng = np.random.default_rng(11)
    n = R.param_count(dims)
    theta = rng.normal(0, 0.7, n)
    x = rng.uniform(-1, 1, (5, dims[0]))
    t = rng.normal(0, 1, (5, dims[-1]))
    g = R.grad(theta, dims, x, t)
    h = 1e-6
    fd = np.empty(n)
    for i in range(n):
        e = np.zeros(n)
        e[i] = h
        fd[i] = (R.loss(theta + e, dims, x, t) - R.loss(theta - e, dims, x, t)) / (2 * h)
    assert np.max(np.abs(fd - g)) <= 1e-7 * max(1.0, np.max(np.abs(g)))


def test_linear_network_gradient_closed_form():
    # one affine layer: y = x W^T + b, L = mean (y - t)^2 -> dW = 2/(B N) (y - t)^T x
    rng = np.random.default_rng(3)
    dims = [3, 2]
    theta = rng.normal(size=R.param_count(dims))
    x = rng.normal(size=(4, 3))
    t = rng.normal(size=(4, 2))
    W, b = theta[:6].reshape(2, 3), theta[6:]
    r = x @ W.T + b - t
    want = np.concatenate([(2 / 8 * r.T @ x).ravel(), 2 / 8 * r.sum(0)])
    assert np.allclose(R.grad(theta, dims, x, t), want, rtol=1e-14, atol=1e-15)


def test_adam_first_step_is_signed_lr():
    # step 1: mhat = g, vhat = g^2 -> update = -lr g / (|g| + eps)
    g = np.array([3.0, -0.5, 1e-3, 0.0])
    th, m, v = R.adam_step(np.zeros(4), g, np.zeros(4), np.zeros(4), 1, 0.01)
    assert np.allclose(th, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-15)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)
    # constant gradient: mhat = g at every step
    th, m, v = np.zeros(1), np.zeros(1), np.zeros(1)
    for s in range(1, 6):
        th, m, v = R.adam_step(th, np.array([2.0]), m, v, s, 0.1)
    assert math.isclose(th[0], -0.5 * 2.0 / (2.0 + 1e-8), rel_tol=1e-12)
