"""Pins of the oracle's FP64 MLP reference (oracle/mlp.py), which checks the
learned part's BF16 kernels, against facts that do not come from it:

* the hand-written backpropagation equals central finite differences of the
  loss, for every parameter;
* with non-negative inputs, weights and biases no ReLU clips, so the network
  is the product of its affine maps and the loss has a closed form;
* the output layer is linear (no ReLU);
* the flat parameter layout of the C interface (per layer W[in][out], b[out]).
"""
import numpy as np

from oracle import mlp as omlp

SIZES = [(4, 6), (6, 5), (5, 3)]


def n_params(sizes):
    return sum(i * o + o for i, o in sizes)


def test_gradient_equals_central_differences():
    rng = np.random.default_rng(11)
    p = rng.normal(0.0, 0.5, n_params(SIZES))
    X = rng.normal(0.0, 1.0, (9, 4))
    T = rng.normal(0.0, 1.0, (9, 3))
    _, g = omlp.loss_and_grad(p, SIZES, X, T)
    h = 1e-6
    fd = np.empty_like(p)
    for k in range(p.size):
        e = np.zeros_like(p)
        e[k] = h
        fd[k] = (omlp.loss_and_grad(p + e, SIZES, X, T)[0]
                 - omlp.loss_and_grad(p - e, SIZES, X, T)[0]) / (2 * h)
    assert np.abs(g - fd).max() < 1e-7 * max(1.0, np.abs(g).max())


def test_unclipped_network_is_a_product_of_affine_maps():
    rng = np.random.default_rng(12)
    p = rng.uniform(0.0, 0.5, n_params(SIZES))
    X = rng.uniform(0.0, 1.0, (7, 4))
    T = rng.normal(0.0, 1.0, (7, 3))
    (W1, b1), (W2, b2), (W3, b3) = omlp.unflatten(p, SIZES)
    Y = np.linalg.multi_dot([X, W1, W2, W3]) + (b1 @ W2 @ W3 + b2 @ W3 + b3)
    loss, _ = omlp.loss_and_grad(p, SIZES, X, T)
    assert abs(loss - np.mean((Y - T) ** 2)) < 1e-13


def test_output_layer_is_linear():
    p = np.zeros(n_params(SIZES))
    p[-3:] = [-5.0, 0.0, 2.0]                 # output biases, all weights zero
    X = np.ones((2, 4))
    T = np.zeros((2, 3))
    loss, g = omlp.loss_and_grad(p, SIZES, X, T)
    assert abs(loss - (25.0 + 0.0 + 4.0) / 3.0) < 1e-14
    # d loss / d b_out = 2 (Y - T) summed over rows / n = 2 * 2 * b / 6
    assert np.allclose(g[-3:], [-10.0 / 3.0, 0.0, 4.0 / 3.0], atol=1e-14)


def test_flat_parameter_layout():
    p = np.arange(n_params(SIZES), dtype=np.float64)
    (W1, b1), (W2, b2), _ = omlp.unflatten(p, SIZES)
    assert W1.shape == (4, 6) and W1[0, 1] == 1.0 and W1[1, 0] == 6.0
    assert b1[0] == 24.0 and W2[0, 0] == 30.0 and b2[0] == 60.0
