"""Pins for the MLP oracle used to check the learned-initial-guess kernels.

Gradients are checked against central finite differences of the loss (a
plain definition of the derivative), Adam's first step against its closed form
(lr * g / (|g| + eps) per component), and the forward pass against a
hand-evaluated one-hidden-unit network.
"""
import numpy as np

from oracle import mlp


def _setup(seed=0, n_in=8, width=6, depth=2, n_out=3, n=11):
    rng = np.random.default_rng(seed)
    shapes = mlp.layer_shapes(n_in, width, depth, n_out)
    n_par = sum(a * b + b for a, b in shapes)
    theta = rng.standard_normal(n_par) * 0.5
    X = rng.standard_normal((n, n_in))
    Y = rng.standard_normal((n, n_out))
    shift = rng.standard_normal(n_in) * 0.1
    scale = 1.0 + rng.random(n_in)
    out_scale = np.array([0.5, 2.0, 1.5])[:n_out]
    return shapes, theta, X, Y, shift, scale, out_scale


def test_gradient_matches_central_differences():
    shapes, theta, X, Y, shift, scale, out_scale = _setup()
    loss, g = mlp.loss_and_grad(theta, shapes, X, Y, shift, scale, out_scale)
    h = 1e-6
    num = np.empty_like(theta)
    for k in range(theta.size):
        e = np.zeros_like(theta)
        e[k] = h
        lp, _ = mlp.loss_and_grad(theta + e, shapes, X, Y, shift, scale, out_scale)
        lm, _ = mlp.loss_and_grad(theta - e, shapes, X, Y, shift, scale, out_scale)
        num[k] = (lp - lm) / (2 * h)
    np.testing.assert_allclose(g, num, rtol=1e-6, atol=1e-9)


def test_forward_of_a_hand_evaluated_network():
    # one input, one tanh unit, one output: y = s_out * (w2 tanh(w1 (x - c) k + b1) + b2)
    shapes = mlp.layer_shapes(1, 1, 1, 1)
    w1, b1, w2, b2 = 0.7, -0.2, 1.3, 0.4
    theta = np.array([w1, b1, w2, b2])
    x = np.array([[0.9]])
    y, _ = mlp.forward(theta, shapes, x, np.array([0.1]), np.array([2.0]), np.array([3.0]))
    expect = 3.0 * (w2 * np.tanh(w1 * (0.9 - 0.1) * 2.0 + b1) + b2)
    assert abs(y[0, 0] - expect) < 1e-15


def test_node_features_recover_a_linear_temperature_gradient():
    # for T linear in x the interpolant is exact (P1 and P2): grad T is the constant vector
    from paper_1804_10060_gb300 import meshgen
    for degree in (1, 2):
        coords, cells = meshgen.box_kuhn(3, 2, 2, 1.5, 1.0, 1.0)
        coords = meshgen.jitter_interior(coords, 0.3, 0.2, 4)
        if degree == 2:
            coords, cells, _ = meshgen.p1_to_p2(coords, cells)
        a = np.array([0.3, -1.2, 2.5])
        T = 7.0 + coords @ a
        F = mlp.node_features(coords, cells, T, dist=coords[:, 0])
        np.testing.assert_allclose(F[:, 4:7], np.tile(a, (coords.shape[0], 1)), rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(F[:, 3], T)
        np.testing.assert_allclose(F[:, 7], coords[:, 0])


def test_node_features_p2_quadratic_centroid_gradient():
    # T = x^2 on one P2 cell: grad T_h at the centroid is (2 x_c, 0, 0) exactly
    from paper_1804_10060_gb300 import meshgen
    X = np.array([[0.0, 0, 0], [1.0, 0, 0], [0, 1.0, 0], [0, 0, 1.0]]) * 0.8 + 0.3
    coords, cells, _ = meshgen.p1_to_p2(X, np.array([[0, 1, 2, 3]]))
    T = coords[:, 0] ** 2
    F = mlp.node_features(coords, cells, T)
    xc = X[:, 0].mean()
    np.testing.assert_allclose(F[:, 4], 2 * xc, rtol=1e-12)
    np.testing.assert_allclose(F[:, 5:7], 0.0, atol=1e-12)


def test_first_adam_step_closed_form():
    rng = np.random.default_rng(1)
    theta = rng.standard_normal(20)
    g = rng.standard_normal(20)
    t1, m, v = mlp.adam_step(theta, g, np.zeros(20), np.zeros(20), 1, lr=0.01)
    # bias-corrected m = g, v = g^2  =>  step = lr * g / (|g| + eps)
    np.testing.assert_allclose(theta - t1, 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)
