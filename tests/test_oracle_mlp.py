"""Pins of the oracle MLP: back-propagated gradients against central finite differences."""
import numpy as np

from oracle import mlp
from paper_2512_13550_gb300 import inputs


def test_mlp_gradient_matches_finite_differences():
    F, H, O, B = 5, 7, 2, 11
    theta = mlp.init(F, H, O, seed=3) + 0.05 * inputs.normal(9, mlp.count(F, H, O))
    X = inputs.normal(10, B * F).reshape(B, F)
    T = inputs.normal(11, B * O).reshape(B, O)
    loss, g = mlp.loss_and_grad(theta, X, T, F, H, O)
    eps = 1e-6
    for k in range(0, theta.size, 3):
        e = np.zeros_like(theta)
        e[k] = eps
        fd = (mlp.loss_and_grad(theta + e, X, T, F, H, O)[0] - mlp.loss_and_grad(theta - e, X, T, F, H, O)[0]) / (2 * eps)
        assert abs(fd - g[k]) < 1e-6 * max(1.0, abs(fd))


def test_mlp_forward_shapes_and_relu():
    F, H = 3, 4
    theta = np.zeros(mlp.count(F, H))
    theta[-1] = 0.7  # b3
    Y, (Z1, A1, Z2, A2) = mlp.forward(theta, np.ones((2, F)), F, H)
    np.testing.assert_allclose(Y, 0.7)
    assert A1.min() >= 0 and A2.min() >= 0
