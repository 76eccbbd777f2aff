"""Pins of the FP64 reference network: GELU against its definition and the
chain-rule gradient against central differences."""
import numpy as np
from scipy.integrate import quad

from oracle import mlp


def test_gelu_is_x_times_normal_cdf():
    for x in (-3.0, -0.7, 0.0, 0.4, 2.5):
        cdf = quad(lambda t: np.exp(-0.5 * t * t) / np.sqrt(2 * np.pi), -np.inf, x)[0]
        assert abs(mlp.gelu(x) - x * cdf) < 1e-12
        h = 1e-6
        assert abs(mlp.gelu_grad(x) - (mlp.gelu(x + h) - mlp.gelu(x - h)) / (2 * h)) < 1e-8


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(0)
    theta = rng.standard_normal(mlp.NPARAM) * 0.2
    norm = np.concatenate([rng.standard_normal(16), rng.uniform(0.5, 2, 16), rng.standard_normal(2),
                           rng.uniform(0.5, 2, 2)])
    X = rng.standard_normal((13, 16))
    T = rng.standard_normal((13, 2))
    loss, g = mlp.loss_and_grad(theta, norm, X, T)
    idx = rng.choice(mlp.NPARAM, 40, replace=False)
    for k in idx:
        e = np.zeros(mlp.NPARAM)
        e[k] = 1e-6
        fd = (mlp.loss_and_grad(theta + e, norm, X, T)[0] - mlp.loss_and_grad(theta - e, norm, X, T)[0]) / 2e-6
        assert abs(fd - g[k]) < 1e-7 * max(1.0, abs(g[k])) + 1e-9, (k, fd, g[k])
