"""Pins of the FP64 reference network (oracle/mlp.py): central finite
differences of the loss against its reverse-mode gradient, and the layout."""
import numpy as np

from oracle import mlp


def test_param_count_and_layout():
    assert mlp.param_count() == 32 * 256 + 256 + 4 * (256 * 256 + 256)
    p = np.arange(mlp.param_count(), dtype=np.float64)
    (W0, b0) = mlp.unpack(p)[0]
    assert W0.shape == (32, 256) and W0[1, 0] == 256 and b0[0] == 32 * 256


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    p = rng.uniform(-1, 1, mlp.param_count()) / np.sqrt(256)
    x = rng.normal(size=(5, 32))
    t = rng.normal(size=(5, 256))
    loss, g = mlp.loss_and_grad(p, x, t)
    idx = rng.choice(mlp.param_count(), 40, replace=False)
    # include weights and biases of the first and last layers
    idx = np.concatenate([idx, [0, 32 * 256 + 3, mlp.param_count() - 1, mlp.param_count() - 300]])
    h = 1e-6
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (mlp.loss_and_grad(pp, x, t)[0] - mlp.loss_and_grad(pm, x, t)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])) + 1e-9, (i, fd, g[i])


def test_gelu_matches_its_definition():
    x = np.linspace(-5, 5, 101)
    from scipy.stats import norm
    assert np.allclose(mlp.gelu(x), x * norm.cdf(x), atol=1e-14)
    h = 1e-6
    assert np.allclose(mlp.gelu_grad(x), (mlp.gelu(x + h) - mlp.gelu(x - h)) / (2 * h), atol=1e-8)
