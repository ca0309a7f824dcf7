"""Pins of the oracle MLP (learned Newton start): GELU closed forms, gradient
against central differences, a dropped term is caught."""
import numpy as np

from oracle import mlp


def test_gelu_values():
    assert mlp.gelu(np.array([0.0]))[0] == 0.0
    assert abs(mlp.gelu(np.array([6.0]))[0] - 6.0) < 1e-7
    assert abs(mlp.gelu(np.array([-6.0]))[0]) < 1e-7
    assert abs(mlp.gelu_grad(np.array([0.0]))[0] - 0.5) < 1e-15
    x = np.linspace(-3, 3, 13)
    h = 1e-6
    fd = (mlp.gelu(x + h) - mlp.gelu(x - h)) / (2 * h)
    assert np.abs(fd - mlp.gelu_grad(x)).max() < 1e-8


def test_gradient_fd():
    rng = np.random.default_rng(0)
    shp = mlp.shapes(7, 16, 3, 5)
    P = mlp.nparams(7, 16, 3, 5)
    p = rng.standard_normal(P) * 0.3
    X = rng.standard_normal((11, 7))
    Y = rng.standard_normal((11, 5))
    norm = np.concatenate([rng.standard_normal(7) * 0.1, 1 + rng.random(7), rng.standard_normal(5) * 0.1, 1 + rng.random(5)])
    L, g = mlp.loss_grad(p, shp, X, Y, norm)
    h = 1e-6
    idx = rng.choice(P, 60, replace=False)
    for k in idx:
        e = np.zeros(P)
        e[k] = h
        fd = (mlp.loss_grad(p + e, shp, X, Y, norm)[0] - mlp.loss_grad(p - e, shp, X, Y, norm)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(fd)), (k, fd, g[k])


def test_prediction_units():
    rng = np.random.default_rng(1)
    shp = mlp.shapes(3, 8, 2, 2)
    p = np.zeros(mlp.nparams(3, 8, 2, 2))
    norm = np.array([0, 0, 0, 1, 1, 1, 5.0, -2.0, 3.0, 4.0])
    out = mlp.predict(p, shp, rng.standard_normal((4, 3)), norm)
    assert np.allclose(out, [5.0, -2.0])      # zero network -> y_mean
