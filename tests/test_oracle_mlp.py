"""Pins of the oracle MLP (learned Newton start): GELU closed forms, gradient
against central differences, the network's closed form in the affine regime of GELU
(standardisation, packing and layer order), the zero network."""
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


def test_affine_regime_closed_form():
    """With every pre-activation >= 10, GELU(z) = z (1 + erf(z / sqrt 2)) / 2 equals z in FP64
    (1 - erf(10 / sqrt 2) ~ 1.5e-23), so the network is the composition of its affine maps:
    y = y_std * (W_L(...(W_1 h + b_1)...) + b_L) + y_mean with h = (x - x_mean) / x_std and the
    parameters packed per layer as W[out][in] row-major, then b[out]."""
    rng = np.random.default_rng(2)
    n_in, width, depth, n_out = 3, 5, 3, 2
    shp = mlp.shapes(n_in, width, depth, n_out)
    layers = [(rng.uniform(0.1, 0.5, (o, i)), np.full(o, 10.0) + rng.random(o)) for o, i in shp]
    p = np.concatenate([np.concatenate([W.ravel(), b]) for W, b in layers])
    assert p.size == mlp.nparams(n_in, width, depth, n_out)
    xm, xs = rng.standard_normal(n_in), 1.0 + rng.random(n_in)
    ym, ys = rng.standard_normal(n_out), 1.0 + rng.random(n_out)
    norm = np.concatenate([xm, xs, ym, ys])
    X = xm + xs * rng.uniform(0.0, 1.0, (6, n_in))          # standardised inputs in [0, 1]
    h = (X - xm) / xs
    for W, b in layers:
        h = np.array([[sum(W[o, i] * row[i] for i in range(W.shape[1])) + b[o] for o in range(W.shape[0])]
                      for row in h])
    expect = h * ys + ym
    got = mlp.predict(p, shp, X, norm)
    assert np.abs(got - expect).max() <= 1e-13 * np.abs(expect).max()
