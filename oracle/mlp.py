"""ORACLE — test infrastructure only.

Plain FP64 reference of the learned Newton-start network (an addition to
the method; the paper is silent on the Newton predictor): a multilayer
perceptron with exact-erf GELU, inputs standardised by (x - x_mean)/x_std,
trained on the mean squared error of standardised targets (y - y_mean)/y_std.
Parameters are packed per linear map as W[out][in] row-major then b[out].
Forward and backward are written layer by layer with numpy (no autograd).
"""
import numpy as np
from scipy.special import erf


def shapes(n_in, width, depth, n_out):
    dims = [n_in] + [width] * depth + [n_out]
    return [(dims[l + 1], dims[l]) for l in range(depth + 1)]


def nparams(n_in, width, depth, n_out):
    return sum(o * i + o for o, i in shapes(n_in, width, depth, n_out))


def unpack(p, shp):
    out, k = [], 0
    for o, i in shp:
        W = p[k:k + o * i].reshape(o, i)
        k += o * i
        b = p[k:k + o]
        k += o
        out.append((W, b))
    return out


def gelu(x):
    return 0.5 * x * (1.0 + erf(x / np.sqrt(2.0)))


def gelu_grad(x):
    return 0.5 * (1.0 + erf(x / np.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / np.sqrt(2.0 * np.pi)


def forward(p, shp, X, norm):
    """raw features X [N, n_in] -> standardised outputs [N, n_out], caches"""
    n_in = shp[0][1]
    n_out = shp[-1][0]
    xm, xs = norm[:n_in], norm[n_in:2 * n_in]
    h = (X - xm) / xs
    layers = unpack(np.asarray(p, np.float64), shp)
    cache = [h]
    zs = []
    for l, (W, b) in enumerate(layers):
        z = h @ W.T + b
        zs.append(z)
        h = gelu(z) if l < len(layers) - 1 else z
        cache.append(h)
    return h, (cache, zs, layers)


def predict(p, shp, X, norm):
    n_in, n_out = shp[0][1], shp[-1][0]
    ym, ys = norm[2 * n_in:2 * n_in + n_out], norm[2 * n_in + n_out:]
    out, _ = forward(p, shp, X, norm)
    return out * ys + ym


def loss_grad(p, shp, X, Y, norm):
    """MSE of standardised targets and its gradient w.r.t. the packed parameters"""
    n_in, n_out = shp[0][1], shp[-1][0]
    ym, ys = norm[2 * n_in:2 * n_in + n_out], norm[2 * n_in + n_out:]
    out, (cache, zs, layers) = forward(p, shp, X, norm)
    t = (Y - ym) / ys
    N = X.shape[0]
    r = out - t
    loss = np.mean(r * r)
    d = 2.0 * r / r.size
    grads = []
    for l in range(len(layers) - 1, -1, -1):
        W, b = layers[l]
        if l < len(layers) - 1:
            d = d * gelu_grad(zs[l])
        gW = d.T @ cache[l]
        gb = d.sum(0)
        grads.append((gW, gb))
        d = d @ W
    g = []
    for gW, gb in reversed(grads):
        g += [gW.ravel(), gb]
    return loss, np.concatenate(g)
