"""Plain FP64 reference of the troubled-cell MLP (test infrastructure only).

The network classifies a cell as troubled from 44 features: for each of the 4
conservative components, the 3x3 neighbourhood of cell averages normalised by the
stencil's mean and by the larger of its range and the TVB threshold, and the cell's
two first Legendre moments (x and y slopes) normalised the same way.  Architecture 44 -> 64 -> 64 -> 1, ReLU,
sigmoid output, binary cross-entropy loss, Adam updates.  Everything below is
written out with numpy array operations in FP64; no part of it is shared with
the CUDA kernels.

Parameter vector layout (7105 values): W1[64][44], b1[64], W2[64][64], b2[64],
w3[64], b3[1].
"""
from __future__ import annotations

import numpy as np

NIN, NH = 44, 64
SIZES = [("W1", (NH, NIN)), ("b1", (NH,)), ("W2", (NH, NH)), ("b2", (NH,)), ("w3", (NH,)), ("b3", (1,))]
NPARAM = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(theta):
    out, o = {}, 0
    for name, shape in SIZES:
        k = int(np.prod(shape))
        out[name] = theta[o:o + k].reshape(shape)
        o += k
    return out


def pack(parts):
    return np.concatenate([np.asarray(parts[name], dtype=np.float64).reshape(-1) for name, _ in SIZES])


def init_params(seed=0):
    """He-uniform weights, zero biases."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, shape in SIZES:
        if name.startswith("b"):
            p[name] = np.zeros(shape)
        else:
            fan_in = shape[-1] if len(shape) == 2 else NH
            lim = np.sqrt(6.0 / fan_in)
            p[name] = rng.uniform(-lim, lim, shape)
    return pack(p)


def features(avg3x3, slopes, thr=0.0):
    """avg3x3: [..., 4, 9] cell averages of the 3x3 stencil (row-major, centre = 4);
    slopes: [..., 4, 2] the centre cell's first Legendre moments (c_x, c_y);
    thr: the TVB threshold M hx hy of the mesh.
    Returns [..., 44]: per component (v - mean) / den, then the slopes / den, with
    den = max(range, thr) + delta and delta = 1e-6 max|v| + 1e-30.  The threshold floor
    keeps deviations below the TVB threshold below 1 (the plain indicator cannot flag
    them); delta maps flat stencils to features near 0 instead of rounding noise."""
    avg3x3 = np.asarray(avg3x3, dtype=np.float64)
    slopes = np.asarray(slopes, dtype=np.float64)
    mean = avg3x3.mean(axis=-1, keepdims=True)
    rng_ = avg3x3.max(axis=-1, keepdims=True) - avg3x3.min(axis=-1, keepdims=True)
    delta = 1e-6 * np.abs(avg3x3).max(axis=-1, keepdims=True) + 1e-30
    den = np.maximum(rng_, thr) + delta
    z = (avg3x3 - mean) / den
    s = slopes / den
    lead = avg3x3.shape[:-2]
    return np.concatenate([z.reshape(lead + (36,)), s.reshape(lead + (8,))], axis=-1)


def forward(theta, X):
    """logits z and the activations needed by backward"""
    p = unpack(theta)
    a1 = X @ p["W1"].T + p["b1"]
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.maximum(a2, 0.0)
    z = h2 @ p["w3"] + p["b3"][0]
    return z, (X, a1, h1, a2, h2)


def sigmoid(z):
    return np.where(z >= 0, 1.0 / (1.0 + np.exp(-np.abs(z))), np.exp(-np.abs(z)) / (1.0 + np.exp(-np.abs(z))))


def bce(z, y):
    """mean binary cross-entropy from logits: softplus(z) - y z"""
    return float(np.mean(np.maximum(z, 0.0) + np.log1p(np.exp(-np.abs(z))) - y * z))


def loss(theta, X, y):
    z, _ = forward(theta, X)
    return bce(z, y)


def backward(theta, X, y):
    """gradient of the mean BCE with respect to the parameter vector (FP64)"""
    p = unpack(theta)
    z, (X, a1, h1, a2, h2) = forward(theta, X)
    B = X.shape[0]
    dz = (sigmoid(z) - y) / B
    g = {}
    g["w3"] = h2.T @ dz
    g["b3"] = np.array([dz.sum()])
    dh2 = np.outer(dz, p["w3"]) * (a2 > 0)
    g["W2"] = dh2.T @ h1
    g["b2"] = dh2.sum(axis=0)
    dh1 = (dh2 @ p["W2"]) * (a1 > 0)
    g["W1"] = dh1.T @ X
    g["b1"] = dh1.sum(axis=0)
    return pack(g)


def adam(theta, m, v, grad, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """one Adam step (Kingma & Ba); t is the 1-based step count"""
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
