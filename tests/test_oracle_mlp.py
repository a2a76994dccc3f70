"""Pins of the FP64 reference MLP (troubled-cell classifier): finite-difference gradients,
closed forms of the loss, invariances and the threshold floor of the features, and learning a separable set."""
import numpy as np

from oracle import mlp


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(0)
    theta = mlp.init_params(1)
    X = rng.normal(size=(16, mlp.NIN))
    y = (rng.uniform(size=16) > 0.5).astype(float)
    g = mlp.backward(theta, X, y)
    idx = rng.choice(mlp.NPARAM, 60, replace=False)
    for i in idx:
        e = np.zeros(mlp.NPARAM)
        h = 1e-6
        e[i] = h
        fd = (mlp.loss(theta + e, X, y) - mlp.loss(theta - e, X, y)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_bce_closed_forms():
    z = np.array([0.0, 2.0, -3.0, 40.0, -40.0])
    y = np.array([1.0, 0.0, 1.0, 1.0, 0.0])
    ref = [np.log(2.0), np.log(1 + np.exp(2.0)), np.log(1 + np.exp(3.0)), 0.0, 0.0]
    for zi, yi, ri in zip(z, y, ref):
        assert abs(mlp.bce(np.array([zi]), np.array([yi])) - ri) < 1e-12
    assert np.allclose(mlp.sigmoid(np.array([0.0, 800.0, -800.0])), [0.5, 1.0, 0.0])


def test_features_scale_shift_and_threshold():
    rng = np.random.default_rng(2)
    a = rng.uniform(0.5, 2.0, size=(3, 4, 9))
    s = rng.normal(size=(3, 4, 2))
    f = mlp.features(a, s)
    assert f.shape == (3, 44)
    # scaling values, slopes and threshold together leaves the features unchanged
    assert np.allclose(mlp.features(7.0 * a, 7.0 * s, 7.0 * 0.01), mlp.features(a, s, 0.01), rtol=0, atol=1e-12)
    # a shift changes only delta = 1e-6 max|v|
    assert np.allclose(mlp.features(a + 3.0, s), f, rtol=0, atol=1e-5)
    # without a threshold: z spans exactly [.,.] of range 1 (up to delta)
    z = f[:, :36].reshape(3, 4, 9)
    assert np.allclose(z.max(-1) - z.min(-1), 1.0, rtol=0, atol=1e-5)
    # below the threshold: (v - mean) / (thr + delta), slopes likewise
    b = 1.0 + 1e-3 * rng.uniform(size=(4, 9))
    sb = 1e-3 * rng.normal(size=(4, 2))
    fb = mlp.features(b, sb, thr=0.05)
    den = 0.05 + 1e-6 * b.max(-1, keepdims=True)
    assert np.allclose(fb[:36].reshape(4, 9), (b - b.mean(-1, keepdims=True)) / den, rtol=1e-12, atol=0)
    assert np.allclose(fb[36:].reshape(4, 2), sb / den, rtol=1e-12, atol=0)
    assert np.abs(fb).max() < 0.05


def test_adam_learns_a_separable_set():
    rng = np.random.default_rng(3)
    X = rng.normal(size=(512, mlp.NIN))
    y = (X[:, 3] - 0.5 * X[:, 40] > 0).astype(float)
    theta = mlp.init_params(4)
    m = np.zeros_like(theta)
    v = np.zeros_like(theta)
    l0 = mlp.loss(theta, X, y)
    for t in range(1, 301):
        theta, m, v = mlp.adam(theta, m, v, mlp.backward(theta, X, y), t, lr=3e-3)
    assert mlp.loss(theta, X, y) < 0.1 * l0
    z, _ = mlp.forward(theta, X)
    assert np.mean((z > 0) == (y > 0.5)) > 0.97
