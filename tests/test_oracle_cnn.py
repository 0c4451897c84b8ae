"""Pins of the FP64 warm-start network reference (oracle/cnn.py)."""
import numpy as np
import pytest
from scipy.signal import correlate2d

from oracle import cnn
from oracle import geometry as geo


def test_conv_matches_scipy_correlate():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((2, 3, 7, 7))
    W = rng.standard_normal((4, 3, 3, 3))
    b = rng.standard_normal(4)
    y = cnn.conv3x3(x, W, b)
    for bb in range(2):
        for co in range(4):
            ref = b[co] + sum(correlate2d(x[bb, ci], W[co, ci], mode="same", boundary="fill") for ci in range(3))
            assert np.allclose(y[bb, co], ref, atol=1e-12)


def _problem(seed=1, n=6, eps=0.2, n_gs=2, hidden=3, B=2):
    rng = np.random.default_rng(seed)
    nv = int(geo.subaperture_mask(n, eps).sum())
    NP = 2 * n_gs
    npar = sum(co * ci * 9 + co for (co, ci) in cnn.layer_shapes(NP, hidden))
    params = rng.standard_normal(npar) * 0.4
    s = rng.standard_normal((B, NP * nv))
    t = rng.standard_normal((B, NP * nv))
    return params, s, t, n, eps, hidden


def test_gradient_matches_finite_differences():
    params, s, t, n, eps, hidden = _problem()
    loss, g = cnn.loss_and_grad(params, s, t, n, eps, hidden, 0.7, 1.3)
    rng = np.random.default_rng(2)
    idx = rng.choice(len(params), 40, replace=False)
    h = 1e-6
    for i in idx:
        e = np.zeros_like(params)
        e[i] = h
        lp, _ = cnn.loss_and_grad(params + e, s, t, n, eps, hidden, 0.7, 1.3)
        lm, _ = cnn.loss_and_grad(params - e, s, t, n, eps, hidden, 0.7, 1.3)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_identity_network_is_relu():
    # centre-tap identity kernels, zero biases: each layer copies its input, the
    # ReLUs clip negatives, so zeta_0 = out_scale * in_scale * max(s, 0)
    n, eps, n_gs = 6, 0.2, 2
    NP = 2 * n_gs
    hidden = NP
    params = []
    for (co, ci) in cnn.layer_shapes(NP, hidden):
        W = np.zeros((co, ci, 3, 3))
        for c in range(min(co, ci)):
            W[c, c, 1, 1] = 1.0
        params += [W.ravel(), np.zeros(co)]
    params = np.concatenate(params)
    nv = int(geo.subaperture_mask(n, eps).sum())
    s = np.random.default_rng(4).standard_normal((3, NP * nv))
    z, _ = cnn.forward(params, s, n, eps, hidden, 0.5, 3.0)
    assert np.allclose(z, 1.5 * np.maximum(s, 0.0), atol=1e-14)


def test_hybrid_input_gradient_matches_finite_differences():
    params, s, t, n, eps, hidden = _problem(seed=6)
    rng = np.random.default_rng(7)
    pre = rng.standard_normal(s.shape)
    NP = 4
    npar = sum(co * ci * 9 + co for (co, ci) in zip([hidden, hidden, hidden, NP], [2 * NP, hidden, hidden, hidden]))
    params = rng.standard_normal(npar) * 0.3
    loss, g = cnn.loss_and_grad(params, s, t, n, eps, hidden, 0.7, 1.3, pre)
    for i in rng.choice(len(params), 25, replace=False):
        e = np.zeros_like(params)
        e[i] = 1e-6
        fd = (cnn.loss_and_grad(params + e, s, t, n, eps, hidden, 0.7, 1.3, pre)[0]
              - cnn.loss_and_grad(params - e, s, t, n, eps, hidden, 0.7, 1.3, pre)[0]) / 2e-6
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd))
