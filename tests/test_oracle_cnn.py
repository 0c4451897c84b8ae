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


# --------------------------------------------------------------------------- Adam (Kingma & Ba 2015)
def test_adam_first_step_closed_form():
    # at t = 1 the bias corrections undo the moment decay exactly:
    # m_hat = g, v_hat = g^2, so the step is lr g / (|g| + eps)
    rng = np.random.default_rng(3)
    w, g = rng.standard_normal(50), rng.standard_normal(50)
    w1, m1, v1 = cnn.adam_step(w, g, np.zeros(50), np.zeros(50), 1, 0.01)
    assert np.allclose(w1, w - 0.01 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    assert np.allclose(m1, 0.1 * g) and np.allclose(v1, 0.001 * g * g)


def test_adam_constant_gradient_moves_lr_per_step():
    # a constant gradient keeps m_hat = g and v_hat = g^2 at every step (the
    # corrections 1 - beta^t are exactly the weights the moments have
    # accumulated), so T steps move each parameter by T lr sign(g); a wrong
    # correction exponent or a missing correction fails this
    g = np.array([0.3, -2.0, 5e-3])
    w = np.zeros(3)
    m = v = np.zeros(3)
    for t in range(1, 31):
        w, m, v = cnn.adam_step(w, g, m, v, t, 0.05)
    assert np.allclose(w, -30 * 0.05 * np.sign(g) * np.abs(g) / (np.abs(g) + 1e-8), rtol=1e-12, atol=1e-13)


def test_adam_scale_invariance():
    # scaling every gradient by c > 0 leaves the steps unchanged (while |g| >> eps)
    rng = np.random.default_rng(4)
    gs = rng.standard_normal((5, 20))
    gs = np.sign(gs) * np.maximum(np.abs(gs), 0.1)         # |g| >= 0.1: eps / sqrt(v_hat) <= 1e-7
    w0 = wa = wb = rng.standard_normal(20)
    ma = va = mb = vb = np.zeros(20)
    for t in range(1, 6):
        wa, ma, va = cnn.adam_step(wa, gs[t - 1], ma, va, t, 0.02)
        wb, mb, vb = cnn.adam_step(wb, 37.0 * gs[t - 1], mb, vb, t, 0.02)
    assert np.allclose(wa, wb, rtol=0, atol=1e-7)
    assert np.abs(wa - w0).min() > 1e-3                    # the steps did move every parameter


def test_adam_two_step_worked_example():
    # w0 = (1, -2, 0.5), lr 0.1, g1 = (0.5, -1, 0), g2 = (-0.5, 2, 1), worked
    # out by hand to 30 digits:
    #   t = 1: m = (0.05, -0.1, 0), v = (2.5e-4, 1e-3, 0); m_hat = g1,
    #          v_hat = g1^2; w1 = (0.900000002, -1.900000001, 0.5)
    #   t = 2: m = (-0.005, 0.11, 0.1), v = (4.9975e-4, 4.999e-3, 1e-3);
    #          m_hat = m / 0.19, v_hat = v / 0.001999 = (0.25, 2.50075..., 0.50025...)
    #          w2 = w1 - 0.1 m_hat / (sqrt(v_hat) + 1e-8)
    w, m, v = cnn.adam_step([1.0, -2.0, 0.5], [0.5, -1.0, 0.0], np.zeros(3), np.zeros(3), 1, 0.1)
    assert np.allclose(w, [0.90000000199999996, -1.90000000099999999, 0.5], rtol=0, atol=1e-15)
    w, m, v = cnn.adam_step(w, [-0.5, 2.0, 1.0], m, v, 2, 0.1)
    assert np.allclose(m, [-0.005, 0.11, 0.1], rtol=0, atol=1e-15)
    assert np.allclose(v, [4.9975e-4, 4.999e-3, 1e-3], rtol=0, atol=1e-15)
    assert np.allclose(w, [0.905263159789473646, -1.936610353472075088, 0.425586318695406514], rtol=0, atol=1e-14)
