"""FP64 reference of the warm-start network (oracle; test infrastructure only).

The network is the library's addition (the paper's solvers start from zero or
the previous estimate, Sec. 5): per frame, the 2 nGS slope planes on the n x n
subaperture grid (slopes * in_scale at valid subapertures, 0 elsewhere) go
through 3 x 3 convolutions (zero padding) 2nGS -> H -> H -> H -> 2nGS with
ReLU after the first three; zeta_0 = out_scale * output at the valid
subapertures.  Parameters are one vector: per layer W [Cout][Cin][3][3], b [Cout].
Loss: ||zeta_0 - t||^2 / ||t||^2 over the batch.

Everything is written out with numpy loops over the 9 taps; gradients are the
plain chain rule.  Pinned by tests/test_oracle_cnn.py (scipy correlate2d,
central finite differences).

Training uses Adam (Kingma & Ba, "Adam: a method for stochastic
optimization", ICLR 2015, Algorithm 1); ``adam_step`` is that algorithm's
update written out in FP64, pinned by tests/test_oracle_cnn.py (closed forms
for the first step and for a constant gradient, scale invariance, and a
worked two-step example).
"""

import numpy as np

from . import geometry as geo


def layer_shapes(n_planes, hidden):
    ch = [n_planes, hidden, hidden, hidden, n_planes]
    return [(ch[l + 1], ch[l]) for l in range(4)]


def unpack(params, n_planes, hidden):
    out, off = [], 0
    for (co, ci) in layer_shapes(n_planes, hidden):
        W = params[off:off + co * ci * 9].reshape(co, ci, 3, 3)
        off += co * ci * 9
        b = params[off:off + co]
        off += co
        out.append((W, b))
    assert off == len(params)
    return out


def conv3x3(x, W, b):
    """y[b, co, i, j] = b[co] + sum_ci sum_{di,dj} W[co, ci, di+1, dj+1] x[b, ci, i+di, j+dj] (zero padding)."""
    B, Cin, n, _ = x.shape
    xp = np.zeros((B, Cin, n + 2, n + 2))
    xp[:, :, 1:-1, 1:-1] = x
    y = np.zeros((B, W.shape[0], n, n)) + b[None, :, None, None]
    for di in range(3):
        for dj in range(3):
            patch = xp[:, :, di:di + n, dj:dj + n]                    # x[b, ci, i+di-1, j+dj-1]
            y += np.einsum("oc,bcij->boij", W[:, :, di, dj], patch)
    return y


def to_grid(vec, n, mask):
    """[B][NP * n_vs] valid entries -> [B][NP][n][n] grids."""
    B = vec.shape[0]
    nv = int(mask.sum())
    NP = vec.shape[1] // nv
    g = np.zeros((B, NP, n, n))
    g[:, :, mask] = vec.reshape(B, NP, nv)
    return g


def from_grid(g, mask):
    B, NP = g.shape[:2]
    return g[:, :, mask].reshape(B, -1)


def unpack_any(params, cin, cout, hidden):
    ch = [cin, hidden, hidden, hidden, cout]
    out, off = [], 0
    for l in range(4):
        co, ci = ch[l + 1], ch[l]
        W = params[off:off + co * ci * 9].reshape(co, ci, 3, 3)
        off += co * ci * 9
        out.append((W, params[off:off + co]))
        off += co
    assert off == len(params)
    return out


def forward(params, slopes, n, obstruction, hidden, in_scale, out_scale, pre=None, pre_gain=1.0):
    """Returns (zeta_0 [B][N], activations) in FP64.

    With ``pre`` (the preconditioner estimate M^{-1} s, [B][N]) the input grid
    has the extra planes pre / out_scale and zeta_0 = pre_gain pre + out_scale * output.
    """
    mask = geo.subaperture_mask(n, obstruction)
    NP = slopes.shape[1] // int(mask.sum())
    grid = to_grid(np.asarray(slopes, np.float64) * in_scale, n, mask)
    if pre is not None:
        grid = np.concatenate([grid, to_grid(np.asarray(pre, np.float64) / out_scale, n, mask)], axis=1)
    layers = unpack_any(np.asarray(params, np.float64), grid.shape[1], NP, hidden)
    acts = [grid]
    for l, (W, b) in enumerate(layers):
        y = conv3x3(acts[-1], W, b)
        if l < 3:
            y = np.maximum(y, 0.0)
        acts.append(y)
    z = out_scale * from_grid(acts[-1], mask)
    if pre is not None:
        z = z + pre_gain * np.asarray(pre, np.float64)
    return z, acts


def loss_and_grad(params, slopes, target, n, obstruction, hidden, in_scale, out_scale, pre=None, pre_gain=1.0):
    """Loss ||z - t||^2 / ||t||^2 and its gradient with respect to params (FP64)."""
    mask = geo.subaperture_mask(n, obstruction)
    z, acts = forward(params, slopes, n, obstruction, hidden, in_scale, out_scale, pre, pre_gain)
    NP = slopes.shape[1] // int(mask.sum())
    layers = unpack_any(np.asarray(params, np.float64), acts[0].shape[1], NP, hidden)
    t = np.asarray(target, np.float64)
    den = np.sum(t * t)
    loss = np.sum((z - t) ** 2) / den
    gz = 2.0 * (z - t) / den
    dy = out_scale * to_grid(gz, n, mask)
    grads = []
    for l in range(3, -1, -1):
        W, b = layers[l]
        if l < 3:
            dy = dy * (acts[l + 1] > 0)
        x = acts[l]
        B, Cin, _, _ = x.shape
        xp = np.zeros((B, Cin, n + 2, n + 2))
        xp[:, :, 1:-1, 1:-1] = x
        dW = np.zeros_like(W)
        for di in range(3):
            for dj in range(3):
                dW[:, :, di, dj] = np.einsum("boij,bcij->oc", dy, xp[:, :, di:di + n, dj:dj + n])
        db = dy.sum(axis=(0, 2, 3))
        grads.append((dW, db))
        # dx[b, ci, i, j] = sum_co sum_taps W[co, ci, di, dj] dy[b, co, i - (di-1), j - (dj-1)]
        dyp = np.zeros((B, W.shape[0], n + 2, n + 2))
        dyp[:, :, 1:-1, 1:-1] = dy
        dx = np.zeros_like(x)
        for di in range(3):
            for dj in range(3):
                dx += np.einsum("oc,boij->bcij", W[:, :, di, dj], dyp[:, :, 2 - di:2 - di + n, 2 - dj:2 - dj + n])
        dy = dx
    flat = []
    for (dW, db) in reversed(grads):
        flat.append(dW.ravel())
        flat.append(db)
    return loss, np.concatenate(flat)


def adam_step(w, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015, Algorithm 1) at step t >= 1, FP64.

    First and second moment estimates m <- beta1 m + (1 - beta1) g and
    v <- beta2 v + (1 - beta2) g^2, their bias-corrected values
    m / (1 - beta1^t) and v / (1 - beta2^t), and the parameter step
    w <- w - lr m_hat / (sqrt(v_hat) + eps).  Returns (w, m, v); the inputs
    are not modified."""
    w = np.asarray(w, np.float64)
    g = np.asarray(g, np.float64)
    m = beta1 * np.asarray(m, np.float64) + (1.0 - beta1) * g
    v = beta2 * np.asarray(v, np.float64) + (1.0 - beta2) * g * g
    m_hat = m / (1.0 - beta1 ** t)
    v_hat = v / (1.0 - beta2 ** t)
    return w - lr * m_hat / (np.sqrt(v_hat) + eps), m, v
