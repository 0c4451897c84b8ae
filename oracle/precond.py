"""FP64 reference of the block-circulant preconditioner (oracle; test infrastructure only).

The preconditioner is the library's addition (the paper runs its solvers
unpreconditioned and names preconditioning an open problem, Sec. 6).  Written
out plainly: the slope covariance of every plane pair is evaluated at every
lag of a P x P torus, Delta in [-P/2, P/2)^2 (periodised), from the same point
covariances as covariance.py (Hudgin two-point slopes, cone factor and
h_k (alpha_i - alpha_j) shift per layer); its 2-D FFT gives per frequency a
(2 nGS) x (2 nGS) matrix K(f), made Hermitian; eigenvalues are clamped at zero,
c sigma_g^2 is added on the diagonal, and the matrix is inverted:
    M^{-1} x = W_s IFFT2( (K_+(f) + c Sigma)^{-1} FFT2(W_s^T x) ).
numpy's FFT and eigh are the library steps.
"""

import numpy as np

from . import covariance as cov
from . import geometry as geo
from . import turbulence as turb


def periodised_generators(cfg, P):
    """t[p, q, di, dj] for lags di, dj in [-P/2, P/2) (array index lag + P/2)."""
    if not cov.uniform_grid(cfg):
        raise NotImplementedError("the block-circulant preconditioner needs one grid for all guide stars")
    n, D = cfg["n"], cfg["D"]
    d = D / n
    gs = cfg["gs"]
    NP = 2 * len(gs)
    lag = np.arange(-(P // 2), P - P // 2)
    LY, LX = np.meshgrid(lag, lag, indexing="ij")
    t = np.zeros((NP, NP, P, P))
    for p in range(NP):
        for q in range(NP):
            gi, ci = divmod(p, 2)
            gj, cj = divmod(q, 2)
            oi, wi = cov.slope_stencil(cfg, ci, d)
            oj, wj = cov.slope_stencil(cfg, cj, d)
            for (h, frac) in cfg["layers"]:
                gam = cov.cone_factor(gs[gi][2], h)
                r0k = turb.layer_r0(cfg["r0"], frac)
                sh = h * (np.array(gs[gi][:2]) - np.array(gs[gj][:2]))
                for ou, wu in zip(oi, wi):
                    for ov, wv in zip(oj, wj):
                        dx = gam * (LX * d + ou[0] - ov[0]) + sh[0]
                        dy = gam * (LY * d + ou[1] - ov[1]) + sh[1]
                        t[p, q] += wu * wv * turb.vk_covariance(np.hypot(dx, dy), r0k, cfg["L0"])
    return t


def noise_floor(cfg):
    """sigma_g^2 of each guide star for the preconditioner: noise_sigma^2, or with
    elongated-spot blocks (cfg["noise_cov"]) the mean of (s_xx + s_yy) / 2 over
    the guide star's valid subapertures, the blocks' mean eigenvalue."""
    C = cfg.get("noise_cov")
    if C is None:
        return np.asarray(cfg["noise_sigma"], np.float64) ** 2
    mask = geo.subaperture_mask(cfg["n"], cfg["obstruction"])
    C = np.asarray(C, np.float64)
    return np.array([0.5 * (C[g][mask][:, 0] + C[g][mask][:, 1]).mean() for g in range(len(cfg["gs"]))])


def spectra(cfg, P, floor=3.0):
    """M(f) = (K_+(f) + floor diag(sigma^2))^{-1} as [ky][kx][p][q] (rfft2 half spectrum)."""
    t = periodised_generators(cfg, P)
    NP = t.shape[0]
    lag = np.arange(-(P // 2), P - P // 2) % P
    wrapped = np.zeros_like(t)
    wrapped[:, :, lag[:, None], lag[None, :]] = t
    K = np.fft.rfft2(wrapped)                                  # [p][q][ky][kx]
    K = np.transpose(K, (2, 3, 0, 1))
    K = 0.5 * (K + np.conj(np.swapaxes(K, 2, 3)))
    ev, V = np.linalg.eigh(K)
    sig2 = np.repeat(noise_floor(cfg), 2)
    Kp = np.einsum("yxpk,yxk,yxqk->yxpq", V, np.maximum(ev, 0.0), V.conj()) + floor * np.diag(sig2)
    return np.linalg.inv(Kp)


def apply(cfg, x, P, floor=3.0, M=None):
    """M^{-1} x for x [B][N] (valid slopes), FP64."""
    if M is None:
        M = spectra(cfg, P, floor)
    n = cfg["n"]
    mask = geo.subaperture_mask(n, cfg["obstruction"])
    v = geo.valid_list(mask)
    x = np.atleast_2d(np.asarray(x, np.float64))
    B = x.shape[0]
    NP = M.shape[-1]
    planes = np.zeros((B, NP, P, P))
    planes[:, :, v[:, 0], v[:, 1]] = x.reshape(B, NP, -1)
    X = np.fft.rfft2(planes)
    Y = np.einsum("yxpq,bqyx->bpyx", M, X)
    y = np.fft.irfft2(Y, s=(P, P))
    return y[:, :, v[:, 0], v[:, 1]].reshape(B, -1)
