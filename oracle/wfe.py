"""Analytic wave-front error of a reconstructor (oracle; test infrastructure only).

Eq. analytical1-3 (Sec. 3): for a target beta and a reconstructor R,

    sigma^2 = Trace(Sigma_phi_phi - R Sigma_s_phi - Sigma_phi_s R^T
                    + R Sigma_ss R^T) + Trace(R Sigma_eta_eta R^T),

here over the valid phase points with piston removed (P = I - 1 1^T / n,
slopes do not see piston) and divided by their number (mean square error per
point).  Sigma_phi_phi is the target's phase covariance: a target at infinity
sees layer k through the pupil shifted by h_k beta, so entry (u, v) is
sum_k B_k(|x_u - x_v|).  Sigma_phi_s is the projection the reconstructor uses
(covariance.cos_interp); R defaults to the MMSE R = Sigma_phi_s A^{-1}.
Everything is formed densely and the formula is evaluated as printed.
"""

import numpy as np

from . import covariance as cov
from . import geometry as geo
from . import solve
from . import turbulence as turb


def phase_covariance(cfg):
    """Sigma_phi_phi on the valid phase points (n_vphi x n_vphi)."""
    xy = geo.phase_points(cfg["n"], cfg["D"], cfg["obstruction"])
    dx = xy[:, None, 0] - xy[None, :, 0]
    dy = xy[:, None, 1] - xy[None, :, 1]
    rho = np.hypot(dx, dy)
    C = np.zeros_like(rho)
    for (_, frac) in cfg["layers"]:
        C += turb.vk_covariance(rho, turb.layer_r0(cfg["r0"], frac), cfg["L0"])
    return C


def analytic_wfe(cfg, target=0, R=None, A=None):
    """Mean square piston-removed error per phase point [rad^2], Eq. analytical1-3."""
    F = cov.cos_interp(cfg, target)
    Css = cov.css_dense(cfg)
    Ceta = cov.noise_matrix(cfg)
    if R is None:
        R = solve.reconstructor(F, Css + Ceta if A is None else A)
    Cpp = phase_covariance(cfg)
    E = Cpp - R @ F.T - F @ R.T + R @ Css @ R.T + R @ Ceta @ R.T
    n = E.shape[0]
    P = np.eye(n) - np.ones((n, n)) / n
    return float(np.trace(P @ E @ P) / n)
