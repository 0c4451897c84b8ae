"""Tip/tilt/focus removal for split tomography (oracle; test infrastructure only).

Sec. 2.F, "Mode removal": with laser guide stars, tip, tilt and focus are not
measurable, so they are removed from the measurements and from the estimate.
For WFS i, Z_s,i (2 n_vs x 3) holds in each column the slopes of one mode on
the valid subapertures, and M_s,i = I - Z_s,i Z_s,i^+ (^+ the pseudo-inverse);
M_s is block diagonal over the WFS.  M_phi = I - Z_phi Z_phi^+ acts on the
valid phase points (Z_phi: n_vphi x 3).  The masked system of Eq. SAap1 and
the projection of Eq. SAap2 become

    M_s W_s (Sigma_ss + Sigma_eta_eta) W_s^T M_s zeta = M_s s,
    phi = M_phi W_phi Sigma_phi_s W_s^T M_s zeta.

The modes are tip x, tilt y and focus x^2 + y^2 in pupil coordinates.  Their
slopes are formed here by sampling the mode at the two points of every
Hudgin-like slope (Appendix A.2), the same points the covariances use.  The
system is singular (its null space is spanned by the modes), so the solution
is the minimum-norm least-squares one, from numpy's lstsq.
"""

import numpy as np

from . import covariance as cov
from . import geometry as geo
from . import solve

MODES = ("tip", "tilt", "focus")


def _mode(name, xy):
    x, y = xy[..., 0], xy[..., 1]
    if name == "tip":
        return x
    if name == "tilt":
        return y
    return x * x + y * y


def slope_modes(cfg):
    """Z_s of one WFS: (2 n_vs, 3), the two-point slopes of tip, tilt, focus."""
    if not cov.uniform_grid(cfg):
        raise NotImplementedError("mode removal here takes one grid for all guide stars")
    pts, w, gsidx = cov.slope_points(cfg)
    one = gsidx == 0
    pts, w = pts[one], w[one]
    return np.stack([(w * _mode(m, pts)).sum(axis=1) for m in MODES], axis=1)


def phase_modes(cfg):
    """Z_phi: (n_vphi, 3), tip, tilt and focus on the valid phase points."""
    xy = geo.phase_points(cfg["n"], cfg["D"], cfg["obstruction"])
    return np.stack([_mode(m, xy) for m in MODES], axis=1)


def removal(Z):
    """I - Z Z^+."""
    return np.eye(Z.shape[0]) - Z @ np.linalg.pinv(Z)


def slope_removal(cfg):
    """M_s: block diagonal over the guide stars, one M_s,i per WFS."""
    Mi = removal(slope_modes(cfg))
    return np.kron(np.eye(len(cfg["gs"])), Mi)


def phase_removal(cfg):
    return removal(phase_modes(cfg))


def reconstruct(cfg, s, A=None, targets=None):
    """Minimum-norm zeta of M_s A M_s zeta = M_s s for the columns of s
    (N x k), and phi [target] (n_vphi x k) = M_phi Sigma_phi_s M_s zeta."""
    A = cov.system_matrix(cfg) if A is None else A
    Ms = slope_removal(cfg)
    AM = Ms @ A @ Ms
    zeta = np.linalg.lstsq(AM, Ms @ s, rcond=None)[0]
    Mp = phase_removal(cfg)
    targets = range(len(cfg["targets"])) if targets is None else targets
    phi = [Mp @ (cov.cos_interp(cfg, t) @ (Ms @ zeta)) for t in targets]
    return zeta, phi


def relative_residual(cfg, A, s, zeta):
    """||M_s s - M_s A M_s zeta|| / ||M_s s|| per column."""
    Ms = slope_removal(cfg)
    return solve.relative_residual(Ms @ A @ Ms, Ms @ s, zeta)
