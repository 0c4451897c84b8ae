"""Pins of the oracle's tip/tilt/focus removal (Sec. 2.F, mode removal)."""
import numpy as np
import pytest

from conftest import small_cfg
from oracle import covariance as cov
from oracle import geometry as geo
from oracle import modes


@pytest.mark.parametrize("n,eps", [(4, 0.0), (7, 0.2), (10, 0.28)])
def test_slope_modes_closed_form(n, eps):
    # two-point differences across a subaperture of width d centred at (xc, yc):
    # x -> d, y -> 0 (x slope); x^2 + y^2 -> 2 d xc (x slope), 2 d yc (y slope)
    cfg = small_cfg(n=n, obstruction=eps, D=0.5 * n)
    d = cfg["D"] / n
    c = geo.subaperture_centres(n, cfg["D"], eps)
    nv = len(c)
    Z = modes.slope_modes(cfg)
    assert Z.shape == (2 * nv, 3)
    one, zero = np.ones(nv), np.zeros(nv)
    assert np.allclose(Z[:, 0], np.r_[d * one, zero], atol=1e-14)
    assert np.allclose(Z[:, 1], np.r_[zero, d * one], atol=1e-14)
    assert np.allclose(Z[:, 2], np.r_[2 * d * c[:, 0], 2 * d * c[:, 1]], atol=1e-13)


def test_phase_modes_values():
    cfg = small_cfg(n=6, obstruction=0.2, D=3.0)
    xy = geo.phase_points(6, 3.0, 0.2)
    Z = modes.phase_modes(cfg)
    assert np.array_equal(Z[:, 0], xy[:, 0]) and np.array_equal(Z[:, 1], xy[:, 1])
    assert np.allclose(Z[:, 2], np.hypot(xy[:, 0], xy[:, 1]) ** 2, rtol=1e-14)


@pytest.mark.parametrize("which", ["slope", "phase"])
def test_removal_is_an_orthogonal_projector(which):
    cfg = small_cfg(n=7, n_gs=2, obstruction=0.2, D=4.2)
    M = modes.slope_removal(cfg) if which == "slope" else modes.phase_removal(cfg)
    Z = modes.slope_modes(cfg) if which == "slope" else modes.phase_modes(cfg)
    assert np.allclose(M, M.T, atol=1e-13)
    assert np.allclose(M @ M, M, atol=1e-12)
    if which == "slope":
        nv2 = Z.shape[0]
        assert np.abs(M[:nv2, :nv2] @ Z).max() < 1e-12          # WFS 0
        assert np.abs(M[nv2:, nv2:] @ Z).max() < 1e-12          # WFS 1
        assert np.abs(M[:nv2, nv2:]).max() == 0                   # block diagonal
        assert round(np.trace(M)) == M.shape[0] - 3 * 2
    else:
        assert np.abs(M @ Z).max() < 1e-12
        assert round(np.trace(M)) == M.shape[0] - 3


@pytest.mark.parametrize("lgs", [False, True])
def test_reconstruct_minimum_norm_and_mode_blind(lgs):
    cfg = small_cfg(n=6, lgs=lgs, obstruction=0.2, D=3.6, noise=0.2, targets=((0.0, 0.0), (8e-6, 4e-6)))
    A = cov.system_matrix(cfg)
    rng = np.random.default_rng(3)
    s = rng.standard_normal((A.shape[0], 2))
    zeta, phi = modes.reconstruct(cfg, s, A)
    Ms = modes.slope_removal(cfg)
    # the least-squares system is solved: its residual vanishes (consistent system)
    assert (modes.relative_residual(cfg, A, s, zeta) < 1e-10).all()
    # the minimum-norm solution has no component along the removed modes
    assert np.abs(Ms @ zeta - zeta).max() < 1e-10 * np.abs(zeta).max()
    # the estimate holds none of the removed phase modes
    Zp = modes.phase_modes(cfg)
    for p in phi:
        assert np.abs(Zp.T @ p).max() < 1e-10 * np.abs(p).max() * len(p)
    # blind to tip/tilt/focus in the measurements: adding them to every WFS
    # (a different mix per WFS) changes neither zeta nor phi
    Zs = modes.slope_modes(cfg)
    add = np.concatenate([Zs @ rng.standard_normal((3, 2)) for _ in cfg["gs"]])
    zeta2, phi2 = modes.reconstruct(cfg, s + 10 * add, A)
    assert np.allclose(zeta2, zeta, atol=1e-9 * np.abs(zeta).max())
    for p, p2 in zip(phi, phi2):
        assert np.allclose(p2, p, atol=1e-9 * np.abs(p).max())
    # and the removal changes the estimate (it is not the identity)
    phi_full = cov.cos_interp(cfg, 0) @ np.linalg.solve(A, s)
    assert np.linalg.norm(phi[0] - phi_full) > 0.05 * np.linalg.norm(phi_full)
