"""Pins of the oracle's Fried slope model (Appendix A)."""
import numpy as np
import pytest

from conftest import small_cfg
from oracle import covariance as cov
from oracle import geometry as geo
from paper_1806_07938_gb300 import workloads as W


def _slopes(cfg, phase):
    """Slopes of a phase function through the oracle's slope points (first WFS)."""
    pts, w, gsidx = cov.slope_points(cfg)
    one = gsidx == 0
    return (w[one] * phase(pts[one])).sum(axis=1)


def test_fried_slopes_closed_form():
    # x^2 y^2: Hudgin x-slope 4 x h y^2, Fried 4 x h (y^2 + h^2), h = d/2 (and
    # symmetrically in y); x and xy agree between the models
    base = small_cfg(n=6, obstruction=0.2, D=3.0)
    d = base["D"] / base["n"]
    h = d / 2
    c = geo.subaperture_centres(6, 3.0, 0.2)
    x, y = c[:, 0], c[:, 1]
    f = lambda p: p[..., 0] ** 2 * p[..., 1] ** 2
    hud = _slopes(base, f)
    fri = _slopes(dict(base, slope_model="fried"), f)
    nv = len(c)
    assert np.allclose(hud[:nv], 4 * x * h * y ** 2) and np.allclose(hud[nv:], 4 * y * h * x ** 2)
    assert np.allclose(fri[:nv], 4 * x * h * (y ** 2 + h ** 2)) and np.allclose(fri[nv:], 4 * y * h * (x ** 2 + h ** 2))
    g = lambda p: p[..., 0] * p[..., 1] + 3 * p[..., 0]
    assert np.allclose(_slopes(base, g), _slopes(dict(base, slope_model="fried"), g))


def test_fried_does_not_see_the_waffle():
    # (-1)^(i+j) on the corner grid: zero Fried slopes everywhere; the same
    # pattern sampled at edge midpoints by a smooth extension is seen by Hudgin
    cfg = dict(small_cfg(n=6, obstruction=0.0, D=3.0), slope_model="fried")
    d = cfg["D"] / cfg["n"]
    waffle = lambda p: np.cos(np.pi * (p[..., 0] / d + 3)) * np.cos(np.pi * (p[..., 1] / d + 3))
    assert np.abs(_slopes(cfg, waffle)).max() < 1e-12
    tilted = lambda p: waffle(p) + 0.1 * p[..., 0]
    assert np.allclose(_slopes(cfg, tilted)[:len(_slopes(cfg, tilted)) // 2], 0.1 * d)


@pytest.mark.parametrize("lgs", [False, True])
def test_fried_covariance_spd_and_toeplitz(lgs):
    cfg = dict(small_cfg(n=5, lgs=lgs, obstruction=0.2), slope_model="fried")
    C = cov.css_dense(cfg)
    assert np.allclose(C, C.T, atol=1e-12 * np.abs(C).max())
    assert np.linalg.eigvalsh(C + np.diag(cov.noise_variance(cfg))).min() > 0
    # the Fried covariance differs from Hudgin's (a different model)
    H = cov.css_dense(small_cfg(n=5, lgs=lgs, obstruction=0.2))
    assert np.abs(C - H).max() > 0.02 * np.abs(H).max()


def test_fried_covariance_matches_simulated_screens():
    # empirical covariance of Fried slopes (four corners, traced here from
    # scratch) on simulated screens against the oracle's Fried Sigma_ss
    cfg = dict(name="mcf", D=1.5, obstruction=0.0, n=3, r0=0.15, L0=1.0, layers=[(12e3, 1.0)],
               gs=[(10 * W.ARCSEC, -5 * W.ARCSEC, 90e3), (25 * W.ARCSEC, 5 * W.ARCSEC, 90e3)],
               targets=[(0.0, 0.0)], noise_sigma=[0.0, 0.0], slope_model="fried")
    n, D = 3, 1.5
    d = D / n
    cen = geo.subaperture_centres(n, D, 0.0)
    h, _ = cfg["layers"][0]
    rows = []
    for (ax, ay, H) in cfg["gs"]:
        gam = 1 - h / H
        for comp in (0, 1):
            e = np.zeros(2); e[comp] = d / 2
            f = np.zeros(2); f[1 - comp] = d / 2
            for c in cen:
                corners = [c + e + f, c - e + f, c + e - f, c - e - f]
                rows.append([gam * q + h * np.array([ax, ay]) for q in corners])
    pts = np.array(rows)                      # (N, 4, 2)
    wts = np.array([0.5, -0.5, 0.5, -0.5])
    rng = np.random.Generator(np.random.Philox(key=[3, 17]))
    pix, Npx, S = d / 32, 512, []
    for _ in range(1500):
        for scr in W.screen_pair(rng, Npx, pix, cfg["r0"], cfg["L0"]):
            sh = rng.uniform(0, Npx * pix, size=2)
            vals = W.bilinear(scr, pix, pts[..., 0] + sh[0], pts[..., 1] + sh[1])
            S.append((vals * wts).sum(axis=1))
    S = np.array(S)
    emp = S.T @ S / len(S)
    C = cov.css_dense(cfg)
    M = len(S)
    dg = np.diag(C)
    z2 = float(np.mean((emp - C) ** 2 / ((np.outer(dg, dg) + C ** 2) / M)))
    Hm = cov.css_dense(dict(cfg, slope_model="hudgin"))
    z2h = float(np.mean((emp - Hm) ** 2 / ((np.outer(np.diag(Hm), np.diag(Hm)) + Hm ** 2) / M)))
    print(z2, z2h)
    assert z2 < 2.5 and z2h > 4 * z2
