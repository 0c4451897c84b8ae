"""Pins of the oracle's analytic wave-front error (Sec. 3, Eq. analytical1-3)."""
import numpy as np

from oracle import covariance as cov
from oracle import geometry as geo
from oracle import solve
from oracle import wfe
from paper_1806_07938_gb300 import workloads as W


def _cfg(noise=0.3):
    # small natural-star system on a fine simulated screen (as the covariance pin)
    return dict(name="mcw", D=1.5, obstruction=0.0, n=3, r0=0.15, L0=1.0, layers=[(8e3, 1.0)],
                gs=[(15 * W.ARCSEC, 0.0, 0.0), (-15 * W.ARCSEC, 5 * W.ARCSEC, 0.0)],
                targets=[(0.0, 0.0)], noise_sigma=[noise, noise])


def _monte_carlo(cfg, R, n_screens):
    """Mean square piston-removed error of R on Hudgin slopes of simulated screens."""
    n, D = cfg["n"], cfg["D"]
    d = D / n
    cen = geo.subaperture_centres(n, D, 0.0)
    php = geo.phase_points(n, D, 0.0)
    h, _ = cfg["layers"][0]
    pts = []
    for (ax, ay, _) in cfg["gs"]:
        for comp in (0, 1):
            off = np.zeros(2); off[comp] = d / 2
            for c in cen:
                pts.append([c + off + h * np.array([ax, ay]), c - off + h * np.array([ax, ay])])
    pts = np.array(pts)
    pix, N = d / 32, 512
    rng = np.random.Generator(np.random.Philox(key=[9, 13]))
    sig = np.asarray(cov.noise_variance(cfg)) ** 0.5
    errs = []
    for _ in range(n_screens // 2):
        for scr in W.screen_pair(rng, N, pix, cfg["r0"], cfg["L0"]):
            sh = rng.uniform(0, N * pix, size=2)
            s = (W.bilinear(scr, pix, pts[:, 0, 0] + sh[0], pts[:, 0, 1] + sh[1])
                 - W.bilinear(scr, pix, pts[:, 1, 0] + sh[0], pts[:, 1, 1] + sh[1]))
            s = s + sig * rng.standard_normal(len(s))
            phi = W.bilinear(scr, pix, php[:, 0] + sh[0], php[:, 1] + sh[1])
            e = phi - R @ s
            e = e - e.mean()
            errs.append(np.mean(e * e))
    errs = np.array(errs)
    return errs.mean(), errs.std() / np.sqrt(len(errs))


def test_analytic_wfe_matches_monte_carlo():
    cfg = _cfg()
    F = cov.cos_interp(cfg, 0)
    A = cov.system_matrix(cfg)
    R = solve.reconstructor(F, A)
    ana = wfe.analytic_wfe(cfg, 0, R=R)
    mc, se = _monte_carlo(cfg, R, 3000)
    print(ana, mc, se)
    assert abs(mc - ana) <= 4 * se + 0.03 * ana
    # a reconstructor built for the wrong layer altitude (ground instead of 8 km)
    # is worse, and the formula follows the simulation for it too
    bad = dict(cfg, layers=[(0.0, 1.0)])
    R0 = solve.reconstructor(cov.cos_interp(bad, 0), cov.system_matrix(bad))
    ana0 = wfe.analytic_wfe(cfg, 0, R=R0)
    mc0, se0 = _monte_carlo(cfg, R0, 3000)
    print(ana0, mc0, se0)
    assert ana0 > 1.2 * ana and abs(mc0 - ana0) <= 4 * se0 + 0.03 * ana0


def test_mmse_is_the_minimum_and_the_short_form():
    cfg = _cfg()
    F = cov.cos_interp(cfg, 0)
    A = cov.system_matrix(cfg)
    R = solve.reconstructor(F, A)
    best = wfe.analytic_wfe(cfg, 0, R=R)
    rng = np.random.default_rng(1)
    for _ in range(3):
        assert wfe.analytic_wfe(cfg, 0, R=R + 1e-3 * rng.standard_normal(R.shape)) > best
    # for the MMSE R the error covariance is Sigma_phi_phi - F A^{-1} F^T
    n = F.shape[0]
    P = np.eye(n) - np.ones((n, n)) / n
    short = np.trace(P @ (wfe.phase_covariance(cfg) - F @ np.linalg.solve(A, F.T)) @ P) / n
    assert abs(short - best) <= 1e-10 * best
    # more noise, more error
    assert wfe.analytic_wfe(_cfg(noise=0.6), 0) > best
