"""Brute-force pin: the oracle's Sigma_ss against the empirical covariance of
Hudgin slopes measured on simulated von Karman phase screens.

The screens come from the PSD (Appendix A.1), not from the covariance the
oracle evaluates, and the rays are traced here from scratch (laser star at H,
layer at h: pupil point p lands at (1 - h/H) p + h alpha).  A wrong sign of the
h*alpha shift or a wrong cone factor fails this test (checked below).
"""
import numpy as np

from oracle import covariance as cov
from oracle import geometry as geo
from paper_1806_07938_gb300 import workloads as W


def _cfg():
    return dict(name="mc", D=1.5, obstruction=0.0, n=3, r0=0.15, L0=1.0,
                layers=[(15e3, 1.0)], gs=[(10 * W.ARCSEC, -5 * W.ARCSEC, 90e3), (25 * W.ARCSEC, 5 * W.ARCSEC, 90e3)],
                targets=[(0.0, 0.0)], noise_sigma=[0.0, 0.0])


def _empirical(cfg, n_screens, sign):
    n, D = cfg["n"], cfg["D"]
    d = D / n
    cen = geo.subaperture_centres(n, D, cfg["obstruction"])
    h, _ = cfg["layers"][0]
    pix, N = d / 32, 512
    pts = []
    for (ax, ay, H) in cfg["gs"]:
        gam = 1 - h / H
        for comp in (0, 1):
            off = np.zeros(2); off[comp] = d / 2
            for c in cen:
                pts.append([gam * (c + off) + sign * h * np.array([ax, ay]),
                            gam * (c - off) + sign * h * np.array([ax, ay])])
    pts = np.array(pts)                                   # (N, 2, 2)
    rng = np.random.Generator(np.random.Philox(key=[7, 11]))
    S = []
    for _ in range(n_screens // 2):
        for scr in W.screen_pair(rng, N, pix, cfg["r0"], cfg["L0"]):
            # random placement of the pupil on the periodic screen keeps samples independent of pixel phase
            sh = rng.uniform(0, N * pix, size=2)
            a = W.bilinear(scr, pix, pts[:, 0, 0] + sh[0], pts[:, 0, 1] + sh[1])
            b = W.bilinear(scr, pix, pts[:, 1, 0] + sh[0], pts[:, 1, 1] + sh[1])
            S.append(a - b)
    S = np.array(S)
    return S.T @ S / len(S)


def test_empirical_covariance_matches():
    cfg = _cfg()
    C = cov.css_dense(cfg)
    emp = _empirical(cfg, 4000, +1.0)

    M = 4000
    # chi-square-like statistic: each sample-covariance entry has variance
    # (C_aa C_bb + C_ab^2) / M for Gaussian slopes
    def z2(model, emp_, sl=(slice(None), slice(None))):
        d = np.diag(model)
        var = (np.outer(d, d) + model ** 2) / M
        return float(np.mean(((emp_ - model) ** 2 / var)[sl]))
    nv = C.shape[0] // 4
    cross = (slice(0, 2 * nv), slice(2 * nv, 4 * nv))        # guide star 0 vs guide star 1
    # the h*alpha shift with the wrong sign, and a missing cone factor, give other matrices
    Cw = cov.css_dense(dict(cfg, gs=[(-ax, -ay, H) for (ax, ay, H) in cfg["gs"]]))
    Cf = cov.css_dense(dict(cfg, gs=[(ax, ay, 0.0) for (ax, ay, _) in cfg["gs"]]))
    good, good_x = z2(C, emp), z2(C, emp, cross)
    print(good, good_x, z2(Cw, emp, cross), z2(Cf, emp))
    assert good < 2.5 and good_x < 2.5
    assert z2(Cw, emp, cross) > 8 * good_x
    assert z2(Cf, emp) > 3.5 * good
