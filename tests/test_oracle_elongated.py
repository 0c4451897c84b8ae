"""Pins of the oracle's elongated-spot noise covariance (Sec. 2.F): one 2 x 2
block per subaperture coupling its x- and y-slope noise."""
import numpy as np

from conftest import small_cfg
from oracle import covariance as cov
from oracle import geometry as geo
from paper_1806_07938_gb300 import workloads as W


def elongated(n=6, k=3.0, sigma=0.15, lgs=True):
    cfg = small_cfg(n=n, lgs=lgs, obstruction=0.2, D=0.6 * n, noise=sigma)
    cfg["noise_cov"] = W.elongated_noise(cfg, sigma, k)
    return cfg


def test_block_noise_matches_sampled_noise():
    # draw slope noise on the full grid [g][x|y][i][j] from each subaperture's
    # 2 x 2 covariance (explicit 2 x 2 Cholesky factor), select the valid
    # subapertures as the slope vector is laid out, and compare the sample
    # covariance with the oracle's matrix entry by entry (6 standard errors)
    cfg = elongated()
    S = cov.noise_matrix(cfg)
    mask = geo.subaperture_mask(cfg["n"], cfg["obstruction"])
    C = cfg["noise_cov"]
    a, b, c = C[..., 0], C[..., 2], C[..., 1]
    l11 = np.sqrt(a)
    l21 = b / l11
    l22 = np.sqrt(c - l21 ** 2)
    rng = np.random.default_rng(2024)
    M, chunk = 200_000, 20_000
    acc = np.zeros_like(S)
    for _ in range(M // chunk):
        u = rng.standard_normal((chunk, 2) + C.shape[:3])           # [m][2][g][i][j]
        ex = l11 * u[:, 0]
        ey = l21 * u[:, 0] + l22 * u[:, 1]
        eta = np.stack([ex, ey], axis=2)                            # [m][g][x|y][i][j]
        v = eta[..., mask].reshape(chunk, -1)
        acc += v.T @ v
    E = acc / M
    d = np.diag(S)
    se = np.sqrt((np.outer(d, d) + S ** 2) / M)
    assert np.abs(E - S).max() > 0                                  # the comparison is live
    assert (np.abs(E - S) <= 6 * se).all()
    # the cross terms are resolved: the largest |s_xy| is many standard errors
    assert np.abs(S - np.diag(d)).max() > 50 * se.max()


def test_isotropic_blocks_reduce_to_white_noise():
    # no elongation (k = 0), and natural stars at any k: sigma^2 I
    for cfg in (elongated(k=0.0), elongated(k=3.0, lgs=False)):
        S = cov.noise_matrix(cfg)
        assert np.array_equal(S, np.diag(cov.noise_variance(dict(cfg, noise_cov=None))))
        A = cov.system_matrix(cfg)
        assert np.array_equal(A, cov.system_matrix(dict(cfg, noise_cov=None)))


def test_block_noise_structure():
    cfg = elongated(n=7)
    S = cov.noise_matrix(cfg)
    nv = int(geo.subaperture_mask(7, 0.2).sum())
    assert np.array_equal(S, S.T)
    # each row couples only the slope of the other axis in its own subaperture
    off = S - np.diag(np.diag(S))
    rows, cols = np.nonzero(off)
    assert (np.abs(rows - cols) == nv).all()
    assert (rows // (2 * nv) == cols // (2 * nv)).all()
    # smallest eigenvalue sigma^2 (the side-launch blocks are sigma^2 (I + e^2 v v^T))
    assert abs(np.linalg.eigvalsh(S).min() - 0.15 ** 2) <= 1e-12
    # r0 / noise-scaled system: Sigma_ss(r0) + nu Sigma_eta_eta
    A = cov.system_matrix_r0(cfg, 0.1, noise_scale=2.5)
    assert np.abs(A - cov.css_dense(dict(cfg, r0=0.1)) - 2.5 * S).max() <= 1e-14 * np.abs(A).max()


def test_noise_weighted_reconstructor_is_optimal():
    # the MMSE reconstructor built with the true (block) noise has a smaller
    # mean square error under that noise than one built assuming white noise
    # (Eq. analytical1 evaluated for both with the true covariances)
    from oracle import solve, wfe
    cfg = small_cfg(n=8, lgs=True, obstruction=0.2, D=4.8, noise=0.3, targets=((0.0, 0.0),))
    cfg["noise_cov"] = W.elongated_noise(cfg, 0.3, 4.0)
    best = wfe.analytic_wfe(cfg, 0)
    F = cov.cos_interp(cfg, 0)
    R_white = solve.reconstructor(F, cov.system_matrix(dict(cfg, noise_cov=None)))
    mismatched = wfe.analytic_wfe(cfg, 0, R=R_white)
    assert mismatched > best * (1 + 1e-3)


def test_analytic_wfe_noise_term_matches_sampled_noise():
    # Eq. analytical1 with the turbulence switched off (r0 -> 1e9: every
    # covariance scales as r0^{-5/3}) keeps only the noise term of a fixed R:
    # mean square of P R eta over eta drawn from each subaperture's 2 x 2 block
    from oracle import solve, wfe
    cfg = elongated(n=6, k=4.0)
    R = solve.reconstructor(cov.cos_interp(cfg, 0), cov.system_matrix(cfg))
    quiet = dict(cfg, r0=1e9)
    ana = wfe.analytic_wfe(quiet, 0, R=R)
    mask = geo.subaperture_mask(cfg["n"], cfg["obstruction"])
    C = cfg["noise_cov"]
    l11 = np.sqrt(C[..., 0])
    l21 = C[..., 2] / l11
    l22 = np.sqrt(C[..., 1] - l21 ** 2)
    rng = np.random.default_rng(77)
    vals = []
    for _ in range(10):
        u = rng.standard_normal((4000, 2) + C.shape[:3])
        eta = np.stack([l11 * u[:, 0], l21 * u[:, 0] + l22 * u[:, 1]], axis=2)[..., mask].reshape(4000, -1)
        e = eta @ R.T
        e = e - e.mean(axis=1, keepdims=True)
        vals.append(np.mean(e * e, axis=1))
    vals = np.concatenate(vals)
    mc, se = vals.mean(), vals.std() / np.sqrt(len(vals))
    assert abs(mc - ana) <= 4 * se
    # dropping the x/y coupling of the blocks moves the term by many errors
    flat = cfg["noise_cov"].copy()
    flat[..., 2] = 0.0
    ana_flat = wfe.analytic_wfe(dict(quiet, noise_cov=flat), 0, R=R)
    assert abs(ana_flat - ana) > 10 * se


def test_preconditioner_floor_with_block_noise():
    # without elongation the floor is noise_sigma^2 and the spectra are those of
    # the white-noise system; elongation raises each laser star's floor to the
    # blocks' mean eigenvalue, above sigma^2, and M stays positive definite
    from oracle import precond
    base = small_cfg(n=6, lgs=True, obstruction=0.2, D=3.6, noise=0.15)
    iso = dict(base, noise_cov=W.elongated_noise(base, 0.15, 0.0))
    assert np.allclose(precond.noise_floor(iso), 0.15 ** 2, rtol=1e-15, atol=0)
    assert np.array_equal(precond.spectra(iso, 12), precond.spectra(base, 12))
    el = dict(base, noise_cov=W.elongated_noise(base, 0.15, 3.0))
    fl = precond.noise_floor(el)
    assert (fl > 0.15 ** 2).all()
    M = precond.spectra(el, 12)
    assert np.linalg.eigvalsh(0.5 * (M + np.conj(np.swapaxes(M, -1, -2)))).min() > 0
