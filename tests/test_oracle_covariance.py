"""Pins of the oracle's dense covariances (Sec. 2.D structure, Appendix A.2 Hudgin-like model)."""
import numpy as np
import pytest

from oracle import covariance as cov
from oracle import geometry as geo
from oracle import turbulence as turb
from conftest import small_cfg


def _D(vec, cfg, k):
    h, frac = cfg["layers"][k]
    return turb.vk_structure_function(np.hypot(vec[..., 0], vec[..., 1]), turb.layer_r0(cfg["r0"], frac), cfg["L0"])


@pytest.mark.parametrize("lgs", [False, True])
def test_symmetric_positive_definite(lgs):
    cfg = small_cfg(n=5, lgs=lgs, obstruction=0.2)
    C = cov.css_dense(cfg)
    assert np.abs(C - C.T).max() <= 1e-12 * np.abs(C).max()
    w = np.linalg.eigvalsh(C)
    assert w.min() > -1e-10 * w.max()
    A = cov.system_matrix(cfg)
    np.linalg.cholesky(A)
    assert np.linalg.eigvalsh(A).min() >= 0.1 ** 2 * (1 - 1e-8)


@pytest.mark.parametrize("lgs", [False, True])
def test_toeplitz_invariance(lgs):
    # Sec. 2.D: with a common guide-star altitude every Theta_pq depends only on
    # the subaperture separation (2RBT); the oracle never assumes it.
    cfg = small_cfg(n=6, lgs=lgs, obstruction=0.25)
    C = cov.css_dense(cfg)
    v = geo.valid_list(geo.subaperture_mask(cfg["n"], cfg["obstruction"]))
    nv = len(v)
    scale = np.abs(C).max()
    for p in range(2 * len(cfg["gs"])):
        for q in range(2 * len(cfg["gs"])):
            blk = C[p * nv:(p + 1) * nv, q * nv:(q + 1) * nv]
            seen = {}
            for a in range(nv):
                for b in range(nv):
                    key = (v[a, 0] - v[b, 0], v[a, 1] - v[b, 1])
                    if key in seen:
                        assert abs(seen[key] - blk[a, b]) <= 1e-11 * scale
                    else:
                        seen[key] = blk[a, b]


@pytest.mark.parametrize("lgs", [False, True])
def test_zero_lag_values(lgs):
    # Hudgin model at zero lag: var(s_x) = sum_k D_k(gamma_k d); cov(s_x, s_y) = 0 (isotropy)
    cfg = small_cfg(n=5, lgs=lgs)
    C = cov.css_dense(cfg)
    nv = geo.subaperture_mask(cfg["n"], cfg["obstruction"]).sum()
    d = cfg["D"] / cfg["n"]
    expect = 0.0
    for k, (h, frac) in enumerate(cfg["layers"]):
        gam = 1 - h / 90e3 if lgs else 1.0
        expect += turb.vk_structure_function(gam * d, turb.layer_r0(cfg["r0"], frac), cfg["L0"])
    assert np.allclose(np.diag(C), expect, rtol=1e-12)
    for g in range(len(cfg["gs"])):
        xy = C[(2 * g) * nv:(2 * g + 1) * nv, (2 * g + 1) * nv:(2 * g + 2) * nv]
        assert np.abs(np.diag(xy)).max() <= 1e-12 * expect


@pytest.mark.parametrize("lgs", [False, True])
def test_paper_hudgin_formulas(lgs):
    # Appendix A.2: Sigma_sxsx = 1/2 [-2D(Delta) + D(Delta + d_x) + D(Delta - d_x)] and
    # Sigma_sxsy = 1/2 [D(Delta + d_x/2 + d_y/2) - D(Delta - d_x/2 + d_y/2) - D(Delta + d_x/2 - d_y/2)
    #                    + D(Delta - d_x/2 - d_y/2)]   (the paper prints the last sign as "-"; "+" is
    #                    what the point-covariance derivation gives and Sigma_sxsy(0) = 0 requires),
    # Delta_k = gamma_k (c_a - c_b) + h_k (alpha_a - alpha_b), offsets gamma_k d (cone reading).
    cfg = small_cfg(n=5, lgs=lgs, obstruction=0.2)
    C = cov.css_dense(cfg)
    cen = geo.subaperture_centres(cfg["n"], cfg["D"], cfg["obstruction"])
    nv = len(cen)
    d = cfg["D"] / cfg["n"]
    gs = cfg["gs"]
    for (ga, gb) in [(0, 0), (0, 1), (2, 1)]:
        ref_xx = np.zeros((nv, nv)); ref_yy = np.zeros((nv, nv)); ref_xy = np.zeros((nv, nv))
        for k, (h, frac) in enumerate(cfg["layers"]):
            gam = 1 - h / 90e3 if lgs else 1.0
            Delta = gam * (cen[:, None, :] - cen[None, :, :]) + h * (np.array(gs[ga][:2]) - np.array(gs[gb][:2]))
            ex = np.array([gam * d, 0.0]); ey = np.array([0.0, gam * d])
            ref_xx += 0.5 * (-2 * _D(Delta, cfg, k) + _D(Delta + ex, cfg, k) + _D(Delta - ex, cfg, k))
            ref_yy += 0.5 * (-2 * _D(Delta, cfg, k) + _D(Delta + ey, cfg, k) + _D(Delta - ey, cfg, k))
            ref_xy += 0.5 * (_D(Delta + ex / 2 + ey / 2, cfg, k) - _D(Delta - ex / 2 + ey / 2, cfg, k)
                             - _D(Delta + ex / 2 - ey / 2, cfg, k) + _D(Delta - ex / 2 - ey / 2, cfg, k))
        sc = np.abs(ref_xx).max()
        blk = lambda p, q: C[p * nv:(p + 1) * nv, q * nv:(q + 1) * nv]
        assert np.abs(blk(2 * ga, 2 * gb) - ref_xx).max() <= 1e-10 * sc
        assert np.abs(blk(2 * ga + 1, 2 * gb + 1) - ref_yy).max() <= 1e-10 * sc
        assert np.abs(blk(2 * ga, 2 * gb + 1) - ref_xy).max() <= 1e-10 * sc


def test_cone_is_a_scaled_pupil():
    # one laser star at H and one layer at h sees the same statistics as a natural
    # star looking at a pupil scaled by gamma = 1 - h/H through a ground layer
    H, h = 90e3, 12e3
    gam = 1 - h / H
    lgs = small_cfg(n=5, n_gs=1, lgs=True, layers=((h, 1.0),), D=4.0)
    ngs = small_cfg(n=5, n_gs=1, lgs=False, layers=((0.0, 1.0),), D=4.0 * gam)
    lgs["gs"] = [(0.0, 0.0, H)]
    ngs["gs"] = [(0.0, 0.0, 0.0)]
    A, B = cov.css_dense(lgs), cov.css_dense(ngs)
    assert np.abs(A - B).max() <= 1e-11 * np.abs(A).max()


def test_phase_slope_paper_formula_ngs():
    # Appendix A.2: Sigma_phi_sx = 1/2 [D(Delta - d_x/2) - D(Delta + d_x/2)], Delta = (c_b - q) + h (alpha - beta)
    cfg = small_cfg(n=5, lgs=False, targets=((5e-5, -3e-5),))
    Cos = cov.cos_exact(cfg, 0)
    q = geo.phase_points(cfg["n"], cfg["D"], cfg["obstruction"])
    cen = geo.subaperture_centres(cfg["n"], cfg["D"], cfg["obstruction"])
    nv = len(cen)
    d = cfg["D"] / cfg["n"]
    beta = np.array(cfg["targets"][0])
    for g in range(3):
        ref_x = np.zeros((len(q), nv)); ref_y = np.zeros((len(q), nv))
        for k, (h, frac) in enumerate(cfg["layers"]):
            Delta = (cen[None, :, :] - q[:, None, :]) + h * (np.array(cfg["gs"][g][:2]) - beta)
            ex = np.array([d, 0.0]); ey = np.array([0.0, d])
            ref_x += 0.5 * (_D(Delta - ex / 2, cfg, k) - _D(Delta + ex / 2, cfg, k))
            ref_y += 0.5 * (_D(Delta - ey / 2, cfg, k) - _D(Delta + ey / 2, cfg, k))
        sc = np.abs(ref_x).max()
        assert np.abs(Cos[:, 2 * g * nv:(2 * g + 1) * nv] - ref_x).max() <= 1e-10 * sc
        assert np.abs(Cos[:, (2 * g + 1) * nv:(2 * g + 2) * nv] - ref_y).max() <= 1e-10 * sc


def test_new_grid_reduces_to_exact_for_natural_stars():
    cfg = small_cfg(n=6, lgs=False, obstruction=0.2, targets=((1e-5, 2e-5),))
    assert cov.new_grid_size(cfg) == cfg["n"] + 1
    A, B = cov.cos_exact(cfg, 0), cov.cos_interp(cfg, 0)
    assert np.abs(A - B).max() <= 1e-10 * np.abs(A).max()


def test_bilinear_weights_are_interpolating():
    cfg = small_cfg(n=8, lgs=True, obstruction=0.25)
    q = geo.phase_points(cfg["n"], cfg["D"], cfg["obstruction"])
    for k in range(len(cfg["layers"])):
        I = cov.bilinear_weights(cfg, k)
        nodes = cov.new_grid_nodes(cfg, k)
        assert np.allclose(I.sum(axis=1), 1.0, atol=1e-14)
        assert (I >= -1e-15).all()
        # exact on affine functions
        assert np.allclose(I @ nodes, q, atol=1e-12)


def test_new_grid_covariance_is_toeplitz():
    # Xi'_{q,k} between the gamma_k d-spaced grid and the slopes is 2RBT (Sec. 2.D)
    cfg = small_cfg(n=5, lgs=True, obstruction=0.0, targets=((2e-5, 0.0),))
    npr = cov.new_grid_size(cfg)
    v = geo.valid_list(geo.subaperture_mask(cfg["n"], 0.0))
    nv = len(v)
    for k in range(len(cfg["layers"])):
        X = cov.cos_new_grid_layer(cfg, 0, k)
        scale = np.abs(X).max()
        for p in (0, 1, 4):
            blk = X[:, p * nv:(p + 1) * nv]
            seen = {}
            for a in range(npr * npr):
                for b in range(nv):
                    key = (a // npr - v[b, 0], a % npr - v[b, 1])
                    if key in seen:
                        assert abs(seen[key] - blk[a, b]) <= 1e-11 * scale
                    else:
                        seen[key] = blk[a, b]


def test_new_grid_size_rule():
    cfg = small_cfg(n=74, lgs=True, layers=((0.0, 0.5), (20000.0, 0.5)))
    assert cov.new_grid_size(cfg) == 97      # ceil(74 / (1 - 20/90)) + 1


@pytest.mark.parametrize("lgs", [False, True])
def test_covariance_scales_as_r0_to_minus_five_thirds(lgs):
    # von Karman: B(rho) = c_v (L0/r0)^{5/3} * (a function of rho / L0), so every
    # covariance (slope-slope and phase-slope) scales as r0^{-5/3} at fixed Cn^2
    # fractions; the per-frame r0 system of the solver relies on it
    cfg = small_cfg(n=5, lgs=lgs, obstruction=0.2, D=3.0)
    base = cov.css_dense(cfg)
    for r0 in (0.10, 0.2):
        c = (r0 / cfg["r0"]) ** (-5.0 / 3.0)
        got = cov.css_dense(dict(cfg, r0=r0))
        assert np.abs(got - c * base).max() <= 1e-12 * np.abs(c * base).max()
        F = c * cov.cos_interp(cfg, 0)
        assert np.abs(cov.cos_interp(dict(cfg, r0=r0), 0) - F).max() <= 1e-12 * np.abs(F).max()
        # and not as r0^{+5/3} or r0^{-5/6}
        assert np.abs(got - base).max() > 0.3 * np.abs(base).max()
    A = cov.system_matrix_r0(cfg, cfg["r0"])
    assert np.array_equal(A, cov.system_matrix(cfg))
    # the noise term is the configuration's, times the frame's noise scale
    A2 = cov.system_matrix_r0(cfg, 0.1, noise_scale=2.5)
    nv = cov.noise_variance(cfg)
    assert np.allclose(np.diag(A2) - np.diag(cov.css_dense(dict(cfg, r0=0.1))), 2.5 * nv, rtol=1e-13)


def test_css_block_is_a_block_of_the_dense_matrix():
    # the column-restricted form used to time a principal block of the ELT
    # matrix: the same entries as the dense matrix's rows and columns
    from conftest import small_cfg
    cfg = small_cfg(n=6, lgs=True, obstruction=0.2, D=3.0)
    S = cov.css_dense(cfg)
    rng = np.random.default_rng(3)
    rows = rng.choice(S.shape[0], 17, replace=False)
    cols = rng.choice(S.shape[0], 11, replace=False)
    assert np.array_equal(cov.css_block(cfg, rows, cols), S[np.ix_(rows, cols)])
    assert np.array_equal(cov.css_rows(cfg, rows), S[rows])
