"""Pins of the oracle with guide stars on grids of their own (the uneven MOAO
system: natural stars on coarse grids beside laser stars on fine ones,
Sec. 2.D; blocks between them are not Toeplitz)."""
import numpy as np
import pytest

from oracle import covariance as cov
from oracle import geometry as geo
from oracle import modes
from conftest import small_cfg


def _mixed(n_lgs=9, n_ngs=3, obstruction=0.2):
    """Two laser stars on an n_lgs grid and one natural star on an n_ngs grid."""
    lgs = small_cfg(n=n_lgs, n_gs=2, lgs=True, obstruction=obstruction)
    ngs = small_cfg(n=n_ngs, n_gs=1, lgs=False, obstruction=obstruction, radius_arcsec=30.0)
    cfg = dict(lgs, gs=list(lgs["gs"]) + list(ngs["gs"]), gs_n=[n_lgs, n_lgs, n_ngs],
               noise_sigma=[0.1, 0.1, 0.2])
    return cfg, lgs, ngs


def test_uniform_gs_n_is_the_default():
    cfg = small_cfg(n=6, lgs=True, obstruction=0.2)
    same = dict(cfg, gs_n=[6] * len(cfg["gs"]))
    assert np.array_equal(cov.css_dense(cfg), cov.css_dense(same))


def test_diagonal_blocks_are_the_single_grid_systems():
    # each star's own block pair depends only on its grid, direction and
    # altitude: the laser-star block of the mixed system is the laser-only
    # system's Sigma_ss, the natural-star block the natural-only one's
    cfg, lgs, ngs = _mixed()
    C = cov.css_dense(cfg)
    nl = 2 * 2 * int(geo.subaperture_mask(9, 0.2).sum())
    nn = 2 * int(geo.subaperture_mask(3, 0.2).sum())
    assert C.shape == (nl + nn, nl + nn)
    scale = np.abs(C).max()
    assert np.abs(C[:nl, :nl] - cov.css_dense(lgs)).max() <= 1e-14 * scale
    assert np.abs(C[nl:, nl:] - cov.css_dense(ngs)).max() <= 1e-14 * scale
    assert np.abs(C - C.T).max() <= 1e-12 * scale
    # the noise of each star sits on its own slopes
    nv = cov.noise_variance(cfg)
    assert np.allclose(nv[:nl], 0.01) and np.allclose(nv[nl:], 0.04)
    np.linalg.cholesky(cov.system_matrix(cfg))


@pytest.mark.parametrize("H", [0.0, 90e3])
def test_coarse_slopes_are_sums_of_fine_slopes(H):
    # Two stars in one direction at one altitude, on grids of 12 and 4
    # subapertures: a coarse subaperture covers 3 x 3 fine ones, and its
    # two-point x-slope phi(c + 3d/2) - phi(c - 3d/2) is the sum of the three
    # fine x-slopes on the row through its centre (the phase differences
    # telescope), whatever the covariance function.  So each coarse row of
    # Sigma_ss is the sum of three fine rows, against every column.
    base = small_cfg(n=12, n_gs=1, lgs=H > 0, D=4.0, obstruction=0.0)
    g = tuple(base["gs"][0])
    cfg = dict(base, gs=[g, g], gs_n=[12, 4], noise_sigma=[0.1, 0.1])
    fine = geo.subaperture_mask(12, 0.0)
    coarse = geo.subaperture_mask(4, 0.0)
    fidx = -np.ones((12, 12), dtype=np.int64)
    fidx[fine] = np.arange(fine.sum())
    nvf, nvc = int(fine.sum()), int(coarse.sum())
    cols = np.arange(2 * nvf + 2 * nvc)
    checked = 0
    for e, (i, j) in enumerate(geo.valid_list(coarse)):
        for comp in (0, 1):
            if comp == 0:
                cells = [(3 * i + 1, 3 * j + k) for k in range(3)]
            else:
                cells = [(3 * i + k, 3 * j + 1) for k in range(3)]
            if any(not fine[c] for c in cells):
                continue
            frows = [comp * nvf + fidx[c] for c in cells]
            crow = 2 * nvf + comp * nvc + e
            want = cov.css_block(cfg, frows, cols).sum(axis=0)
            got = cov.css_block(cfg, [crow], cols)[0]
            assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()
            checked += 1
    assert checked >= 16


def test_uniform_grid_only_parts_refuse_mixed_grids():
    cfg, _, _ = _mixed()
    with pytest.raises(NotImplementedError):
        modes.slope_modes(cfg)
    with pytest.raises(NotImplementedError):
        cov.add_noise(np.zeros((2, 2)), dict(cfg, noise_cov=np.zeros((3, 9, 9, 3))))


def _empirical_mixed(cfg, n_screens):
    """Sample covariance of two-point slopes traced through simulated
    single-layer screens, each star on its own grid (rays traced here, not by
    the oracle: pupil point p of star (alpha, H) lands at (1 - h/H) p + h alpha)."""
    from paper_1806_07938_gb300 import workloads as W
    D = cfg["D"]
    h, _ = cfg["layers"][0]
    pts = []
    for g, (ax, ay, H) in enumerate(cfg["gs"]):
        n = cfg["gs_n"][g]
        d = D / n
        gam = 1.0 - h / H if H > 0 else 1.0
        for comp in (0, 1):
            off = np.zeros(2)
            off[comp] = d / 2
            for c in geo.subaperture_centres(n, D, cfg["obstruction"]):
                shift = h * np.array([ax, ay])
                pts.append([gam * (c + off) + shift, gam * (c - off) + shift])
    pts = np.array(pts)
    pix, N = D / 6 / 32, 512
    rng = np.random.Generator(np.random.Philox(key=[13, 17]))
    S = []
    for _ in range(n_screens // 2):
        for scr in W.screen_pair(rng, N, pix, cfg["r0"], cfg["L0"]):
            sh = rng.uniform(0, N * pix, size=2)
            a = W.bilinear(scr, pix, pts[:, 0, 0] + sh[0], pts[:, 0, 1] + sh[1])
            b = W.bilinear(scr, pix, pts[:, 1, 0] + sh[0], pts[:, 1, 1] + sh[1])
            S.append(a - b)
    S = np.array(S)
    return S.T @ S / len(S)


def test_cross_block_matches_simulated_screens():
    # a laser star on a 6 x 6 grid and a natural star on a 2 x 2 grid in
    # nearby directions, one layer at 2 km (overlapping footprints, strongly
    # correlated slopes): the oracle's whole matrix, and its cross block in
    # particular, against the sample covariance of slopes on simulated
    # screens; the cross block computed as if the natural star's slopes
    # spanned the fine grid's subaperture size fits far worse
    from paper_1806_07938_gb300 import workloads as W
    cfg = dict(name="mc_mixed", D=1.5, obstruction=0.0, n=6, r0=0.15, L0=1.0, layers=[(2e3, 1.0)],
               gs=[(5 * W.ARCSEC, 0.0, 90e3), (-5 * W.ARCSEC, 5 * W.ARCSEC, 0.0)], gs_n=[6, 2],
               targets=[(0.0, 0.0)], noise_sigma=[0.0, 0.0])
    C = cov.css_dense(cfg)
    M = 4000
    emp = _empirical_mixed(cfg, M)
    nl = 2 * int(geo.subaperture_mask(6, 0.0).sum())

    def z2(model, sl):
        d = np.diag(C)
        var = (np.outer(d, d) + C ** 2) / M
        return float(np.mean(((emp - model) ** 2 / var)[sl]))
    cross = (slice(0, nl), slice(nl, C.shape[0]))
    # the wrong model: the natural star's slopes over fine-grid subaperture size
    wrong = dict(cfg, gs_n=[6, 6])
    Cw_full = cov.css_dense(wrong)
    cen6 = geo.subaperture_centres(6, 1.5, 0.0)
    cen2 = geo.subaperture_centres(2, 1.5, 0.0)
    # the fine-grid natural-star slopes nearest the coarse centres stand in for them
    pick = [int(np.argmin(np.hypot(*(cen6 - c).T))) for c in cen2]
    nf = len(cen6)
    rows = [nl + comp * nf + k for comp in (0, 1) for k in pick]
    Cw = C.copy()
    Cw[:nl, nl:] = Cw_full[:nl][:, rows]
    good = z2(C, (slice(None), slice(None)))
    good_x, bad_x = z2(C, cross), z2(Cw, cross)
    print(good, good_x, bad_x)
    assert good < 2.5 and good_x < 2.5
    assert bad_x > 4 * good_x


@pytest.mark.parametrize("H", [0.0, 90e3])
def test_coarse_projection_columns_are_sums_of_fine_columns(H):
    # the same telescoping on the projection side: each coarse slope's column
    # of Sigma_phi_s (Eq. covIterative2) is the sum of the three fine columns
    # along its centre line, for every target phase point
    base = small_cfg(n=12, n_gs=1, lgs=H > 0, D=4.0, obstruction=0.0, targets=((5e-5, -2e-5),))
    g = tuple(base["gs"][0])
    cfg = dict(base, gs=[g, g], gs_n=[12, 4], noise_sigma=[0.1, 0.1])
    F = cov.cos_exact(cfg, 0)
    fine = geo.subaperture_mask(12, 0.0)
    coarse = geo.subaperture_mask(4, 0.0)
    fidx = -np.ones((12, 12), dtype=np.int64)
    fidx[fine] = np.arange(fine.sum())
    nvf, nvc = int(fine.sum()), int(coarse.sum())
    scale = np.abs(F).max()
    checked = 0
    for e, (i, j) in enumerate(geo.valid_list(coarse)):
        for comp in (0, 1):
            cells = [(3 * i + 1, 3 * j + k) for k in range(3)] if comp == 0 else \
                [(3 * i + k, 3 * j + 1) for k in range(3)]
            if any(not fine[c] for c in cells):
                continue
            want = sum(F[:, comp * nvf + fidx[c]] for c in cells)
            assert np.abs(F[:, 2 * nvf + comp * nvc + e] - want).max() <= 1e-12 * scale
            checked += 1
    assert checked >= 16
