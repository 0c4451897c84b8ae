"""The seeded input generator (shared by both sides; no reconstructor arithmetic)."""
import numpy as np

from paper_1806_07938_gb300 import workloads as W


def small():
    return dict(W.config("lgs_mid"), n=8, D=8 * 39.0 / 74)


def test_sequence_step0_is_the_frame_and_noise_is_fresh():
    cfg = small()
    grids = W._grids(cfg)
    seq, sig = W.slope_sequence(cfg, 2, 3, seed=4, dt=0.0)
    _, sig_f = W.slope_frames(cfg, 1, seed=4)
    assert np.array_equal(sig, sig_f)
    for j in range(2):
        clean = W._clean_frame(cfg, 4, j, 512, grids)
        for t in range(3):
            # dt = 0: every step sees the same screens; only the noise differs
            resid = (seq[t, j] - clean) / sig[:, None, None, None]
            assert abs(resid.std() - 1.0) < 0.15
        assert not np.array_equal(seq[0, j], seq[1, j])


def test_sequence_frozen_flow_moves_the_screens():
    cfg = small()
    a, _ = W.slope_sequence(cfg, 1, 2, seed=4, dt=1e-3)
    b, _ = W.slope_sequence(cfg, 1, 2, seed=4, dt=0.05)
    d_small = np.std(a[1] - a[0])
    d_large = np.std(b[1] - b[0])
    assert d_large > 2 * d_small          # 50 ms of wind decorrelates far more than 1 ms
    c, _ = W.slope_sequence(cfg, 1, 2, seed=4, dt=1e-3)
    assert np.array_equal(a, c)           # deterministic


def test_elongated_noise_model():
    # side-launch elongation (Sec. 2.F): sigma^2 (I + (k/D)^2 v v^T), v from the
    # launch point at 0.55 D on the star's azimuth to the subaperture centre
    from paper_1806_07938_gb300 import workloads as W
    cfg = W.config("lgs_mid")
    C = W.elongated_noise(cfg, 0.2, k=2.0)
    n, D = cfg["n"], cfg["D"]
    assert C.shape == (len(cfg["gs"]), n, n, 3)
    sxx, syy, sxy = C[..., 0], C[..., 1], C[..., 2]
    det = sxx * syy - sxy ** 2
    tr = sxx + syy
    # eigenvalues: sigma^2 and sigma^2 (1 + (k |v| / D)^2)
    lo = tr / 2 - np.sqrt((tr / 2) ** 2 - det)
    assert np.allclose(lo, 0.04, rtol=0, atol=1e-12)
    # the long axis points at the launch telescope of each laser star
    for g, (ax, ay, H) in enumerate(cfg["gs"]):
        th = np.arctan2(ay, ax)
        lx, ly = 0.55 * D * np.cos(th), 0.55 * D * np.sin(th)
        c = (np.arange(n) + 0.5) * D / n - D / 2
        vx = c[None, :] - lx
        vy = c[:, None] - ly
        hi = tr[g] - lo[g]
        assert np.allclose(hi, 0.04 * (1 + (2.0 / D) ** 2 * (vx ** 2 + vy ** 2)), rtol=1e-12)
        # (vx, vy) is the eigenvector of the larger eigenvalue
        res_x = (sxx[g] - hi) * vx + sxy[g] * vy
        res_y = sxy[g] * vx + (syy[g] - hi) * vy
        assert np.abs(res_x).max() < 1e-12 and np.abs(res_y).max() < 1e-12
    # natural stars are not elongated
    ngs = W.config("ngs8m")
    Cn = W.elongated_noise(ngs, 0.1, k=3.0)
    assert np.array_equal(Cn[..., 0], np.full(Cn.shape[:3], 0.1 ** 2))
    assert np.array_equal(Cn[..., 2], np.zeros(Cn.shape[:3]))


def test_mixed_grid_frames():
    # guide stars on grids of their own (natural stars on a coarse grid): with
    # one grid for all stars the generator reproduces slope_frames' valid
    # slopes number for number; with mixed grids each star has its own valid
    # count, and its noise level follows its own slopes
    from paper_1806_07938_gb300 import workloads as W
    from oracle import geometry as geo
    cfg = dict(name="mix", D=4.0, obstruction=0.2, n=12, r0=0.15, L0=25.0, layers=[(0.0, 0.6), (8e3, 0.4)],
               gs=W.ring(2, 20 * W.ARCSEC, 90e3) + W.ring(1, 30 * W.ARCSEC, 0.0), targets=[(0.0, 0.0)],
               noise_frac=0.05)
    full, sig = W.slope_frames(cfg, 6, seed=5, screen_px=128)
    mask = geo.subaperture_mask(12, 0.2)
    vec, sig2 = W.slope_frames_mixed(dict(cfg, gs_n=[12, 12, 12]), 6, seed=5, screen_px=128)
    assert np.array_equal(vec, full[..., mask].reshape(6, -1))
    assert np.array_equal(sig, sig2)
    mixed, sig3 = W.slope_frames_mixed(dict(cfg, gs_n=[12, 12, 4]), 6, seed=5, screen_px=128)
    nf, nc = int(mask.sum()), int(geo.subaperture_mask(4, 0.2).sum())
    assert mixed.shape == (6, 2 * 2 * nf + 2 * nc)
    assert np.array_equal(mixed[:, :4 * nf], vec[:, :4 * nf])        # the laser stars are unchanged
    assert np.array_equal(sig3[:2], sig[:2]) and sig3[2] != sig[2]
    assert np.all(np.isfinite(mixed))
