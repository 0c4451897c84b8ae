"""Seeded synthetic workloads: system configurations and slope frames.

This module is the one place that serves both the CUDA path and the CPU
oracle with inputs.  It holds no reconstructor arithmetic: it describes
systems as plain numbers and simulates Shack-Hartmann measurements of
synthetic von Karman phase screens (the paper measures on OOMAO simulations,
which are not available; these frames stand in for them).

Configurations (angles in radians, lengths in metres, r0 at 500 nm):

* ``ngs8m``    -- 8 m pupil, no obstruction, 20 x 20 subapertures, 3 natural
  guide stars on a 30" ring (0, 120, 240 deg), target on axis; layers
  (0 km, 0.7), (8 km, 0.3); r0 = 0.15 m, L0 = 25 m; noise 5 % of slope rms.
* ``elt_ltao`` -- 39 m pupil, 28 % obstruction, 74 x 74 subapertures, 6 laser
  guide stars at 90 km on a 60"-diameter ring, target on axis; 9 layers from 0
  to 20 km (a declared synthetic profile: the paper prints its profile only in
  a figure); r0 = 0.129 m, L0 = 25 m; noise 3 % of slope rms.
* ``lgs_mid``  -- the ``elt_ltao`` system shrunk to 16 x 16 subapertures of the
  same size (8.43 m pupil), for tests the dense oracle finishes in seconds.
* ``elt_moao`` -- the ``elt_ltao`` system with 32 target directions drawn
  uniformly within a 7'-diameter field (seeded, seed 4): the laser-star part
  of a batched MOAO system.

Slope frames: per layer a periodic FFT phase screen with the von Karman PSD
0.0228956 r0^{-5/3} (f^2 + 1/L0^2)^{-11/6} (Appendix A.1; the paper prints the
constant rounded), pixel d/2, 512 pixels.  Rays from each guide star are traced
to each layer with the cone factor 1 - h/H of laser stars; the x-slope of a
subaperture is the trapezoid mean of the phase along its right edge minus that
along its left edge (= d times the subaperture-averaged gradient), likewise in
y.  Gaussian noise of standard deviation ``noise_frac`` times the rms of the
noiseless slopes is added.  Every screen and noise draw comes from numpy's
counter-based Philox generator keyed by (seed, frame, layer), so a frame does
not depend on how many frames are generated with it.

Time sequences (``slope_sequence``): frozen flow, each layer's screen moves
rigidly with its wind vector, so step t samples the screen at x - v t dt; the
screens of a sequence are drawn once, the noise anew at every step.  The wind
profile is synthetic as well (the paper gives none).

Elongated laser spots (``elongated_noise``, Sec. 2.F): a synthetic side-launch
model.  The launch telescope of laser star g sits at radius 0.55 D on the star's
azimuth; a subaperture at pupil position p sees the spot stretched along
u = (p - launch) / |p - launch|, so its slope noise covariance is
sigma^2 (I + (k |p - launch| / D)^2 u u^T) with k the elongation at one
pupil diameter.  Natural stars (H = 0) keep sigma^2 I.

Slopes are returned on the full n x n subaperture grid,
``[frame][gs][x|y][i][j]``; callers select the valid subapertures with the mask
of the side they exercise.
"""

import math

import numpy as np

ARCSEC = math.pi / (180.0 * 3600.0)

NINE_LAYER_H = [0.0, 500.0, 1000.0, 2000.0, 4000.0, 8000.0, 12000.0, 16000.0, 20000.0]
NINE_LAYER_FRAC = [0.40, 0.12, 0.10, 0.09, 0.08, 0.07, 0.06, 0.05, 0.03]
# synthetic frozen-flow wind per layer: speed [m/s], direction [rad]
NINE_LAYER_WIND = [(10.0, 0.0), (8.0, 0.8), (9.0, 1.6), (12.0, 2.4), (15.0, 3.2), (20.0, 4.0), (25.0, 4.8),
                   (18.0, 5.6), (12.0, 0.4)]


def ring(n_gs, radius, height, phase0=0.0):
    """Guide stars evenly spaced on a ring, the first on +x: (ax, ay, H)."""
    return [(radius * math.cos(phase0 + 2 * math.pi * j / n_gs),
             radius * math.sin(phase0 + 2 * math.pi * j / n_gs), height) for j in range(n_gs)]


def config(name):
    """Plain-number system description (see module docstring)."""
    if name == "ngs8m":
        return dict(name=name, D=8.0, obstruction=0.0, n=20, r0=0.15, L0=25.0,
                    layers=[(0.0, 0.7), (8000.0, 0.3)],
                    gs=ring(3, 30 * ARCSEC, 0.0), targets=[(0.0, 0.0)], noise_frac=0.05)
    if name == "elt_ltao":
        return dict(name=name, D=39.0, obstruction=0.28, n=74, r0=0.129, L0=25.0,
                    layers=list(zip(NINE_LAYER_H, NINE_LAYER_FRAC)),
                    gs=ring(6, 30 * ARCSEC, 90e3), targets=[(0.0, 0.0)], noise_frac=0.03)
    if name == "elt_moao":
        cfg = config("elt_ltao")
        rng = np.random.default_rng(4)
        rad = 3.5 * 60 * ARCSEC * np.sqrt(rng.random(32))
        ang = 2 * math.pi * rng.random(32)
        cfg.update(name=name, targets=[(float(r * math.cos(a)), float(r * math.sin(a))) for r, a in zip(rad, ang)])
        return cfg
    if name == "lgs_mid":
        return dict(name=name, D=16 * 39.0 / 74, obstruction=0.28, n=16, r0=0.129, L0=25.0,
                    layers=list(zip(NINE_LAYER_H, NINE_LAYER_FRAC)),
                    gs=ring(6, 30 * ARCSEC, 90e3), targets=[(0.0, 0.0)], noise_frac=0.03)
    raise KeyError(name)


def _rng(seed, frame, stream):
    return np.random.Generator(np.random.Philox(key=[seed, 1_000_003 * frame + stream]))


def screen_pair(rng, N, pix, r0, L0):
    """Two independent periodic von Karman screens (N x N, pixel ``pix``)."""
    f = np.fft.fftfreq(N, d=pix)
    fx, fy = np.meshgrid(f, f, indexing="xy")
    psd = 0.0228956 * r0 ** (-5.0 / 3.0) * (fx * fx + fy * fy + 1.0 / L0 ** 2) ** (-11.0 / 6.0)
    psd[0, 0] = 0.0
    df = 1.0 / (N * pix)
    amp = np.sqrt(psd) * df
    z = (rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))) * amp
    scr = np.fft.fft2(z)
    return scr.real, scr.imag


def bilinear(scr, pix, x, y):
    N = scr.shape[0]
    tx = x / pix + N / 2.0
    ty = y / pix + N / 2.0
    ix = np.floor(tx).astype(np.int64)
    iy = np.floor(ty).astype(np.int64)
    fx, fy = tx - ix, ty - iy
    ix %= N
    iy %= N
    ix1, iy1 = (ix + 1) % N, (iy + 1) % N
    return ((1 - fx) * (1 - fy) * scr[iy, ix] + fx * (1 - fy) * scr[iy, ix1]
            + (1 - fx) * fy * scr[iy1, ix] + fx * fy * scr[iy1, ix1])


def _screens(cfg, seed, f, screen_px):
    """The layer screens of frame (or sequence) ``f``: [(h, frac, screen)]."""
    pix = cfg["D"] / cfg["n"] / 2.0
    screens = []
    rng = _rng(seed, f, 0)
    for k in range(0, len(cfg["layers"]), 2):
        pair = cfg["layers"][k:k + 2]
        # one complex draw gives independent screens for layers k and k+1
        a, b = screen_pair(rng, screen_px, pix, cfg["r0"], cfg["L0"])
        for idx, (h, frac) in enumerate(pair):
            screens.append((h, frac, a if idx == 0 else b))
    return screens


def _clean_frame(cfg, seed, f, screen_px, grids, shifts=None):
    """Noiseless slopes [gs][x|y][n][n] of frame ``f``; shifts[k] = (dx, dy)
    moves layer k's screen by that many metres (frozen flow)."""
    return _sample(cfg, _screens(cfg, seed, f, screen_px), grids, shifts)


def _sample(cfg, screens, grids, shifts=None, stars=None):
    """Noiseless slopes [gs][x|y][n][n] on ``grids`` (stars: the guide-star
    indices to sample, default all; the screens' pixel is D / cfg["n"] / 2)."""
    D = cfg["D"]
    pix = D / cfg["n"] / 2.0
    (cx, cy), (vx, vy), (hx, hy) = grids
    stars = range(len(cfg["gs"])) if stars is None else stars
    n = vx.shape[0]
    out = np.zeros((len(stars), 2, n, n))
    for o, g in enumerate(stars):
        ax, ay, H = cfg["gs"][g]
        pc = np.zeros_like(cx)
        pv = np.zeros_like(vx)
        ph = np.zeros_like(hx)
        for k, (h, frac, scr) in enumerate(screens):
            gam = 1.0 if H == 0.0 else 1.0 - h / H
            s = math.sqrt(frac)                   # layer amplitude: r0_k^{-5/6} = frac^{1/2} r0^{-5/6}
            ox = h * ax - (shifts[k][0] if shifts is not None else 0.0)
            oy = h * ay - (shifts[k][1] if shifts is not None else 0.0)
            pc += s * bilinear(scr, pix, gam * cx + ox, gam * cy + oy)
            pv += s * bilinear(scr, pix, gam * vx + ox, gam * vy + oy)
            ph += s * bilinear(scr, pix, gam * hx + ox, gam * hy + oy)
        # edge means by the trapezoid rule over corner, midpoint, corner
        right = (pc[:-1, 1:] + 2.0 * pv[:, 1:] + pc[1:, 1:]) / 4.0
        left = (pc[:-1, :-1] + 2.0 * pv[:, :-1] + pc[1:, :-1]) / 4.0
        top = (pc[1:, :-1] + 2.0 * ph[1:, :] + pc[1:, 1:]) / 4.0
        bottom = (pc[:-1, :-1] + 2.0 * ph[:-1, :] + pc[:-1, 1:]) / 4.0
        out[o, 0] = right - left
        out[o, 1] = top - bottom
    return out


N_CALIBRATION_FRAMES = 4


def slope_frames(cfg, n_frames, seed=0, screen_px=512, first=0):
    """Noisy slopes [frame][gs][x|y][n][n] (float64) of frames first .. first+n_frames-1
    and the per-GS noise sigma.

    Returns (slopes, noise_sigma): noise_sigma[g] = noise_frac * rms of the
    noiseless slopes of guide star g over frames 0..3 of ``seed`` (always the
    same frames, whatever ``n_frames`` and ``first`` are).
    """
    n, D = cfg["n"], cfg["D"]
    d = D / n
    e = (np.arange(n + 1) - n / 2.0) * d          # corner coordinates
    m = (np.arange(n) + 0.5 - n / 2.0) * d        # centre coordinates
    cy, cx = np.meshgrid(e, e, indexing="ij")     # (n+1, n+1) corners
    vy, vx = np.meshgrid(m, e, indexing="ij")     # (n, n+1) midpoints of vertical edges
    hy, hx = np.meshgrid(e, m, indexing="ij")     # (n+1, n) midpoints of horizontal edges
    grids = ((cx, cy), (vx, vy), (hx, hy))
    n_gs = len(cfg["gs"])
    calib = np.stack([_clean_frame(cfg, seed, f, screen_px, grids) for f in range(N_CALIBRATION_FRAMES)])
    sigma = cfg["noise_frac"] * np.sqrt(np.mean(calib ** 2, axis=(0, 2, 3, 4)))
    noisy = np.zeros((n_frames, n_gs, 2, n, n))
    for i in range(n_frames):
        f = first + i
        noisy[i] = calib[f] if f < N_CALIBRATION_FRAMES else _clean_frame(cfg, seed, f, screen_px, grids)
        rng = _rng(seed, f, 999)
        noisy[i] += sigma[:, None, None, None] * rng.standard_normal((n_gs, 2, n, n))
    return noisy, sigma


def _grids(cfg, n=None):
    n, D = (cfg["n"] if n is None else n), cfg["D"]
    d = D / n
    e = (np.arange(n + 1) - n / 2.0) * d
    m = (np.arange(n) + 0.5 - n / 2.0) * d
    cy, cx = np.meshgrid(e, e, indexing="ij")
    vy, vx = np.meshgrid(m, e, indexing="ij")
    hy, hx = np.meshgrid(e, m, indexing="ij")
    return ((cx, cy), (vx, vy), (hx, hy))


def slope_frames_mixed(cfg, n_frames, seed=0, screen_px=512):
    """Noisy valid slopes [frame][N] (float64) in the solver's vector layout
    for guide stars on grids of their own (cfg["gs_n"]: subapertures across
    the pupil per star, default cfg["n"]; cfg["n"] sets the screens' pixel,
    so it should be the finest grid), and the per-star noise sigma.

    The same screens and recipe as slope_frames: each star samples its own
    grid's edge midpoints and corners; sigma[g] = noise_frac * rms of star g's
    noiseless slopes over frames 0..3; the noise of frame f is drawn from the
    same stream, star after star.  With one grid for all stars the result is
    slope_frames' valid slopes, number for number.
    """
    D, eps, n_gs = cfg["D"], cfg["obstruction"], len(cfg["gs"])
    gs_n = [int(x) for x in cfg.get("gs_n", [cfg["n"]] * n_gs)]
    grids = {n: _grids(cfg, n) for n in set(gs_n)}

    def clean(f):
        scr = _screens(cfg, seed, f, screen_px)
        return [_sample(cfg, scr, grids[gs_n[g]], stars=[g])[0] for g in range(n_gs)]

    calib = [clean(f) for f in range(N_CALIBRATION_FRAMES)]
    sigma = np.array([cfg["noise_frac"] * np.sqrt(np.mean([c[g] ** 2 for c in calib])) for g in range(n_gs)])
    masks = [_subaperture_mask(gs_n[g], eps) for g in range(n_gs)]
    out = []
    for f in range(n_frames):
        sl = calib[f] if f < N_CALIBRATION_FRAMES else clean(f)
        rng = _rng(seed, f, 999)
        vec = []
        for g in range(n_gs):
            noisy = sl[g] + sigma[g] * rng.standard_normal((2, gs_n[g], gs_n[g]))
            vec += [noisy[0][masks[g]], noisy[1][masks[g]]]
        out.append(np.concatenate(vec))
    return np.array(out), sigma


def _subaperture_mask(n, obstruction):
    """Valid subapertures: centre inside the annular pupil (row-major order)."""
    j = np.arange(n)
    q = (2 * j[None, :] + 1 - n) ** 2 + (2 * j[:, None] + 1 - n) ** 2
    return (q <= n * n) & (q >= (obstruction * n) ** 2)


def wind(cfg):
    """Per-layer wind vectors [(vx, vy)] in m/s (the synthetic profile for 9
    layers, 10 m/s along +x otherwise)."""
    if len(cfg["layers"]) == len(NINE_LAYER_WIND):
        return [(v * math.cos(a), v * math.sin(a)) for v, a in NINE_LAYER_WIND]
    return [(10.0, 0.0)] * len(cfg["layers"])


def slope_sequence(cfg, n_seq, n_steps, seed=0, dt=1e-3, screen_px=512, first=0):
    """Frozen-flow time sequences: noisy slopes [step][sequence][gs][x|y][n][n]
    of sequences first .. first+n_seq-1 at times t dt, t = 0 .. n_steps-1, and the
    per-GS noise sigma (the same calibration as slope_frames).  Sequence j uses
    the screens of frame j of ``seed``; step t's noise is drawn from stream
    1000 + t of that frame."""
    grids = _grids(cfg)
    n_gs = len(cfg["gs"])
    calib = np.stack([_clean_frame(cfg, seed, f, screen_px, grids) for f in range(N_CALIBRATION_FRAMES)])
    sigma = cfg["noise_frac"] * np.sqrt(np.mean(calib ** 2, axis=(0, 2, 3, 4)))
    v = wind(cfg)
    n = cfg["n"]
    out = np.zeros((n_steps, n_seq, n_gs, 2, n, n))
    for j in range(n_seq):
        screens = _screens(cfg, seed, first + j, screen_px)
        for t in range(n_steps):
            shifts = [(vx * t * dt, vy * t * dt) for vx, vy in v]
            out[t, j] = _sample(cfg, screens, grids, shifts)
            rng = _rng(seed, first + j, 1000 + t)
            out[t, j] += sigma[:, None, None, None] * rng.standard_normal((n_gs, 2, n, n))
    return out, sigma


def _sequence_job(args):
    cfg, n_seq, n_steps, seed, dt, first = args
    return slope_sequence(cfg, n_seq, n_steps, seed=seed, dt=dt, first=first)


def slope_sequence_parallel(cfg, n_seq, n_steps, seed=0, dt=1e-3, workers=None, chunk=4):
    """slope_sequence on a pool of `spawn` worker processes (identical result)."""
    import multiprocessing as mp
    import os
    from concurrent.futures import ProcessPoolExecutor
    workers = workers or min(32, os.cpu_count() or 1)
    jobs = [(cfg, min(chunk, n_seq - a), n_steps, seed, dt, a) for a in range(0, n_seq, chunk)]
    if workers <= 1 or len(jobs) <= 1:
        return slope_sequence(cfg, n_seq, n_steps, seed=seed, dt=dt)
    with ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn")) as ex:
        parts = list(ex.map(_sequence_job, jobs))
    return np.concatenate([p[0] for p in parts], axis=1), parts[0][1]


def _frames_job(args):
    cfg, n_frames, seed, first = args
    return slope_frames(cfg, n_frames, seed=seed, first=first)


def slope_frames_parallel(cfg, n_frames, seed=0, workers=None, chunk=8):
    """slope_frames on a pool of `spawn` worker processes (identical result)."""
    import multiprocessing as mp
    import os
    from concurrent.futures import ProcessPoolExecutor
    workers = workers or min(32, os.cpu_count() or 1)
    jobs = [(cfg, min(chunk, n_frames - a), seed, a) for a in range(0, n_frames, chunk)]
    if workers <= 1 or len(jobs) <= 1:
        return slope_frames(cfg, n_frames, seed=seed)
    with ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn")) as ex:
        parts = list(ex.map(_frames_job, jobs))
    return np.concatenate([p[0] for p in parts]), parts[0][1]


def elongated_noise(cfg, sigma, k=2.0):
    """Per-subaperture 2 x 2 slope noise covariances [n_gs][n][n][3] (s_xx, s_yy,
    s_xy) of the side-launch elongation model above; ``sigma`` is one value or
    one per guide star."""
    n, D = cfg["n"], cfg["D"]
    d = D / n
    sig = np.broadcast_to(np.asarray(sigma, dtype=np.float64), (len(cfg["gs"]),))
    c = (np.arange(n) + 0.5) * d - D / 2
    Y, X = np.meshgrid(c, c, indexing="ij")
    out = np.zeros((len(cfg["gs"]), n, n, 3))
    for g, (ax, ay, H) in enumerate(cfg["gs"]):
        s2 = sig[g] ** 2
        out[g, :, :, 0] = s2
        out[g, :, :, 1] = s2
        if H <= 0:
            continue
        th = math.atan2(ay, ax)
        vx, vy = X - 0.55 * D * math.cos(th), Y - 0.55 * D * math.sin(th)
        e2 = (k / D) ** 2                                  # (k |v| / D)^2 u u^T = e2 v v^T
        out[g, :, :, 0] += s2 * e2 * vx * vx
        out[g, :, :, 1] += s2 * e2 * vy * vy
        out[g, :, :, 2] = s2 * e2 * vx * vy
    return out


def warm_start_init(n_planes, hidden, seed, last_gain=0.1, cin=None):
    """Seeded He-normal initial parameters of the warm-start network (flat FP32,
    per layer W [Cout][Cin][3][3] then b [Cout]); the last layer scaled by
    last_gain; cin: input channels when they differ from n_planes (the
    network on [r, M r] has 2 n_planes)."""
    rng = np.random.default_rng(seed)
    ch = [n_planes if cin is None else cin, hidden, hidden, hidden, n_planes]
    out = []
    for l in range(4):
        co, ci = ch[l + 1], ch[l]
        W = rng.standard_normal((co, ci, 3, 3)) * np.sqrt(2.0 / (9 * ci))
        if l == 3:
            W *= last_gain
        out += [W.ravel(), 0.01 * rng.standard_normal(co)]
    return np.concatenate(out).astype(np.float32)
