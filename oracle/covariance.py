"""Dense covariance matrices from point covariances (oracle; test infrastructure only).

Measurement model: Hudgin-like two-point slopes (Appendix A.2).  The x-slope of
the subaperture centred at c is the phase difference phi(c + d/2 x) - phi(c - d/2 x),
the y-slope the same along y.  The lambda/(2 pi d) factor of the paper is
dropped: slopes are phase differences in radians, which leaves the
reconstructed phase unchanged (it cancels in Sigma_phi_s Sigma_ss^{-1}).

Layered turbulence and the cone effect (Sec. 2 intro and Sec. 2.D, the
paragraph on LGS sampling): the ray from guide star g (direction alpha_g,
altitude H_g, H_g = 0 meaning a natural star at infinity) to pupil point p
crosses layer k (altitude h_k) at  gamma_gk * p + h_k * alpha_g  with
gamma_gk = 1 - h_k / H_g (1 for a natural star).  A target direction beta at
infinity maps p to p + h_k * beta.  Layers are statistically independent, so

    Sigma_ss[a, b] = sum_k sum_{u in a} sum_{v in b} w_u w_v B_k(|pos_k(u) - pos_k(v)|)

with w = +1 / -1 for the two points of a slope, and likewise one phase point
against one slope for Sigma_phi_s.  Entries are formed directly from these
coordinates; nothing assumes the Toeplitz structure (Sec. 2.D) that the tests
check for.

Vector layout (Sec. 2.D, Eq. for Sigma_{s_i s_j}): guide stars in order, each
as [x-slopes over valid subapertures ; y-slopes over valid subapertures],
subapertures in row-major order.

Guide stars may sample the pupil on grids of their own (the uneven MOAO
system of natural stars on 10 x 10 grids beside laser stars on 74 x 74,
Sec. 2.D: blocks between stars of different grids or altitudes are not
Toeplitz): cfg["gs_n"] lists the subapertures across the pupil of each guide
star (default cfg["n"] for all).  The point-covariance sum above is the same
for any mix; only the slope points change.
"""

import math

import numpy as np

from . import geometry as geo
from . import turbulence as turb


def _gs(cfg):
    return [(float(ax), float(ay), float(h)) for (ax, ay, h) in cfg["gs"]]


def gs_grid(cfg, g):
    """Subapertures across the pupil of guide star g (cfg["gs_n"], else cfg["n"])."""
    return int(cfg.get("gs_n", [cfg["n"]] * len(cfg["gs"]))[g])


def uniform_grid(cfg):
    """True if every guide star samples the pupil on the cfg["n"] grid."""
    return all(gs_grid(cfg, g) == cfg["n"] for g in range(len(cfg["gs"])))


def cone_factor(H, h):
    """gamma = 1 - h/H for a laser star at altitude H, 1 for a natural star (H = 0)."""
    return 1.0 if H == 0.0 else 1.0 - h / H


def slope_points(cfg):
    """Per-slope pupil points and weights of the slope model.

    Hudgin-like (default, cfg["slope_model"] == "hudgin"; Appendix A.2): the
    difference of the phase at the midpoints of the two edges across the
    slope's direction, phi(c + d/2 e) - phi(c - d/2 e).  Fried: the mean of
    that difference along the two other edges, i.e. over the four corners,
    1/2 [phi(c + d/2 (e + f)) - phi(c - d/2 (e - f)) + phi(c + d/2 (e - f)) - phi(c - d/2 (e + f))]
    with f the other axis (Appendix A: the Fried geometry on the corners).

    Returns (pts, w, gsidx): pts (N, K, 2) = [slope][point][x|y] in metres
    (K = 2 Hudgin, 4 Fried), w (N, K) the weights, gsidx (N,) the guide-star
    index of each slope.
    """
    D, eps = cfg["D"], cfg["obstruction"]
    pts, w, gi = [], [], []
    for g in range(len(cfg["gs"])):
        n = gs_grid(cfg, g)
        d = D / n
        c = geo.subaperture_centres(n, D, eps)
        for comp in (0, 1):
            off, wt = slope_stencil(cfg, comp, d)
            for cc in c:
                pts.append([cc + o for o in off])
                w.append(list(wt))
                gi.append(g)
    return np.array(pts), np.array(w), np.array(gi, dtype=np.int64)


def slope_stencil(cfg, comp, d):
    """Offsets from the subaperture centre and weights of the points of one
    slope component (0 = x, 1 = y) in the configuration's slope model."""
    e = np.zeros(2)
    e[comp] = d / 2.0
    f = np.zeros(2)
    f[1 - comp] = d / 2.0
    if cfg.get("slope_model", "hudgin") == "fried":
        return [e + f, -e + f, e - f, -e - f], (0.5, -0.5, 0.5, -0.5)
    return [e, -e], (1.0, -1.0)


def _layer_positions(cfg, pts, gsidx, k):
    """Positions at layer k of the slope points: gamma * p + h_k * alpha."""
    h, _ = cfg["layers"][k]
    gs = _gs(cfg)
    gam = np.array([cone_factor(gs[g][2], h) for g in gsidx])
    alpha = np.array([[gs[g][0], gs[g][1]] for g in gsidx])
    return gam[:, None, None] * pts + h * alpha[:, None, :]


def css_block(cfg, rows, cols):
    """The entries (rows x cols) of the noiseless Sigma_ss (FP64), shape
    (len(rows), len(cols)): the point-covariance sum above for those slopes."""
    pts, w, gsidx = slope_points(cfg)
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    out = np.zeros((len(rows), len(cols)))
    for k, (h, frac) in enumerate(cfg["layers"]):
        r0k = turb.layer_r0(cfg["r0"], frac)
        pos = _layer_positions(cfg, pts, gsidx, k)
        K = pts.shape[1]
        for u in range(K):
            for v in range(K):
                diff = pos[rows, u][:, None, :] - pos[cols, v][None, :, :]
                rho = np.sqrt(diff[..., 0] ** 2 + diff[..., 1] ** 2)
                out += (w[rows, u][:, None] * w[cols, v][None, :]) * turb.vk_covariance(rho, r0k, cfg["L0"])
    return out


def css_rows(cfg, rows):
    """Rows ``rows`` of the noiseless Sigma_ss (FP64), shape (len(rows), N)."""
    return css_block(cfg, rows, np.arange(slope_points(cfg)[0].shape[0]))


def css_dense(cfg, block=512):
    """Full noiseless Sigma_ss (FP64), built in row blocks."""
    N = slope_points(cfg)[0].shape[0]
    out = np.empty((N, N))
    for r0 in range(0, N, block):
        rows = np.arange(r0, min(N, r0 + block))
        out[rows] = css_rows(cfg, rows)
    return out


def noise_variance(cfg):
    """Diagonal of Sigma_eta_eta: sigma_g^2 on every slope of guide star g (Sec. 2.B)."""
    _, _, gsidx = slope_points(cfg)
    sig = np.asarray(cfg["noise_sigma"], dtype=np.float64)
    return sig[gsidx] ** 2


def add_noise(A, cfg, scale=1.0):
    """A += scale * Sigma_eta_eta on valid slopes, in place.

    Without ``cfg["noise_cov"]`` the noise is white per guide star: the
    diagonal sigma_g^2 (Sec. 2.B).  With it (elongated laser spots, Sec. 2.F)
    Sigma_eta_eta is block diagonal with one 2 x 2 block per subaperture:
    ``noise_cov[g][i][j] = (s_xx, s_yy, s_xy)`` is the covariance of the x- and
    y-slope noise of subaperture (i, j) of guide star g, whose two slopes sit at
    rows off_g + e and off_g + n_valid + e (e its row-major valid index)."""
    C = cfg.get("noise_cov")
    if C is None:
        A[np.diag_indices_from(A)] += scale * noise_variance(cfg)
        return A
    if not uniform_grid(cfg):
        raise NotImplementedError("elongated-spot noise blocks need one grid for all guide stars")
    C = np.asarray(C, dtype=np.float64)
    valid = geo.valid_list(geo.subaperture_mask(cfg["n"], cfg["obstruction"]))
    nv = len(valid)
    for g in range(len(cfg["gs"])):
        for e, (i, j) in enumerate(valid):
            sxx, syy, sxy = C[g, i, j]
            ix = 2 * g * nv + e
            iy = ix + nv
            A[ix, ix] += scale * sxx
            A[iy, iy] += scale * syy
            A[ix, iy] += scale * sxy
            A[iy, ix] += scale * sxy
    return A


def noise_matrix(cfg):
    """Dense Sigma_eta_eta on valid slopes (see add_noise)."""
    N = len(noise_variance(cfg))
    return add_noise(np.zeros((N, N)), cfg)


def system_matrix(cfg):
    """A = W_s (Sigma_ss + Sigma_eta_eta) W_s^T on valid slopes (Eq. SAap1)."""
    return add_noise(css_dense(cfg), cfg)


def system_matrix_r0(cfg, r0, noise_scale=1.0):
    """A of a frame seen with Fried parameter r0 (same Cn^2 fractions): Sigma_ss
    formed at that r0 from the point covariances, plus noise_scale times the
    configuration's noise variance (Eq. SAap1 for that frame)."""
    return add_noise(css_dense(dict(cfg, r0=float(r0))), cfg, float(noise_scale))


def cos_exact(cfg, target):
    """Sigma_phi_beta_s on valid phase points x valid slopes (FP64), Eq. covIterative2.

    Target phase point q at layer k sits at q + h_k * beta.
    """
    bx, by = cfg["targets"][target]
    q = geo.phase_points(cfg["n"], cfg["D"], cfg["obstruction"])
    pts, w, gsidx = slope_points(cfg)
    out = np.zeros((len(q), len(pts)))
    for k, (h, frac) in enumerate(cfg["layers"]):
        r0k = turb.layer_r0(cfg["r0"], frac)
        pos = _layer_positions(cfg, pts, gsidx, k)
        qk = q + h * np.array([bx, by])
        for v in range(pts.shape[1]):
            diff = qk[:, None, :] - pos[None, :, v, :]
            rho = np.sqrt(diff[..., 0] ** 2 + diff[..., 1] ** 2)
            out += w[None, :, v] * turb.vk_covariance(rho, r0k, cfg["L0"])
    return out


def new_grid_size(cfg):
    """n' of the common new phase grid (Sec. 2.D / 2.E, LGS Sigma_phi_s).

    The grid of layer k has spacing d_k = gamma_k d and must cover the n + 1
    target phase points spaced d, so n' >= n d / d_k + 1; one n' is shared by
    all layers and set by the smallest gamma (highest layer).  For natural
    stars gamma = 1 and n' = n + 1, the phase grid itself.
    """
    gs = _gs(cfg)
    gmin = 1.0
    for (_, _, H) in gs:
        for (h, _) in cfg["layers"]:
            gmin = min(gmin, cone_factor(H, h))
    return int(math.ceil(cfg["n"] / gmin - 1e-9)) + 1


def _common_cone(cfg, k):
    """gamma_k shared by all guide stars (the interpolated form needs one altitude)."""
    h = cfg["layers"][k][0]
    gams = {cone_factor(H, h) for (_, _, H) in _gs(cfg)}
    if len(gams) != 1:
        raise ValueError("the new-grid Sigma_phi_s needs all guide stars at one altitude")
    return gams.pop()


def new_grid_nodes(cfg, k):
    """Pupil coordinates of the n' x n' nodes of layer k, row-major, spacing gamma_k d,
    centred on the pupil; node (uy, ux) sits at ((ux - (n'-1)/2) d_k, (uy - (n'-1)/2) d_k)."""
    npr = new_grid_size(cfg)
    dk = _common_cone(cfg, k) * cfg["D"] / cfg["n"]
    u = (np.arange(npr) - (npr - 1) / 2.0) * dk
    uy, ux = np.meshgrid(u, u, indexing="ij")
    return np.stack([ux.ravel(), uy.ravel()], axis=1)


def bilinear_weights(cfg, k):
    """I'_k as a dense (n_vphi, n'^2) matrix of bilinear weights (Eq. interp)."""
    npr = new_grid_size(cfg)
    dk = _common_cone(cfg, k) * cfg["D"] / cfg["n"]
    q = geo.phase_points(cfg["n"], cfg["D"], cfg["obstruction"])
    I = np.zeros((len(q), npr * npr))
    for a, (x, y) in enumerate(q):
        tx = x / dk + (npr - 1) / 2.0
        ty = y / dk + (npr - 1) / 2.0
        ix = min(max(int(math.floor(tx)), 0), npr - 2)
        iy = min(max(int(math.floor(ty)), 0), npr - 2)
        fx, fy = tx - ix, ty - iy
        I[a, iy * npr + ix] += (1 - fx) * (1 - fy)
        I[a, iy * npr + ix + 1] += fx * (1 - fy)
        I[a, (iy + 1) * npr + ix] += (1 - fx) * fy
        I[a, (iy + 1) * npr + ix + 1] += fx * fy
    return I


def cos_new_grid_layer(cfg, target, k):
    """Xi'_k: covariance of layer k's target phase on the new grid with all slopes."""
    bx, by = cfg["targets"][target]
    h, frac = cfg["layers"][k]
    r0k = turb.layer_r0(cfg["r0"], frac)
    nodes = new_grid_nodes(cfg, k) + h * np.array([bx, by])
    pts, w, gsidx = slope_points(cfg)
    pos = _layer_positions(cfg, pts, gsidx, k)
    out = np.zeros((len(nodes), len(pts)))
    for v in range(pts.shape[1]):
        diff = nodes[:, None, :] - pos[None, :, v, :]
        rho = np.sqrt(diff[..., 0] ** 2 + diff[..., 1] ** 2)
        out += w[None, :, v] * turb.vk_covariance(rho, r0k, cfg["L0"])
    return out


def cos_interp(cfg, target):
    """Sigma_phi_beta_s = sum_k I'_k Xi'_k (Sec. 2.D, Eq. interp and the sum over layers)."""
    out = None
    for k in range(len(cfg["layers"])):
        term = bilinear_weights(cfg, k) @ cos_new_grid_layer(cfg, target, k)
        out = term if out is None else out + term
    return out


def cos_interp_rows(cfg, target, rows):
    """Rows ``rows`` (valid phase-point indices) of cos_interp, computing only the
    grid nodes those rows interpolate from (same definition, restricted)."""
    rows = np.asarray(rows, dtype=np.int64)
    npr = new_grid_size(cfg)
    bx, by = cfg["targets"][target]
    pts, w, gsidx = slope_points(cfg)
    out = np.zeros((len(rows), len(pts)))
    for k, (h, frac) in enumerate(cfg["layers"]):
        I = bilinear_weights(cfg, k)[rows]
        used = np.nonzero(np.abs(I).sum(axis=0))[0]
        nodes = new_grid_nodes(cfg, k)[used] + h * np.array([bx, by])
        r0k = turb.layer_r0(cfg["r0"], frac)
        pos = _layer_positions(cfg, pts, gsidx, k)
        X = np.zeros((len(used), len(pts)))
        for v in range(pts.shape[1]):
            diff = nodes[:, None, :] - pos[None, :, v, :]
            rho = np.sqrt(diff[..., 0] ** 2 + diff[..., 1] ** 2)
            X += w[None, :, v] * turb.vk_covariance(rho, r0k, cfg["L0"])
        out += I[:, used] @ X
    return out
